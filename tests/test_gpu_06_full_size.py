"""The benchmark's workload (m = n = k = 16384, phi = 1, N = 12; the launch
configuration bench.py times) and the rectangular workloads (4096 x 4096 x 65536,
65536 x 1024 x 1024) checked on sampled outputs: each sampled C_ij is
recomputed by the oracle from row i of A, column j of B and the GPU's exponents
(bit-exact), the Ozaki-II condition is verified exactly for those entries, and the
error against the exact product stays within k 2^-52 (|A||B|)_ij."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,N,samples", [(16384, 16384, 16384, 12, 48), (4096, 4096, 4096, 13, 48),
                                             # the long reduction (two exactness blocks for
                                             # the square moduli) and the tall-skinny shape
                                             (4096, 4096, 65536, 12, 16), (65536, 1024, 1024, 12, 48)])
def test_full_size_sampled(cuda, m, n, k, N, samples):
    A, B = workloads.problem(m, n, k, 1.0, seed=0, device=cuda)
    C = ozk.dgemm(A, B, num_moduli=N)
    sc = ozk.scales(A, B, num_moduli=N)
    torch.cuda.synchronize()
    assert ozk.device_status() == "OZK2_OK"
    rng = np.random.default_rng(m + 3 * k)
    rows = rng.integers(0, m, samples)
    cols = rng.integers(0, n, samples)
    rows[0], cols[0] = m - 1, n - 1
    Ar = A[torch.as_tensor(rows, device=cuda)].cpu().numpy()
    Bc = B[:, torch.as_tensor(cols, device=cuda)].cpu().numpy()
    Cs = C[torch.as_tensor(rows, device=cuda), torch.as_tensor(cols, device=cuda)].cpu().numpy()
    e = sc["e"].cpu().numpy()
    f = sc["f"].cpu().numpy()
    moduli = oz.hybrid_moduli(N)
    for t in range(samples):
        i, j = int(rows[t]), int(cols[t])
        want, cond = oz.emulated_entry(Ar[t], Bc[:, t], e[i], f[j], moduli)
        assert cond, (i, j)
        assert np.float64(want).view(np.uint64) == np.float64(Cs[t]).view(np.uint64), (i, j)
        ex = oz.exact_dot(Ar[t], Bc[:, t])
        ab = oz.exact_abs_dot(Ar[t], Bc[:, t])
        assert abs(float(ex - oz.Fraction(float(Cs[t])))) <= k * 2.0**-52 * float(ab)
