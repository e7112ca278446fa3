"""Accurate-mode scaling on the GPU against the oracle (Sec. III-E).

e', f' and the E4M3 bound operands are integer work: bit-exact.  The bound maxima
R, S come from FP32 tensor-core accumulation, whose order differs from the oracle's
(reading: the oracle rounds the exact product once); both must lie within the
paper's FP32 bound of the exact value.  The exponent rule applied to the GPU's own
R, S must reproduce the GPU's e, f exactly, and e, f agree with the oracle's on
nearly every row / column and by at most 1 elsewhere."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,phi,N", [(256, 256, 256, 0.5, 12), (200, 130, 300, 1.0, 12),
                                         (64, 96, 1000, 2.0, 14), (33, 17, 5, 1.0, 8)])
def test_scales_match_oracle(cuda, m, n, k, phi, N):
    A, B = workloads.problem(m, n, k, phi, seed=m + n)
    A[3] = 0.0
    B[:, 2] = 0.0
    if m > 10:
        A[7, :] *= 1e-310  # subnormal row
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    g = {key: v.cpu().numpy() for key, v in sc.items()}
    r = oz.scaling_exponents(A.numpy(), B.numpy(), N)
    assert np.array_equal(g["eprime"], r["eprime"])
    assert np.array_equal(g["fprime"], r["fprime"])
    assert np.array_equal(g["Abar"][:, :k], r["Abar"])
    assert np.array_equal(g["BbarT"][:, :k], r["Bbar"].T)
    assert np.all(g["Abar"][:, k:] == 0) and np.all(g["BbarT"][:, k:] == 0)
    exact = oz.e4m3_decode_array(r["Abar"]) @ oz.e4m3_decode_array(r["Bbar"])
    bound = (1 + (2 * k + 4) * 2.0**-24)
    Rex, Sex = exact.max(axis=1), exact.max(axis=0)
    # cbar bounds the exact product from above (the purpose of Eq. barCupper) and
    # is within the FP32 summation bound of it
    assert np.all(g["R"] >= Rex) and np.all(g["R"] <= Rex * bound + 1e-30)
    assert np.all(g["S"] >= Sex) and np.all(g["S"] <= Sex * bound + 1e-30)
    # the exponent rule on the GPU's own maxima is bit-exact
    pp, d = r["pprime"], r["delta"]
    zr = ~np.any(A.numpy() != 0, axis=1)
    zc = ~np.any(B.numpy() != 0, axis=0)
    e_from_gpu_R = [oz.final_exponent(g["eprime"][i], g["R"][i], pp, d, zr[i]) for i in range(m)]
    f_from_gpu_S = [oz.final_exponent(g["fprime"][j], g["S"][j], pp, d, zc[j]) for j in range(n)]
    assert list(g["e"]) == e_from_gpu_R
    assert list(g["f"]) == f_from_gpu_S
    agree = (np.sum(g["e"] == r["e"]) + np.sum(g["f"] == r["f"])) / (m + n)
    assert agree >= 0.99
    assert np.max(np.abs(g["e"] - r["e"])) <= 1 and np.max(np.abs(g["f"] - r["f"])) <= 1


@pytest.mark.parametrize("N", [1, 2, 5, 6, 7, 12, 13, 14, 16, 20])
def test_exponent_constant_per_N(cuda, N):
    """P' differs per N; one row and column of ones exercise it through the GPU."""
    A = torch.ones((1, 4), dtype=torch.float64)
    B = torch.ones((4, 1), dtype=torch.float64)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    r = oz.scaling_exponents(A.numpy(), B.numpy(), N)
    assert int(sc["e"][0]) == int(r["e"][0]) and int(sc["f"][0]) == int(r["f"][0])
