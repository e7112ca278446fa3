"""Long reductions split into exactness blocks (reading R12: k > 2^15 for the square
moduli, whose shared accumulator X = A1 B2 + A2 B1 holds 2^15 terms, and k > 2^16 for
the Karatsuba moduli) on problems with several tile rows and columns, so that every GEMM
CTA of the launch runs multi-block units.  The residue products C'_l and the final C
are compared in full with the oracle given the GPU's exponents: C'_l = mod(A'B', p_l)
(Eq. CRTmatmul) from the oracle's digit planes and digit products, C from the oracle's
CRT and inverse scaling (Eqs. CRT_finalreduction, inversescaling)."""
import numpy as np
import pytest

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,N,phi", [(300, 264, 32769, 12, 1.0), (260, 200, 65537, 14, 1.0),
                                         (384, 136, 70000, 12, 2.0), (257, 300, 70000, 14, 0.5)])
def test_long_reduction_bit_exact(cuda, m, n, k, N, phi):
    A, B = workloads.problem(m, n, k, phi, seed=k + m)
    Ad, Bd = A.to(cuda), B.to(cuda)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    res = ozk.residue_products(Ad, Bd, sc["e"], sc["f"], num_moduli=N).cpu().numpy()
    C = ozk.dgemm(Ad, Bd, num_moduli=N).cpu().numpy()
    assert ozk.device_status() == "OZK2_OK"
    e, f = sc["e"].cpu().numpy().astype(np.int64), sc["f"].cpu().numpy().astype(np.int64)
    # A' = trunc(diag(2^e) A) and the columns of B' = trunc(B diag(2^f)), as M 2^s
    da = oz.scaled_decomposition(A.numpy(), e)
    db = oz.scaled_decomposition(B.numpy().T, f)
    moduli = oz.hybrid_moduli(N)
    residues = []
    for l, p in enumerate(moduli):
        pa = oz.digit_split(oz.residues_of_decomposition(*da, p), p)
        pb = [x.T for x in oz.digit_split(oz.residues_of_decomposition(*db, p), p)]
        want = np.asarray(oz.residue_product(pa, pb, p), dtype=np.int64)
        assert np.array_equal(res[l].astype(np.int64), want), f"modulus {p}"
        residues.append(want)
    Cw = oz.unscale(oz.crt_reconstruct(residues, moduli), e, f)
    assert np.array_equal(C.view(np.uint64), Cw.view(np.uint64))
