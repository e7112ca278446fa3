"""Residues, digit planes and residue products on the GPU against the oracle.

Given the same exponents e, f (the GPU's, injected into the oracle), everything is
integer work: the FP8 digit planes (Sec. III-B, III-D) and the residue products
C'_l = mod(A'_l B'_l, p_l) (Eq. CRTmatmul via Eqs. 3matmult-notKaratsuba and
C'-Karatsuba) must be bit-exact.  C'_l is also checked against its plain
definition smod((A'B'), p_l) computed with Python integers."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def oracle_codes(digits):
    lut = {d: oz.e4m3_code_of_integer(d) for d in range(-16, 17)}
    return np.vectorize(lut.get)(digits).astype(np.uint8)


@pytest.mark.parametrize("m,n,k,phi,N", [(64, 48, 100, 0.5, 12), (37, 29, 1100, 2.0, 7),
                                         (16, 16, 40, 1.0, 20), (8, 9, 3, 1.0, 4),
                                         # the unrolled kernels (N = 8 .. 16); at N = 16
                                         # many elements have t' > 0 (the 2^t' mod p path)
                                         (19, 70, 530, 0.5, 8), (33, 17, 257, 1.0, 13),
                                         (40, 33, 300, 1.0, 16)])
def test_digit_planes_bit_exact(cuda, m, n, k, phi, N):
    A, B = workloads.problem(m, n, k, phi, seed=k)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    pa, pb = ozk.residue_planes(A.to(cuda), B.to(cuda), sc["e"], sc["f"], num_moduli=N)
    pa, pb = pa.cpu().numpy(), pb.cpu().numpy()
    e, f = sc["e"].cpu().numpy(), sc["f"].cpu().numpy()
    Aint = oz.integer_rows(A.numpy(), e)
    BintT = oz.integer_rows(B.numpy().T, f)  # columns of B as rows
    plane = 0
    for p in oz.hybrid_moduli(N):
        da = oz.digit_planes(Aint, p)
        db = oz.digit_planes(BintT, p)
        for x in range(len(da)):
            assert np.array_equal(pa[plane + x][:, :k], oracle_codes(da[x])), (p, x)
            assert np.array_equal(pb[plane + x][:, :k], oracle_codes(db[x])), (p, x)
        plane += len(da)
    assert plane == oz.num_digit_planes(N)


@pytest.mark.parametrize("m,n,k,phi,N", [(256, 256, 256, 0.5, 12), (200, 130, 300, 1.0, 12),
                                         (130, 260, 1000, 2.0, 14), (5, 7, 9, 1.0, 20),
                                         (128, 128, 128, 1.0, 6), (129, 127, 700, 1.0, 16)])
def test_residue_products_bit_exact(cuda, m, n, k, phi, N):
    A, B = workloads.problem(m, n, k, phi, seed=3 * m + n)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    res = ozk.residue_products(A.to(cuda), B.to(cuda), sc["e"], sc["f"], num_moduli=N).cpu().numpy()
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy())
    for l, p in enumerate(r["moduli"]):
        assert np.array_equal(res[l].astype(np.int64), r["residues"][l]), f"modulus {p}"


def test_residue_products_long_reduction(cuda):
    """k > 2^16: two exactness blocks whose residues are added mod p."""
    m, n, k, N = 8, 12, 70000, 12
    A, B = workloads.problem(m, n, k, 1.0, seed=11)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    res = ozk.residue_products(A.to(cuda), B.to(cuda), sc["e"], sc["f"], num_moduli=N).cpu().numpy()
    e, f = sc["e"].cpu().numpy(), sc["f"].cpu().numpy()
    Aint = oz.integer_rows(A.numpy(), e)
    Bint = oz.integer_cols(B.numpy(), f)
    direct = Aint.dot(Bint)
    for l, p in enumerate(oz.hybrid_moduli(N)):
        assert np.array_equal(res[l].astype(np.int64), oz.smod(direct, p).astype(np.int64)), p


def test_residue_products_extreme_exponents(cuda):
    """Exponents injected far from the scaling rule exercise the 2^t mod p table
    (a' beyond 2^53) and the shift-out path (a' = 0)."""
    m, n, k, N = 16, 16, 64, 14
    A, B = workloads.problem(m, n, k, 1.0, seed=5)
    e = torch.tensor([60 + 2 * i for i in range(m)], dtype=torch.int32)
    e[0] = -5
    f = torch.tensor([3 * j - 10 for j in range(n)], dtype=torch.int32)
    res = ozk.residue_products(A.to(cuda), B.to(cuda), e, f, num_moduli=N).cpu().numpy()
    Aint = oz.integer_rows(A.numpy(), e.numpy())
    Bint = oz.integer_cols(B.numpy(), f.numpy())
    direct = Aint.dot(Bint)
    for l, p in enumerate(oz.hybrid_moduli(N)):
        assert np.array_equal(res[l].astype(np.int64), oz.smod(direct, p).astype(np.int64)), p
