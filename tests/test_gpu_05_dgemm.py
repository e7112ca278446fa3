"""The whole emulated DGEMM through the C ABI (ozk2_dgemm) against the oracle.

* Bit-exact against the oracle fed with the GPU's exponents (everything after the
  FP32 bound product is integer arithmetic with one final correctly rounded step).
* Against the exact product: |C - AB| <= k 2^-52 (|A||B|) elementwise and within
  2x of native FP64 GEMM's error on the same inputs (N = 12 and 14, paper's generator
  of Sec. V-A).
* Degenerate inputs: empty sizes, k = 1, zero rows/columns, NaN/Inf (reading:
  NaN rows/columns), strided (lda > k) views, the caller-owned workspace entry.
"""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def gpu_dgemm_with_exps(A, B, N, cuda):
    Ad, Bd = A.to(cuda), B.to(cuda)
    C = ozk.dgemm(Ad, Bd, num_moduli=N)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    return C.cpu().numpy(), sc["e"].cpu().numpy(), sc["f"].cpu().numpy()


@pytest.mark.parametrize("m,n,k,phi,N", [(256, 256, 256, 0.5, 12), (200, 130, 300, 1.0, 12),
                                         (130, 260, 1000, 2.0, 14), (64, 64, 64, 1.0, 6),
                                         (17, 300, 129, 1.0, 16), (3, 5, 7, 0.5, 20)])
def test_bit_exact_against_oracle(cuda, m, n, k, phi, N):
    A, B = workloads.problem(m, n, k, phi, seed=0)
    C, e, f = gpu_dgemm_with_exps(A, B, N, cuda)
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=e, f=f)
    assert np.array_equal(C.view(np.uint64), r["C"].view(np.uint64))
    assert ozk.device_status() == "OZK2_OK"


@pytest.mark.parametrize("phi,N", [(0.5, 12), (1.0, 12), (2.0, 14), (1.0, 14)])
def test_error_against_exact_product(cuda, phi, N):
    m, n, k = 128, 128, 2048
    A, B = workloads.problem(m, n, k, phi, seed=1)
    Ad, Bd = A.to(cuda), B.to(cuda)
    C = ozk.dgemm(Ad, Bd, num_moduli=N).cpu().numpy()
    Cnat = (Ad @ Bd).cpu().numpy()
    rng = np.random.default_rng(2)
    idx = [(int(i), int(j)) for i, j in zip(rng.integers(0, m, 96), rng.integers(0, n, 96))]
    An, Bn = A.numpy(), B.numpy()
    emu, nat = [], []
    for i, j in idx:
        ex = oz.exact_dot(An[i], Bn[:, j])
        ab = float(oz.exact_abs_dot(An[i], Bn[:, j]))
        emu.append(abs(float(ex - oz.Fraction(float(C[i, j])))) / ab)
        nat.append(abs(float(ex - oz.Fraction(float(Cnat[i, j])))) / ab)
    emu, nat = np.array(emu), np.array(nat)
    assert emu.max() <= k * 2.0**-52
    assert emu.max() <= 2 * max(nat.max(), 2.0**-53)


def test_empty_and_degenerate_shapes(cuda):
    for (m, n, k) in [(0, 5, 5), (5, 0, 5), (5, 5, 0), (1, 1, 1), (1, 300, 1), (300, 1, 2)]:
        A, B = workloads.problem(m, n, k, 1.0, seed=3)
        C = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12).cpu().numpy()
        assert C.shape == (m, n)
        if k == 0:
            assert np.all(C == 0)
        elif m and n:
            sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=12)
            r = oz.ozk2_dgemm(A.numpy(), B.numpy(), 12, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy())
            assert np.array_equal(C.view(np.uint64), r["C"].view(np.uint64))
            absab = np.abs(A.numpy()) @ np.abs(B.numpy())
            assert np.all(np.abs(C - A.numpy() @ B.numpy()) <= (k + 2) * 2.0**-52 * absab)


def test_zero_rows_and_nonfinite(cuda):
    A, B = workloads.problem(40, 30, 50, 1.0, seed=4)
    A[2] = 0.0
    B[:, 3] = 0.0
    A[5, 7] = float("nan")
    B[9, 11] = float("inf")
    C = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12)
    assert ozk.device_status() == "OZK2_ERR_NONFINITE"
    C = C.cpu().numpy()
    assert np.all(C[2][np.arange(30) != 11] == 0)
    assert np.all(np.isnan(C[5])) and np.all(np.isnan(C[:, 11]))
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=12)
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), 12, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy())
    assert np.array_equal(np.isnan(C), np.isnan(r["C"]))
    ok = ~np.isnan(C)
    assert np.array_equal(C[ok], r["C"][ok])


def test_strided_views_and_caller_workspace(cuda):
    A0, B0 = workloads.problem(100, 90, 80, 1.0, seed=6)
    bigA = torch.zeros((100, 128), dtype=torch.float64)
    bigA[:, :80] = A0
    bigB = torch.zeros((80, 100), dtype=torch.float64)
    bigB[:, :90] = B0
    Ad = bigA.to(cuda)[:, :80]
    Bd = bigB.to(cuda)[:, :90]
    assert Ad.stride(0) == 128 and Bd.stride(0) == 100
    C1 = ozk.dgemm(Ad, Bd, num_moduli=12)
    ws = torch.empty(ozk.workspace_size(100, 90, 80, 12), dtype=torch.uint8, device=cuda)
    C2 = ozk.dgemm(A0.to(cuda), B0.to(cuda), num_moduli=12, workspace=ws)
    assert torch.equal(C1, C2)
    assert ozk.device_status(workspace=ws) == "OZK2_OK"


def test_integer_inputs_exact(cuda):
    rng = np.random.default_rng(7)
    A = torch.as_tensor(rng.integers(-(2**12), 2**12, size=(64, 256)).astype(np.float64))
    B = torch.as_tensor(rng.integers(-(2**12), 2**12, size=(256, 48)).astype(np.float64))
    C = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12).cpu().numpy()
    assert np.array_equal(C, A.numpy() @ B.numpy())
