"""ozk2_dgemm_ex through the C ABI: transposed operands, fast mode and m/n blocking.

* op(A) = A^T and op(B) = B^T read the stored matrices in place: results, exponents and
  status are bit-identical to the row-major call on the materialised operands.
* Fast mode (the Cauchy-Schwarz scaling of Sec. III-E): bit-exact against the oracle in
  fast mode fed with the GPU's exponents; the GPU's squared-norm bounds lie above the
  oracle's (exactly summed, rounded up once) by at most the round-up chain; the
  Ozaki-II condition 2 sum |a'||b'| < P holds exactly; the error stays within
  k 2^-52 |A||B|.
* Blocking (Sec. IV-C): each block of C is bit-exact against the oracle run on that
  block alone; device flags of every block reach ozk2_device_status.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _view(X, trans, cuda):
    """X (CPU, logical matrix) on the device, stored row-major (trans False) or stored
    transposed and handed over as a transposed view (trans True)."""
    if trans:
        return X.T.contiguous().to(cuda).T
    return X.to(cuda)


@pytest.mark.parametrize("m,n,k,N", [(200, 130, 300, 12), (17, 300, 129, 16), (1, 70, 33, 12), (130, 1, 1, 7)])
@pytest.mark.parametrize("ta,tb", [(False, True), (True, False), (True, True)])
def test_transposes_match_row_major(cuda, m, n, k, N, ta, tb):
    A, B = workloads.problem(m, n, k, 1.0, seed=11)
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N)
    Av, Bv = _view(A, ta, cuda), _view(B, tb, cuda)
    C = ozk.dgemm(Av, Bv, num_moduli=N)
    assert torch.equal(C.view(torch.int64), ref.view(torch.int64))
    s0 = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    s1 = ozk.scales(Av, Bv, num_moduli=N)
    for key in ("e", "f", "eprime", "fprime", "R", "S", "Abar", "BbarT"):
        assert torch.equal(s0[key], s1[key]), key
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=s1["e"].cpu().numpy(), f=s1["f"].cpu().numpy())
    assert np.array_equal(C.cpu().numpy().view(np.uint64), r["C"].view(np.uint64))
    assert ozk.device_status() == "OZK2_OK"


def test_transposed_strided_storage(cuda):
    """op(A) = A^T with lda > m and op(B) = B^T with ldb > k (views into wider buffers)."""
    m, n, k = 90, 70, 150
    A, B = workloads.problem(m, n, k, 0.5, seed=12)
    At = torch.zeros((k, m + 37), dtype=torch.float64)
    At[:, :m] = A.T
    Bt = torch.zeros((n, k + 5), dtype=torch.float64)
    Bt[:, :k] = B.T
    Av = At.to(cuda)[:, :m].T
    Bv = Bt.to(cuda)[:, :k].T
    assert Av.stride() == (1, m + 37) and Bv.stride() == (1, k + 5)
    C = ozk.dgemm(Av, Bv, num_moduli=12)
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12)
    assert torch.equal(C, ref)


@pytest.mark.parametrize("m,n,k,phi,N", [(128, 96, 200, 1.0, 13), (40, 300, 1000, 2.0, 14), (5, 7, 3, 0.5, 12),
                                         (64, 64, 64, 1.0, 6)])
def test_fast_mode_bit_exact(cuda, m, n, k, phi, N):
    A, B = workloads.problem(m, n, k, phi, seed=13)
    Ad, Bd = A.to(cuda), B.to(cuda)
    C = ozk.dgemm(Ad, Bd, num_moduli=N, mode="fast").cpu().numpy()
    assert ozk.device_status() == "OZK2_OK"
    sc = ozk.scales(Ad, Bd, num_moduli=N, mode="fast")
    e, f = sc["e"].cpu().numpy(), sc["f"].cpu().numpy()
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=e, f=f, mode="fast")
    assert np.array_equal(C.view(np.uint64), r["C"].view(np.uint64))
    # the GPU bounds: upper bounds of the oracle's exactly summed ones, by a round-up chain
    orc = oz.scaling_exponents(A.numpy(), B.numpy(), N, mode="fast")
    for gpu, ref, cnt in ((sc["R"], orc["R"], k), (sc["S"], orc["S"], k)):
        g = gpu.cpu().numpy().astype(np.float64)
        o = ref.astype(np.float64)
        assert np.all(g >= o)
        assert np.all(g <= o * (1 + (cnt + 2) * 2.0**-23) + 2.0**-120)
    assert np.all((e == orc["e"]) | (e == orc["e"] - 1))
    assert np.all((f == orc["f"]) | (f == orc["f"] - 1))
    if min(m, n) >= 40:
        assert np.mean(e == orc["e"]) > 0.9 and np.mean(f == orc["f"]) > 0.9


def test_fast_mode_condition_exact(cuda):
    m, n, k, N = 24, 20, 300, 12
    A, B = workloads.problem(m, n, k, 1.0, seed=14)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N, mode="fast")
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy(), keep=True)
    P = oz.product_P(r["moduli"])
    lhs = 2 * np.abs(r["Aint"]).astype(object).dot(np.abs(r["Bint"]).astype(object))
    worst = max(int(v) for v in lhs.flat)
    assert worst < P
    assert worst > P / 2**20  # the bound is not wasteful


@pytest.mark.parametrize("phi,N", [(0.5, 14), (1.0, 14), (1.0, 16)])
def test_fast_mode_error_against_exact_product(cuda, phi, N):
    m, n, k = 96, 96, 2048
    A, B = workloads.problem(m, n, k, phi, seed=15)
    C = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N, mode="fast").cpu().numpy()
    rng = np.random.default_rng(3)
    An, Bn = A.numpy(), B.numpy()
    worst = 0.0
    for i, j in zip(rng.integers(0, m, 64), rng.integers(0, n, 64)):
        ex = oz.exact_dot(An[i], Bn[:, j])
        ab = float(oz.exact_abs_dot(An[i], Bn[:, j]))
        worst = max(worst, abs(float(ex - Fraction(float(C[i, j])))) / ab)
    assert worst <= k * 2.0**-52


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_blocked_matches_per_block_oracle(cuda, mode):
    m, n, k, N = 300, 260, 200, 12
    bm, bn = 128, 96
    A, B = workloads.problem(m, n, k, 1.0, seed=16)
    # rows / columns of very different magnitude, so that per-block scaling matters
    A[:64] *= 1e6
    B[:, 200:] *= 1e-9
    Ad, Bd = A.to(cuda), B.to(cuda)
    C = ozk.dgemm(Ad, Bd, num_moduli=N, mode=mode, block=(bm, bn)).cpu().numpy()
    assert ozk.device_status() == "OZK2_OK"
    for i0 in range(0, m, bm):
        for j0 in range(0, n, bn):
            Ab, Bb = Ad[i0:i0 + bm], Bd[:, j0:j0 + bn]
            sc = ozk.scales(Ab, Bb, num_moduli=N, mode=mode)
            r = oz.ozk2_dgemm(A[i0:i0 + bm].numpy(), B[:, j0:j0 + bn].numpy(), N, e=sc["e"].cpu().numpy(),
                              f=sc["f"].cpu().numpy(), mode=mode)
            blk = C[i0:i0 + bm, j0:j0 + bn]
            assert np.array_equal(blk.view(np.uint64), r["C"].view(np.uint64)), (i0, j0)


def test_blocked_transposed_workspace_and_flags(cuda):
    m, n, k, N = 200, 150, 90, 13
    A, B = workloads.problem(m, n, k, 0.5, seed=17)
    A[3, 5] = float("nan")  # in the first block only
    Av, Bv = _view(A, True, cuda), _view(B, True, cuda)
    need = ozk.workspace_size(m, n, k, N, mode="fast", block=(64, 64))
    assert need == ozk.workspace_size(64, 64, k, N, mode="fast")
    ws = torch.empty(need, dtype=torch.uint8, device=cuda)
    C = ozk.dgemm(Av, Bv, num_moduli=N, mode="fast", block=(64, 64), workspace=ws)
    # the first block's flag survives the later blocks
    assert ozk.device_status(workspace=ws) == "OZK2_ERR_NONFINITE"
    C = C.cpu()
    assert torch.all(torch.isnan(C[3])) and not torch.any(torch.isnan(C[4:]))
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N, mode="fast", block=(64, 64)).cpu()
    assert torch.equal(torch.nan_to_num(C), torch.nan_to_num(ref))
    with pytest.raises(ozk.Ozk2Error):
        ozk.dgemm(Av, Bv, num_moduli=N, mode="fast", block=(64, 64), workspace=ws[: need - 256])
