"""Gradients that reuse the forward's exponents and digit planes (ozk2_dgemm_backward).

Given the GPU's forward exponents e, f and its dC exponents g, h (injected into the
oracle's reuse route), every later step is integer work: the residue products and the
final dA = dC B^T, dB = A^T dC must be bit-exact.  The GPU's g, h must satisfy the
Ozaki-II condition 2 sum |G'||B'| < P (and 2 sum |A'||H'| < P) exactly, and agree with the
oracle's own exponent rule up to the FP32 accumulation order of the bound products."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def forward_and_backward(A, B, dC, N, cuda, need_dA=True, need_dB=True):
    Ad, Bd, dCd = A.to(cuda), B.to(cuda), dC.to(cuda)
    m, k = A.shape
    n = B.shape[1]
    ws = torch.empty(ozk.workspace_size(m, n, k, N), dtype=torch.uint8, device=cuda)
    C = ozk.dgemm(Ad, Bd, num_moduli=N, workspace=ws)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    dA, dB = ozk.dgemm_backward(Ad, Bd, dCd, ws, N, need_dA=need_dA, need_dB=need_dB)
    g, h = ozk.backward_exponents(m, n, k, N)
    torch.cuda.synchronize()
    return C, sc, dA, dB, g, h


@pytest.mark.parametrize("m,n,k,N,phi", [(40, 36, 50, 12, 1.0), (300, 130, 70, 13, 0.5), (129, 257, 100, 16, 2.0),
                                         (5, 7, 3, 12, 1.0), (260, 200, 300, 12, 1.0)])
def test_backward_bit_exact(cuda, m, n, k, N, phi):
    A, B = workloads.problem(m, n, k, phi, seed=m + 3 * n)
    dC = workloads.normal_matrix(m, n, seed=k)
    C, sc, dA, dB, g, h = forward_and_backward(A, B, dC, N, cuda)
    assert ozk.device_status() == "OZK2_OK"
    e, f = sc["e"].cpu().numpy(), sc["f"].cpu().numpy()
    gn, hn = g.cpu().numpy(), h.cpu().numpy()
    r = oz.reuse_gradients(A.numpy(), B.numpy(), dC.numpy(), N, e=e, f=f, g=gn, h=hn)
    assert np.array_equal(dA.cpu().numpy().view(np.uint64), r["dA"].view(np.uint64))
    assert np.array_equal(dB.cpu().numpy().view(np.uint64), r["dB"].view(np.uint64))
    # the GPU's exponents satisfy the condition exactly
    moduli = oz.hybrid_moduli(N)
    P = oz.product_P(moduli)
    G = oz.dc_integers_for_dA(dC.numpy(), gn, f)
    Bi = oz.integer_cols(B.numpy(), f)
    lhs = 2 * np.abs(G).dot(np.abs(Bi).T)  # exact (object arrays of Python ints)
    assert max(int(x) for x in lhs.ravel()) < P
    H = oz.dc_integers_for_dB(dC.numpy(), hn, e)
    Ai = oz.integer_rows(A.numpy(), e)
    lhs = 2 * np.abs(Ai).T.dot(np.abs(H))
    assert max(int(x) for x in lhs.ravel()) < P
    # and follow the oracle's rule up to the bound products' FP32 summation order
    go = oz.reuse_side_exponents(dC.numpy(), B.numpy(), moduli)[0]
    ho = oz.reuse_side_exponents(dC.numpy().T, A.numpy().T, moduli)[0]
    assert np.abs(gn - go).max() <= 1 and np.mean(gn == go) >= 0.95
    assert np.abs(hn - ho).max() <= 1 and np.mean(hn == ho) >= 0.95


def test_backward_accuracy_next_to_fresh_and_native(cuda):
    """Sampled entries against the exact product: within 2x of native FP64 (as the
    forward), at N = 12, phi = 1."""
    m, n, k, N = 300, 280, 260, 12
    A, B = workloads.problem(m, n, k, 1.0, seed=31)
    dC = workloads.normal_matrix(m, n, seed=32)
    C, sc, dA, dB, g, h = forward_and_backward(A, B, dC, N, cuda)
    natA = (dC.to(cuda) @ B.to(cuda).T).cpu().numpy()
    natB = (A.to(cuda).T @ dC.to(cuda)).cpu().numpy()
    rng = np.random.default_rng(3)
    An, Bn, Cn = A.numpy(), B.numpy(), dC.numpy()
    worst = [0.0, 0.0, 0.0, 0.0]
    for _ in range(24):
        i, j, hh = int(rng.integers(0, m)), int(rng.integers(0, n)), int(rng.integers(0, k))
        ex, ab = oz.exact_dot(Cn[i], Bn[hh]), float(oz.exact_abs_dot(Cn[i], Bn[hh]))
        worst[0] = max(worst[0], abs(float(ex - oz.Fraction(float(dA[i, hh])))) / ab)
        worst[1] = max(worst[1], abs(float(ex - oz.Fraction(float(natA[i, hh])))) / ab)
        ex, ab = oz.exact_dot(An[:, hh], Cn[:, j]), float(oz.exact_abs_dot(An[:, hh], Cn[:, j]))
        worst[2] = max(worst[2], abs(float(ex - oz.Fraction(float(dB[hh, j])))) / ab)
        worst[3] = max(worst[3], abs(float(ex - oz.Fraction(float(natB[hh, j])))) / ab)
    assert worst[0] <= 2 * max(worst[1], 2.0**-53)
    assert worst[2] <= 2 * max(worst[3], 2.0**-53)


def test_backward_nonfinite_and_partial(cuda):
    m, n, k, N = 60, 50, 40, 12
    A, B = workloads.problem(m, n, k, 1.0, seed=33)
    dC = workloads.normal_matrix(m, n, seed=34)
    dC[3, 7] = float("nan")
    B[5, 9] = float("inf")
    A[11, 13] = -float("inf")
    C, sc, dA, dB, g, h = forward_and_backward(A, B, dC, N, cuda)
    assert ozk.device_status() == "OZK2_ERR_NONFINITE"
    dA, dB = dA.cpu().numpy(), dB.cpu().numpy()
    assert np.isnan(dA[3]).all() and np.isnan(dA[:, 5]).all()
    assert np.isnan(dB[:, 7]).all() and np.isnan(dB[13]).all()
    r = oz.reuse_gradients(A.numpy(), B.numpy(), dC.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy(),
                           g=g.cpu().numpy(), h=h.cpu().numpy())
    assert np.array_equal(dA.view(np.uint64), r["dA"].view(np.uint64))
    assert np.array_equal(dB.view(np.uint64), r["dB"].view(np.uint64))
    # one gradient only
    A2, B2 = workloads.problem(70, 30, 20, 1.0, seed=35)
    dC2 = workloads.normal_matrix(70, 30, seed=36)
    _, _, dA2, dB2, _, _ = forward_and_backward(A2, B2, dC2, N, cuda, need_dB=False)
    assert dB2 is None
    _, _, dA3, dB3, _, _ = forward_and_backward(A2, B2, dC2, N, cuda)
    assert torch.equal(dA2, dA3)
    _, _, dA4, dB4, _, _ = forward_and_backward(A2, B2, dC2, N, cuda, need_dA=False)
    assert dA4 is None and torch.equal(dB4, dB3)


def test_backward_argument_checks(cuda):
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A, B = workloads.problem(20, 10, 30, 1.0, seed=37, device=cuda)
    dC = torch.ones(20, 10, dtype=torch.float64, device=cuda)
    ws = torch.empty(ozk.workspace_size(20, 10, 30, 12), dtype=torch.uint8, device=cuda)
    ozk.dgemm(A, B, num_moduli=12, workspace=ws)
    dA = torch.full((20, 30), 9.0, dtype=torch.float64, device=cuda)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    # forward workspace too small, or host memory: refused, nothing written
    s = lib.ozk2_dgemm_backward(20, 10, 30, p(A), 30, p(B), 10, p(dC), 10, p(dA), 30, None, 10, 12, p(ws),
                                ws.numel() - 1, None, 0, st)
    assert s == 1
    hws = torch.zeros(ws.numel(), dtype=torch.uint8).pin_memory()
    s = lib.ozk2_dgemm_backward(20, 10, 30, p(A), 30, p(B), 10, p(dC), 10, p(dA), 30, None, 10, 12, p(hws),
                                hws.numel(), None, 0, st)
    assert s == 1
    torch.cuda.synchronize()
    assert (dA == 9.0).all().item()
    # empty reduction: dB (k x n) of an m = 0 product is zero
    dB = torch.full((30, 10), 9.0, dtype=torch.float64, device=cuda)
    s = lib.ozk2_dgemm_backward(0, 10, 30, None, 30, p(B), 10, None, 10, None, 30, p(dB), 10, 12, p(ws), ws.numel(),
                                None, 0, st)
    assert s == 0
    torch.cuda.synchronize()
    assert (dB == 0.0).all().item()
