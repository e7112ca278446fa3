"""Differentiable emulated product (OzakiMatmul): forward and both gradients.

* torch.autograd.gradcheck on a small problem (finite differences of the emulated
  forward against the emulated backward).
* Central finite differences of L = sum(W * (A B)) at 64^3 against dA, dB.
* The gradients are the emulated products dC B^T and A^T dC: bit-identical to the plain
  call on materialised transposes and to the oracle fed with the GPU's exponents.
* At 8192 x 4096 x 4096 (W ~ N(0, 1)): sampled entries of C, dA and dB against exact
  rational dot products, within k 2^-52 (|.||.|).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _leaf(X, cuda):
    return X.to(cuda).requires_grad_(True)


@pytest.mark.parametrize("reuse", [True, False])
def test_gradcheck_small(cuda, reuse):
    A, B = workloads.problem(8, 5, 6, 1.0, seed=20)
    Ad, Bd = _leaf(A, cuda), _leaf(B, cuda)
    assert torch.autograd.gradcheck(lambda a, b: ozk.matmul(a, b, 14, reuse=reuse), (Ad, Bd), eps=1e-6, atol=1e-9,
                                    rtol=1e-7)


@pytest.mark.parametrize("reuse", [True, False])
def test_finite_differences_64(cuda, reuse):
    n = 64
    A, B = workloads.problem(n, n, n, 1.0, seed=21)
    W = workloads.normal_matrix(n, n, seed=23)
    Ad, Bd, Wd = _leaf(A, cuda), _leaf(B, cuda), W.to(cuda)
    (ozk.matmul(Ad, Bd, 14, reuse=reuse) * Wd).sum().backward()
    torch_gA, torch_gB = (Wd @ B.to(cuda).T).cpu().numpy(), (A.to(cuda).T @ Wd).cpu().numpy()
    gA, gB = Ad.grad.cpu().numpy(), Bd.grad.cpu().numpy()

    def loss(a, b):
        return float((ozk.dgemm(a, b, num_moduli=14) * Wd).sum())

    rng = np.random.default_rng(5)
    h = 2.0**-12
    scale = float((W.abs() @ B.abs().T).max())
    for i, j in zip(rng.integers(0, n, 12), rng.integers(0, n, 12)):
        ap, am = A.clone(), A.clone()
        ap[i, j] += h
        am[i, j] -= h
        fd = (loss(ap.to(cuda), B.to(cuda)) - loss(am.to(cuda), B.to(cuda))) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-9 * scale
        bp, bm = B.clone(), B.clone()
        bp[i, j] += h
        bm[i, j] -= h
        fd = (loss(A.to(cuda), bp.to(cuda)) - loss(A.to(cuda), bm.to(cuda))) / (2 * h)
        assert abs(fd - gB[i, j]) <= 1e-9 * float((A.abs().T @ W.abs()).max())
    # and against torch float64's gradients: within a few FP64 roundings of the scale
    assert np.abs(gA - torch_gA).max() <= n * 2.0**-52 * scale
    assert np.abs(gB - torch_gB).max() <= n * 2.0**-52 * float((A.abs().T @ W.abs()).max())


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_fresh_gradients_are_emulated_products(cuda, mode):
    """reuse=False: each gradient is a fresh emulation of the transposed product."""
    m, k, n, N = 70, 50, 40, 13
    A, B = workloads.problem(m, n, k, 1.0, seed=24)
    W = workloads.normal_matrix(m, n, seed=26)
    Ad, Bd, Wd = _leaf(A, cuda), _leaf(B, cuda), W.to(cuda)
    C = ozk.matmul(Ad, Bd, N, mode, reuse=False)
    C.backward(Wd)
    assert torch.equal(C.detach(), ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N, mode=mode))
    BT = B.T.contiguous().to(cuda)
    AT = A.T.contiguous().to(cuda)
    assert torch.equal(Ad.grad, ozk.dgemm(Wd, BT, num_moduli=N, mode=mode))
    assert torch.equal(Bd.grad, ozk.dgemm(AT, Wd, num_moduli=N, mode=mode))
    sc = ozk.scales(Wd, BT, num_moduli=N, mode=mode)
    r = oz.ozk2_dgemm(W.numpy(), B.numpy().T.copy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy(), mode=mode)
    assert np.array_equal(Ad.grad.cpu().numpy().view(np.uint64), r["C"].view(np.uint64))
    assert ozk.device_status() == "OZK2_OK"


def test_reuse_gradients_are_the_backward_call(cuda):
    """The default (reuse=True): the gradients are ozk2_dgemm_backward's, bit-identical to
    the oracle's reuse route given the GPU's exponents."""
    m, k, n, N = 70, 50, 40, 13
    A, B = workloads.problem(m, n, k, 1.0, seed=24)
    W = workloads.normal_matrix(m, n, seed=26)
    Ad, Bd, Wd = _leaf(A, cuda), _leaf(B, cuda), W.to(cuda)
    C = ozk.matmul(Ad, Bd, N)
    C.backward(Wd)
    g, h = ozk.backward_exponents(m, n, k, N)  # before anything else reuses the library workspace
    assert torch.equal(C.detach(), ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N))
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    r = oz.reuse_gradients(A.numpy(), B.numpy(), W.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy(),
                           g=g.cpu().numpy(), h=h.cpu().numpy())
    assert np.array_equal(Ad.grad.cpu().numpy().view(np.uint64), r["dA"].view(np.uint64))
    assert np.array_equal(Bd.grad.cpu().numpy().view(np.uint64), r["dB"].view(np.uint64))
    assert ozk.device_status() == "OZK2_OK"


@pytest.mark.parametrize("reuse", [True, False])
def test_only_requested_gradients(cuda, reuse):
    A, B = workloads.problem(30, 20, 10, 1.0, seed=27)
    Ad, Bd = _leaf(A, cuda), B.to(cuda)
    ozk.matmul(Ad, Bd, reuse=reuse).sum().backward()  # broadcast (zero-stride) upstream gradient
    assert Bd.grad is None
    ones = torch.ones(30, 20, dtype=torch.float64, device=cuda)
    if reuse:
        ws = torch.empty(ozk.workspace_size(30, 20, 10, 12), dtype=torch.uint8, device=cuda)
        ozk.dgemm(A.to(cuda), B.to(cuda), workspace=ws)
        ref = ozk.dgemm_backward(A.to(cuda), B.to(cuda), ones, ws, need_dB=False)[0]
    else:
        ref = ozk.dgemm(ones, B.T.contiguous().to(cuda))
    assert torch.equal(Ad.grad, ref)


def _rel_err(x, exact, absdot):
    return abs(float(exact - Fraction(float(x)))) / float(absdot)


def test_full_size_sampled(cuda):
    m, k, n, N = 8192, 4096, 4096, 12
    A = workloads.phi_matrix(m, k, 1.0, 0, device=cuda)
    B = workloads.phi_matrix(k, n, 1.0, 1, device=cuda)
    W = workloads.normal_matrix(m, n, 2, device=cuda)
    Ad, Bd = A.clone().requires_grad_(True), B.clone().requires_grad_(True)
    C = ozk.matmul(Ad, Bd, N)
    C.backward(W)
    assert ozk.device_status() == "OZK2_OK"
    rng = np.random.default_rng(8)
    An, Bn, Wn = A.cpu().numpy(), B.cpu().numpy(), W.cpu().numpy()
    Cn, gA, gB = C.detach().cpu().numpy(), Ad.grad.cpu().numpy(), Bd.grad.cpu().numpy()
    for _ in range(12):
        i, j, h = int(rng.integers(0, m)), int(rng.integers(0, n)), int(rng.integers(0, k))
        assert _rel_err(Cn[i, j], oz.exact_dot(An[i], Bn[:, j]), oz.exact_abs_dot(An[i], Bn[:, j])) <= k * 2.0**-52
        assert _rel_err(gA[i, h], oz.exact_dot(Wn[i], Bn[h]), oz.exact_abs_dot(Wn[i], Bn[h])) <= n * 2.0**-52
        assert _rel_err(gB[h, j], oz.exact_dot(An[:, h], Wn[:, j]), oz.exact_abs_dot(An[:, h], Wn[:, j])) <= m * 2.0**-52
