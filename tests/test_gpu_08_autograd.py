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


def test_gradcheck_small(cuda):
    A, B = workloads.problem(8, 5, 6, 1.0, seed=20)
    Ad, Bd = _leaf(A, cuda), _leaf(B, cuda)
    assert torch.autograd.gradcheck(lambda a, b: ozk.matmul(a, b, 14), (Ad, Bd), eps=1e-6, atol=1e-9, rtol=1e-7)


def test_finite_differences_64(cuda):
    n = 64
    A, B = workloads.problem(n, n, n, 1.0, seed=21)
    W = workloads.normal_matrix(n, n, seed=23)
    Ad, Bd, Wd = _leaf(A, cuda), _leaf(B, cuda), W.to(cuda)
    (ozk.matmul(Ad, Bd, 14) * Wd).sum().backward()
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


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_gradients_are_emulated_products(cuda, mode):
    m, k, n, N = 70, 50, 40, 13
    A, B = workloads.problem(m, n, k, 1.0, seed=24)
    W = workloads.normal_matrix(m, n, seed=26)
    Ad, Bd, Wd = _leaf(A, cuda), _leaf(B, cuda), W.to(cuda)
    C = ozk.matmul(Ad, Bd, N, mode)
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


def test_only_requested_gradients(cuda):
    A, B = workloads.problem(30, 20, 10, 1.0, seed=27)
    Ad, Bd = _leaf(A, cuda), B.to(cuda)
    ozk.matmul(Ad, Bd).sum().backward()  # broadcast (zero-stride) upstream gradient
    assert Bd.grad is None
    ref = ozk.dgemm(torch.ones(30, 20, dtype=torch.float64, device=cuda), B.T.contiguous().to(cuda))
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
