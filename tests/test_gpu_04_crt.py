"""CRT reconstruction and inverse scaling on the GPU (Eqs. CRT_finalreduction and
inversescaling) against the oracle's big-integer CRT and correctly rounded
conversion, on random residues with exponents that reach subnormal results and
overflow."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz

pytestmark = pytest.mark.gpu


def random_residues(rng, moduli, m, n):
    return np.stack([rng.integers(-(p // 2), p - p // 2, size=(m, n)) for p in moduli]).astype(np.int16)


@pytest.mark.parametrize("N", [1, 2, 6, 7, 12, 13, 14, 16, 20])
def test_crt_bit_exact(cuda, N):
    rng = np.random.default_rng(N)
    moduli = oz.hybrid_moduli(N)
    m, n = 37, 45
    res = random_residues(rng, moduli, m, n)
    e = rng.integers(-60, 60, size=m)
    f = rng.integers(-60, 60, size=n)
    C = ozk.crt(torch.as_tensor(res).to(cuda), torch.as_tensor(e), torch.as_tensor(f)).cpu().numpy()
    Cint = oz.crt_reconstruct([r.astype(np.int64) for r in res], moduli)
    want = oz.unscale(Cint, e, f)
    assert np.array_equal(C.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("shift", [-1200, -950, -900, 900, 1100, 1150, 1180, 1250])
def test_crt_subnormal_and_overflow(cuda, shift):
    rng = np.random.default_rng(abs(shift))
    N = 12
    moduli = oz.hybrid_moduli(N)
    m, n = 16, 24
    res = random_residues(rng, moduli, m, n)
    res[:, 0, 0] = 0  # an exact zero
    e = np.full(m, shift // 2) + rng.integers(-3, 4, size=m)
    f = np.full(n, shift - shift // 2) + rng.integers(-3, 4, size=n)
    C = ozk.crt(torch.as_tensor(res).to(cuda), torch.as_tensor(e), torch.as_tensor(f)).cpu().numpy()
    want = oz.unscale(oz.crt_reconstruct([r.astype(np.int64) for r in res], moduli), e, f)
    assert np.array_equal(C.view(np.uint64), want.view(np.uint64))


def test_crt_extreme_residues(cuda):
    """Residue combinations whose CRT value sits next to +-P/2."""
    N = 12
    moduli = oz.hybrid_moduli(N)
    P = oz.product_P(moduli)
    vals = [P // 2 - 1, -(P // 2), -(P // 2) + 1, P // 2 - 12345, 0, 1, -1, P // 3, -(P // 3)]
    X = np.array(vals, dtype=object).reshape(1, -1)
    res = np.stack([oz.smod(X, p).astype(np.int64) for p in moduli]).astype(np.int16)
    e = np.array([0])
    f = np.zeros(len(vals), dtype=np.int64)
    C = ozk.crt(torch.as_tensor(res).to(cuda), torch.as_tensor(e), torch.as_tensor(f)).cpu().numpy()
    want = np.array([[oz.round_scaled_to_double(v, 0) for v in vals]])
    assert np.array_equal(C.view(np.uint64), want.view(np.uint64))
