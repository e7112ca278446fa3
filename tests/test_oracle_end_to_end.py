"""End-to-end pins for the oracle's emulated DGEMM.

* Integer-valued inputs whose products and sums are exact in FP64: the
  emulation must return exactly A @ B (numpy float64, exact here).
* Error against the exact product (Python-integer dot products) on the paper's
  generator a = (U - 0.5) exp(phi N(0,1)) (Sec. V-A), per N: within
  k 2^-52 (|A||B|)_ij and improving with N by about log2 sqrt(p) bits per extra
  modulus until the FP64 floor (Table 2: bits ~ log2 sqrt(P/2)).
* Non-finite inputs and empty shapes (readings R10, degenerate cases).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz


def gen(shape, phi, rng):
    return (rng.random(shape) - 0.5) * np.exp(phi * rng.standard_normal(shape))


def rel_errors(A, B, C, samples):
    out = []
    for i, j in samples:
        ex = oz.exact_dot(A[i], B[:, j])
        ab = oz.exact_abs_dot(A[i], B[:, j])
        err = abs(float(ex - Fraction(float(C[i, j]))))
        out.append(err / float(ab) if ab else err)
    return np.array(out)


def test_integer_inputs_are_exact():
    rng = np.random.default_rng(0)
    A = rng.integers(-(2**10), 2**10, size=(16, 32)).astype(np.float64)
    B = rng.integers(-(2**10), 2**10, size=(32, 12)).astype(np.float64)
    C = oz.ozk2_dgemm(A, B, 12)["C"]
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0])
def test_error_bound_and_monotone_in_N(phi):
    rng = np.random.default_rng(int(phi * 4))
    m, k, n = 12, 256, 12
    A, B = gen((m, k), phi, rng), gen((k, n), phi, rng)
    samples = [(i, j) for i in range(m) for j in range(n)]
    worst = {}
    for N in [6, 8, 10, 12, 14, 16]:
        C = oz.ozk2_dgemm(A, B, N)["C"]
        worst[N] = rel_errors(A, B, C, samples).max()
    # FP64-level N satisfies the elementwise bound |C - AB| <= k 2^-52 |A||B|
    for N in (12, 14, 16):
        assert worst[N] <= k * 2.0**-52
    # error shrinks with N (allowing equality once the FP64 rounding floor is reached)
    Ns = sorted(worst)
    for a, b in zip(Ns, Ns[1:]):
        assert worst[b] <= worst[a] * 1.01 or worst[b] <= 2.0**-52
    # about 2 * 4.5 bits per two extra moduli while far from the floor
    gain = math.log2(worst[6] / worst[10])
    assert 12 <= gain <= 24


def test_accuracy_against_fp64_matmul():
    """At N = 12 on normal data the emulation is as accurate as FP64 GEMM (Sec. V-A)."""
    rng = np.random.default_rng(21)
    m, k, n = 8, 512, 8
    A, B = rng.standard_normal((m, k)), rng.standard_normal((k, n))
    C = oz.ozk2_dgemm(A, B, 12)["C"]
    samples = [(i, j) for i in range(m) for j in range(n)]
    e_emu = rel_errors(A, B, C, samples)
    e_nat = rel_errors(A, B, A @ B, samples)
    assert e_emu.max() <= 2 * max(e_nat.max(), 2.0**-53)


def test_nonfinite_rows_and_columns():
    rng = np.random.default_rng(3)
    A, B = gen((5, 7), 1.0, rng), gen((7, 4), 1.0, rng)
    A[1, 2] = np.nan
    B[3, 2] = np.inf
    r = oz.ozk2_dgemm(A, B, 12)
    C = r["C"]
    assert np.all(np.isnan(C[1])) and np.all(np.isnan(C[:, 2]))
    # other entries are unaffected: equal to the emulation with the bad entries zeroed
    A0, B0 = A.copy(), B.copy()
    A0[1, 2] = 0.0
    B0[3, 2] = 0.0
    C0 = oz.ozk2_dgemm(A0, B0, 12)["C"]
    mask = np.ones_like(C, dtype=bool)
    mask[1] = False
    mask[:, 2] = False
    assert np.array_equal(C[mask], C0[mask])


@pytest.mark.parametrize("shape", [(0, 3, 4), (3, 0, 4), (3, 4, 0), (0, 0, 0), (1, 1, 1)])
def test_empty_and_unit_shapes(shape):
    m, k, n = shape
    rng = np.random.default_rng(1)
    A, B = gen((m, k), 1.0, rng), gen((k, n), 1.0, rng)
    C = oz.ozk2_dgemm(A, B, 12)["C"]
    assert C.shape == (m, n)
    if k == 0:
        assert np.all(C == 0)
    if shape == (1, 1, 1):
        assert C[0, 0] == A[0, 0] * B[0, 0]
