"""Pins for accurate-mode scaling (Sec. III-E) and the Ozaki-II condition (Sec. II).

The scaling vectors must satisfy 2 sum_h |a'_ih| |b'_hj| < P for every (i, j)
(Eq. condition); this is checked with exact integers.  The FP32 constants P'
and delta are checked for the round-down property with an independent
high-precision evaluation (the decimal module).
"""
import decimal
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz


def gen(shape, phi, rng):
    return (rng.random(shape) - 0.5) * np.exp(phi * rng.standard_normal(shape))


def test_delta_is_round_down():
    d = oz.delta_constant()
    exact = Fraction(-1) / (2 - Fraction(1, 1 << 21))
    assert d.dtype == np.float32
    assert Fraction(float(d)) <= exact < Fraction(float(np.nextafter(d, np.float32(np.inf))))
    assert float(d) == float.fromhex("-0x1.000006p-1")


def _log2_decimal(n):
    decimal.getcontext().prec = 80
    return decimal.Decimal(n).ln() / decimal.Decimal(2).ln()


@pytest.mark.parametrize("N", [1, 2, 6, 7, 12, 13, 14, 16, 20])
def test_pprime_is_round_down(N):
    moduli = oz.hybrid_moduli(N)
    pp = oz.p_prime_constant(moduli)
    P = oz.product_P(moduli)
    exact = (_log2_decimal(P - 1) - 1) / 2
    lo = decimal.Decimal(float(pp))
    hi = decimal.Decimal(float(np.nextafter(pp, np.float32(np.inf))))
    assert lo <= exact < hi


def test_prelim_exponent_is_ufp():
    rng = np.random.default_rng(1)
    A = gen((40, 30), 2.0, rng)
    A[7] = 0.0
    A[8, :] = 0.0
    A[8, 3] = 5e-324  # subnormal row maximum
    ep = oz.prelim_exponent_rows(A)
    for i in range(40):
        mx = np.abs(A[i]).max()
        if mx == 0:
            assert ep[i] == 0
        else:
            m, ex = math.frexp(mx)
            assert ep[i] == 7 - (ex - 1)
    assert ep[8] == 7 + 1074


def test_bound_product_error_bound():
    """|AbarBbar - Cbar'| <= (k-1) 2^-24 AbarBbar, hence cbar >= Abar Bbar [Eq. barCupper]."""
    rng = np.random.default_rng(2)
    for (m, k, n) in [(8, 1, 8), (16, 100, 12), (9, 777, 5)]:
        A, B = gen((m, k), 1.0, rng), gen((k, n), 1.0, rng)
        sc = oz.scaling_exponents(A, B, 12)
        exact = oz.e4m3_decode_array(sc["Abar"]) @ oz.e4m3_decode_array(sc["Bbar"])
        cbar = sc["cbar"].astype(np.float64)
        assert np.all(cbar >= exact)
        assert np.all(cbar <= exact * (1 + (2 * k + 4) * 2.0**-24) + 1e-30)


def _check_condition(A, B, N, e=None, f=None):
    r = oz.ozk2_dgemm(A, B, N, e=e, f=f, keep=True)
    P = oz.product_P(r["moduli"])
    Ai = np.abs(r["Aint"]).astype(object)
    Bi = np.abs(r["Bint"]).astype(object)
    lhs = 2 * (Ai.dot(Bi)) if A.shape[1] else np.zeros((A.shape[0], B.shape[1]), dtype=object)
    worst = max((int(v) for v in lhs.flat), default=0)
    return worst, P, r


@pytest.mark.parametrize("phi", [0.0, 0.5, 1.0, 2.0, 4.0])
@pytest.mark.parametrize("N", [6, 12, 16])
def test_condition_holds(phi, N):
    """Eq. condition holds exactly for the accurate-mode exponents."""
    rng = np.random.default_rng(int(phi * 10) + N)
    A, B = gen((12, 37), phi, rng), gen((37, 10), phi, rng)
    worst, P, _ = _check_condition(A, B, N)
    assert worst < P
    # and the scaling is not wasteful: the largest entry uses a good part of P
    assert worst > P / 2**12


def test_condition_holds_degenerate_rows():
    rng = np.random.default_rng(9)
    A, B = gen((6, 20), 1.0, rng), gen((20, 5), 1.0, rng)
    A[0] = 0.0  # zero row
    A[1] = 0.0
    A[1, 4] = 3.0  # row whose only entry meets a zero row of B
    B[4] = 0.0
    A[2, 0] = 1e300  # huge entry next to tiny ones
    A[3] *= 1e-310  # subnormal row
    worst, P, r = _check_condition(A, B, 12)
    assert worst < P
    assert r["e"][0] == 0 and r["eprime"][0] == 0
    assert r["R"][1] == 0 and r["e"][1] == r["eprime"][1] + math.floor(float(r["pprime"]))


def test_exponents_with_injected_bound_maxima():
    """final_exponent is monotone in the bound maximum and reaches the P budget:
    2^(e - e') sqrt(R) lies in [sqrt((P-1)/2)/2^1.001, sqrt((P-1)/2)]."""
    moduli = oz.hybrid_moduli(12)
    P = oz.product_P(moduli)
    pp, d = oz.p_prime_constant(moduli), oz.delta_constant()
    prev = None
    for R in [2.0**-18, 0.37, 1.0, 3.0, 1e3, 12345.678, 2.0**33]:
        R32 = np.float32(R)
        e = oz.final_exponent(0, R32, pp, d, False)
        val = 2.0 ** (2 * e) * float(R32)
        assert val <= (P - 1) / 2
        assert val >= (P - 1) / 2 / 2**2.01
        if prev is not None:
            assert e <= prev
        prev = e


def test_planted_sign_error_is_caught(monkeypatch):
    """A plausible mistake (delta with the wrong sign) breaks Eq. condition."""
    rng = np.random.default_rng(4)
    A, B = gen((8, 64), 1.0, rng), gen((64, 8), 1.0, rng)
    monkeypatch.setattr(oz, "delta_constant", lambda: np.float32(0.5))
    worst, P, _ = _check_condition(A, B, 12)
    assert worst >= P


@pytest.mark.parametrize("phi", [0.5, 1.0, 2.0])
def test_fast_mode_condition_and_cauchy_schwarz(phi):
    """Fast mode (R15): the squared-norm bound dominates ||2^e' a_i||^2, Eq. condition
    holds exactly, and the result is accurate, slightly below accurate mode."""
    rng = np.random.default_rng(int(phi * 7))
    A, B = gen((10, 45), phi, rng), gen((45, 9), phi, rng)
    sc = oz.scaling_exponents(A, B, 13, mode="fast")
    for i in range(10):
        exact = sum(Fraction(float(x)) ** 2 * Fraction(2) ** (2 * int(sc["eprime"][i])) for x in A[i])
        assert Fraction(float(sc["R"][i])) >= exact
    r = oz.ozk2_dgemm(A, B, 13, keep=True, mode="fast")
    P = oz.product_P(r["moduli"])
    lhs = 2 * np.abs(r["Aint"]).astype(object).dot(np.abs(r["Bint"]).astype(object))
    assert max(int(v) for v in lhs.flat) < P
    # fast mode uses fewer bits than accurate mode, never more
    acc = oz.ozk2_dgemm(A, B, 13, keep=True)
    assert np.all(r["e"] <= acc["e"] + 1) and np.all(r["f"] <= acc["f"] + 1)
    assert max(int(v) for v in lhs.flat) > P / 2**16
