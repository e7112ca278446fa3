"""Pins of the oracle's gradient route that reuses the forward's integer matrices A', B'
(dA = dC B^T with B' fixed, dB = A^T dC with A' fixed; the exponents of dC's side take
the whole budget of P).  Pinned by: the Ozaki-II condition (Sec. II Eq. condition) in
exact integers for every entry, the per-entry plain definition (exact integer dot, one
rounding), integer-valued inputs giving the exact product, the exponent rule's margin
checked in exact rationals against injected bound maxima, accuracy against the exact
product next to native FP64 and the fresh emulation, and planted mistakes."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz


def gen(shape, phi, rng):
    return (rng.random(shape) - 0.5) * np.exp(phi * rng.standard_normal(shape))


def problem(m, n, k, phi, seed):
    rng = np.random.default_rng(seed)
    return gen((m, k), phi, rng), gen((k, n), phi, rng), rng.standard_normal((m, n))


@pytest.mark.parametrize("phi,N", [(0.5, 12), (1.0, 12), (2.0, 14), (1.0, 7)])
def test_condition_holds_exactly(phi, N):
    A, B, dC = problem(9, 8, 11, phi, int(10 * phi) + N)
    moduli = oz.hybrid_moduli(N)
    P = oz.product_P(moduli)
    sc = oz.scaling_exponents(A, B, N, moduli)
    e, f = sc["e"], sc["f"]
    g = oz.reuse_side_exponents(dC, B, moduli)[0]
    h = oz.reuse_side_exponents(dC.T, A.T, moduli)[0]
    Bint = oz.integer_cols(B, f)
    Aint = oz.integer_rows(A, e)
    G = oz.dc_integers_for_dA(dC, g, f)
    H = oz.dc_integers_for_dB(dC, h, e)
    for i in range(9):
        for hh in range(11):
            assert 2 * sum(abs(G[i, j]) * abs(Bint[hh, j]) for j in range(8)) < P
    for hh in range(11):
        for j in range(8):
            assert 2 * sum(abs(Aint[i, hh]) * abs(H[i, j]) for i in range(9)) < P


@pytest.mark.parametrize("N,seed", [(12, 1), (16, 2), (6, 3)])
def test_gradients_equal_plain_definition(N, seed):
    A, B, dC = problem(7, 6, 9, 1.0, seed)
    moduli = oz.hybrid_moduli(N)
    r = oz.reuse_gradients(A, B, dC, N)
    sc = oz.scaling_exponents(A, B, N, moduli)
    for i in range(7):
        for hh in range(9):
            v, cond = oz.reuse_gradient_entry_dA(dC[i], B[hh], sc["f"], r["g"][i], moduli)
            assert cond and np.float64(v).view(np.uint64) == np.float64(r["dA"][i, hh]).view(np.uint64)
    for hh in range(9):
        for j in range(6):
            v, cond = oz.reuse_gradient_entry_dB(A[:, hh], dC[:, j], sc["e"], r["h"][j], moduli)
            assert cond and np.float64(v).view(np.uint64) == np.float64(r["dB"][hh, j]).view(np.uint64)


def test_integer_inputs_give_exact_gradients():
    rng = np.random.default_rng(4)
    A = rng.integers(-2**10, 2**10, (6, 8)).astype(np.float64)
    B = rng.integers(-2**10, 2**10, (8, 5)).astype(np.float64)
    dC = rng.integers(-2**10, 2**10, (6, 5)).astype(np.float64)
    r = oz.reuse_gradients(A, B, dC, 14)
    assert np.array_equal(r["dA"], dC @ B.T)
    assert np.array_equal(r["dB"], A.T @ dC)


def test_exponent_rule_margin():
    """2 2^(g - g') R <= P - 1 exactly for R around powers of two, below 1 and huge;
    and one more would break it for most R (the rule wastes at most a bit)."""
    rng = np.random.default_rng(5)
    for N in (6, 12, 20):
        moduli = oz.hybrid_moduli(N)
        P = oz.product_P(moduli)
        Q = oz.reuse_budget_constant(moduli)
        assert Fraction(float(Q)) <= Fraction(math.log2(P - 1) - 1) + Fraction(1, 10**12)
        Rs = [np.float32(2.0**t) for t in range(-20, 40, 3)]
        Rs += [np.nextafter(np.float32(2.0**t), np.float32(np.inf)) for t in range(-10, 30, 5)]
        Rs += [np.nextafter(np.float32(2.0**t), np.float32(0)) for t in range(-10, 30, 5)]
        Rs += [np.float32(v) for v in np.exp(rng.uniform(-30, 60, 60))]
        tight = 0
        for R in Rs:
            d = oz.reuse_exponent(0, R, Q, False)
            assert 2 * Fraction(2) ** d * Fraction(float(R)) <= P - 1, (N, float(R))
            if 2 * Fraction(2) ** (d + 1) * Fraction(float(R)) > P - 1:
                tight += 1
        assert tight >= 0.9 * len(Rs)
    assert oz.reuse_exponent(3, np.float32(5.0), Q, True) == 0
    assert oz.reuse_exponent(3, np.float32(0.0), Q, False) == 3 + math.floor(float(Q))


def test_accuracy_next_to_native_and_fresh():
    """N = 12, normal upstream gradient: within 2x of native FP64 against the exact
    product on sampled entries (the forward's own criterion)."""
    A, B, dC = problem(40, 48, 36, 1.0, 6)
    r = oz.reuse_gradients(A, B, dC, 12)
    worst, worst_nat = 0.0, 0.0
    nat = dC @ B.T
    for i in range(0, 40, 3):
        for hh in range(0, 36, 4):
            ex = oz.exact_dot(dC[i], B[hh])
            ab = float(oz.exact_abs_dot(dC[i], B[hh]))
            worst = max(worst, abs(float(ex - Fraction(float(r["dA"][i, hh])))) / ab)
            worst_nat = max(worst_nat, abs(float(ex - Fraction(float(nat[i, hh])))) / ab)
    assert worst <= 2 * max(worst_nat, 2.0**-53)
    assert worst <= 36 * 2.0**-52


def test_nonfinite_propagation():
    A, B, dC = problem(5, 4, 6, 1.0, 7)
    dC[1, 2] = np.nan
    B[3, 0] = np.inf
    A[2, 4] = -np.inf
    r = oz.reuse_gradients(A, B, dC, 12)
    assert np.isnan(r["dA"][1]).all() and np.isnan(r["dA"][:, 3]).all()
    assert np.isnan(r["dB"][:, 2]).all() and np.isnan(r["dB"][4]).all()
    assert np.isfinite(r["dA"][0, 0]) and np.isfinite(r["dB"][0, 0])


def test_planted_mistakes_are_caught(monkeypatch):
    A, B, dC = problem(8, 7, 9, 1.0, 8)
    moduli = oz.hybrid_moduli(12)
    exact = dC @ B.T

    def run():
        r = oz.reuse_gradients(A, B, dC, 12)
        return np.abs(r["dA"] - exact).max() / np.abs(exact).max()

    assert run() < 1e-15
    orig = oz.dc_integers_for_dA
    # the column exponent added instead of removed
    monkeypatch.setattr(oz, "dc_integers_for_dA", lambda dC_, g, f: orig(dC_, g, -np.asarray(f)))
    assert run() > 1e-6
    monkeypatch.setattr(oz, "dc_integers_for_dA", orig)
    # the per-line shift of the bound maxima dropped: a budget overrun or lost bits
    orig_shift = oz.shifted_row_maxima
    monkeypatch.setattr(oz, "shifted_row_maxima", lambda cbar, shift: orig_shift(cbar, -np.asarray(shift)))
    g_bad = oz.reuse_side_exponents(dC, B * 2.0**40, moduli)[0]
    monkeypatch.setattr(oz, "shifted_row_maxima", orig_shift)
    g_ok = oz.reuse_side_exponents(dC, B * 2.0**40, moduli)[0]
    assert np.any(g_bad > g_ok)  # the planted rule over-spends the budget (condition fails)
