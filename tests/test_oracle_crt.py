"""Pins for residue products, CRT reconstruction and the final rounding.

Residue products C'_l = mod(A'_l B'_l, p_l) are uniquely defined (Eq. CRTmatmul);
the oracle's digit-product route (Eqs. 3matmult-notKaratsuba, C'-Karatsuba) is
compared with the direct big-integer product.  CRT (Eq. CRT_finalreduction)
must return A'B' exactly whenever Eq. condition holds (brute force on tiny
inputs, every N).  Rounding (Eq. inversescaling) is checked on closed-form
cases and against Python's correctly rounded Fraction -> float conversion.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz


def gen(shape, phi, rng):
    return (rng.random(shape) - 0.5) * np.exp(phi * rng.standard_normal(shape))


@pytest.mark.parametrize("N", list(range(1, 21)))
def test_crt_identity(N):
    moduli = oz.hybrid_moduli(N)
    w, P = oz.crt_weights(moduli)
    for l, wl in enumerate(w):
        assert 0 <= wl < P
        for mi, pm in enumerate(moduli):
            assert wl % pm == (1 if l == mi else 0)


@pytest.mark.parametrize("N", [1, 3, 6, 7, 12, 20])
def test_crt_roundtrip_random_integers(N):
    moduli = oz.hybrid_moduli(N)
    P = oz.product_P(moduli)
    rng = np.random.default_rng(N)
    xs = [int(rng.integers(0, 2**62)) * (P // 2**62 + 1) % P - P // 2 for _ in range(200)]
    xs += [-(P // 2), P - 1 - P // 2, 0, 1, -1]
    X = np.array(xs, dtype=object).reshape(1, -1)
    res = [np.array(oz.smod(X, p).astype(np.int64)) for p in moduli]
    back = oz.crt_reconstruct(res, moduli)
    assert list(back.flat) == xs


@pytest.mark.parametrize("N", list(range(1, 21)))
def test_tiny_brute_force_crt_equals_exact_product(N):
    """Route (i) (digits -> residue products -> CRT) equals route (ii) (A'B' in Python ints)."""
    rng = np.random.default_rng(100 + N)
    m, k, n = int(rng.integers(1, 8)), int(rng.integers(1, 8)), int(rng.integers(1, 8))
    A, B = gen((m, k), 1.0, rng), gen((k, n), 1.0, rng)
    r = oz.ozk2_dgemm(A, B, N, keep=True)
    P = oz.product_P(r["moduli"])
    for i in range(m):
        for j in range(n):
            assert oz.condition_lhs_entry(r["Aint"], r["Bint"], i, j) < P
            ex = oz.exact_integer_product_entry(r["Aint"], r["Bint"], i, j)
            assert r["Cint"][i, j] == ex
            for p, Cl in zip(r["moduli"], r["residues"]):
                assert Cl[i, j] == oz.smod(ex, p)


def test_residue_products_equal_direct_definition():
    rng = np.random.default_rng(7)
    A, B = gen((24, 70), 2.0, rng), gen((70, 19), 2.0, rng)
    r = oz.ozk2_dgemm(A, B, 14, keep=True)
    Ai, Bi = r["Aint"], r["Bint"]
    direct = Ai.dot(Bi)
    for p, Cl in zip(r["moduli"], r["residues"]):
        want = oz.smod(direct, p).astype(np.int64)
        assert np.array_equal(Cl, want)


def _planted(monkeypatch, fn):
    monkeypatch.setattr(oz, "residue_product", fn)


@pytest.mark.parametrize("mistake", ["drop_cross_term", "karatsuba_sign", "transpose"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    """Plausible mistakes in the digit-product formulas break the exact comparison."""
    orig = oz.residue_product

    def bad(planesA, planesB, p):
        kind, s = oz.modulus_kind(p)
        if mistake == "drop_cross_term" and kind == "square":
            A1, A2 = planesA
            B1, B2 = planesB
            return oz.smod(s * oz._int_matmul(A1, B2) + oz._int_matmul(A2, B2), p)
        if mistake == "karatsuba_sign" and kind == "karatsuba":
            C1 = oz._int_matmul(planesA[0], planesB[0])
            C2 = oz._int_matmul(planesA[1], planesB[1])
            C3 = oz._int_matmul(planesA[2], planesB[2])
            return oz.smod(s * s * C1 + C2 + s * (C3 - C1 + C2), p)
        if mistake == "transpose":
            return orig(planesA, [x.T.copy() for x in planesB], p)
        return orig(planesA, planesB, p)

    rng = np.random.default_rng(11)
    A, B = gen((9, 9), 1.0, rng), gen((9, 9), 1.0, rng)
    _planted(monkeypatch, bad)
    r = oz.ozk2_dgemm(A, B, 12, keep=True)
    direct = r["Aint"].dot(r["Bint"])
    mism = sum(int(not np.array_equal(Cl, oz.smod(direct, p).astype(np.int64)))
               for p, Cl in zip(r["moduli"], r["residues"]))
    assert mism > 0


def test_rounding_closed_forms():
    f = oz.round_scaled_to_double
    assert f(2**53 + 1, 0) == 2.0**53  # tie to even (down)
    assert f(2**53 + 3, 0) == 2.0**53 + 4  # tie to even (up)
    assert f(-(2**53 + 3), 0) == -(2.0**53 + 4)
    assert f(3, 1075) == 2 * 5e-324  # 1.5 * 2^-1074 ties to 2 * 2^-1074
    assert f(1, 1075) == 0.0  # 0.5 * 2^-1074 ties to 0
    assert f(3, 1076) == 5e-324  # 0.75 * 2^-1074 rounds up
    assert f(1, -1024) == math.inf
    assert f(-1, -1024) == -math.inf
    assert f(2**53 - 1, -971) == float.fromhex("0x1.fffffffffffffp+1023")
    assert f(0, 5) == 0.0
    assert f(12345, -3) == 12345 * 8.0


def test_rounding_matches_fraction_conversion():
    rng = np.random.default_rng(12)
    for _ in range(3000):
        c = int(rng.integers(-(2**62), 2**62)) * int(rng.integers(1, 2**50))
        s = int(rng.integers(-900, 1300))
        want = float(Fraction(c, 1) / Fraction(2) ** s) if s >= 0 else float(Fraction(c * 2 ** (-s)))
        assert oz.round_scaled_to_double(c, s) == want
