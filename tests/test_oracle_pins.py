"""Pins of three oracle functions that the other CPU tests reach only through each other:
the integer conversion trunc(2^e x) (Eqs. def:A', def:B'), the FP32 log2 of the exponent
rule (Eq. mu-computation, reading R4) and the per-entry route emulated_entry that checks
the full-size GPU results.  Each is compared with values fixed independently of the
oracle (hand-computed closed forms, Python's own int(Fraction) truncation, an 80-digit
decimal logarithm rounded to FP32 here, the oracle's step-by-step method), and for each
a plausible mistake is planted in a copy of the function to show that a pin fails."""
import decimal
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2 as oz

# ----------------------------------------------------------------- trunc(2^e x)

# (x, e, trunc(2^e x)) worked out by hand.  Negative non-integers distinguish truncation
# (toward zero, Eq. def:A') from floor; 2^70-scale results lie beyond 64-bit integers;
# 2^-1074 is the smallest subnormal double.
TRUNC_CLOSED_FORMS = [
    (2.5, 0, 2), (-2.5, 0, -2), (-0.75, 1, -1), (0.75, 1, 1), (-0.5, 0, 0), (0.999, 0, 0),
    (1.5, 3, 12), (-1.375, 2, -5), (1000.0, -3, 125), (-1001.0, -3, -125), (-1000.0, -3, -125),
    (7.0, 0, 7), (-7.0, 0, -7), (1.5, 70, 3 * 2**69), (-(2.0**53 - 1), 20, -(2**53 - 1) * 2**20),
    (5e-324, 1074, 1), (5e-324, 1075, 2), (5e-324, 1073, 0), (-3 * 5e-324, 1073, -1),
    (-3 * 5e-324, 1074, -3), (1.0, -1, 0), (-1.0, -1, 0), (0.0, 50, 0), (-0.0, 50, 0),
    (float("nan"), 3, 0), (float("inf"), 3, 0), (float("-inf"), -3, 0),
    (2.0**-1022, 1022 + 60, 2**60), (-(1 + 2.0**-52), 52, -(2**52 + 1)), (-(1 + 2.0**-52), 51, -(2**51)),
]


def trunc_failures(fn):
    return [(x, e, want, fn(x, e)) for x, e, want in TRUNC_CLOSED_FORMS if fn(x, e) != want]


def test_trunc_scaled_closed_forms():
    assert trunc_failures(oz.trunc_scaled) == []


def test_trunc_scaled_matches_fraction_truncation():
    """int(Fraction) truncates toward zero: an independent route to trunc(2^e x)."""
    rng = np.random.default_rng(11)
    xs = np.concatenate([(rng.random(400) - 0.5) * np.exp(rng.normal(0, 8, 400)),
                         rng.standard_normal(100) * 1e-310, [5e-324, -5e-324, 2.0**-1022]])
    for x in xs:
        for e in (-60, -7, -1, 0, 1, 13, 52, 60, 200, 1100):
            assert oz.trunc_scaled(x, e) == int(Fraction(float(x)) * Fraction(2) ** e), (x, e)


def test_planted_floor_is_caught():
    def floor_scaled(x, e):
        x = float(x)
        if not math.isfinite(x) or x == 0.0:
            return 0
        return math.floor(Fraction(x) * Fraction(2) ** e)

    def dropped_sign(x, e):
        return abs(oz.trunc_scaled(x, e))

    assert trunc_failures(floor_scaled)
    assert trunc_failures(dropped_sign)


def test_integer_rows_and_cols_scale_the_right_lines():
    """Row i of A' uses e_i and column j of B' uses f_j (Eqs. def:A', def:B')."""
    rng = np.random.default_rng(12)
    A = (rng.random((5, 7)) - 0.5) * 10
    B = (rng.random((7, 4)) - 0.5) * 10
    e = np.array([3, -2, 40, 0, 61])
    f = np.array([1, 59, -4, 20])
    Ai = oz.integer_rows(A, e)
    Bi = oz.integer_cols(B, f)
    for i in range(5):
        for h in range(7):
            assert Ai[i, h] == int(Fraction(A[i, h]) * Fraction(2) ** int(e[i]))
    for h in range(7):
        for j in range(4):
            assert Bi[h, j] == int(Fraction(B[h, j]) * Fraction(2) ** int(f[j]))


def test_int64_route_equals_python_integers():
    rng = np.random.default_rng(13)
    A = (rng.random((30, 50)) - 0.5) * np.exp(rng.normal(0, 3, (30, 50)))
    A[0, :5] = [-2.5, 2.5, -0.5, 5e-324, -1e-310]
    A[1, 3] = np.nan
    A[2, 4] = -np.inf
    e = rng.integers(-20, 55, 30)
    e[0] = 0
    want = oz.integer_rows(A, e)
    got = oz.integer_rows_int64(A, e)
    assert got.dtype == np.int64
    assert all(int(got[i, h]) == want[i, h] for i in range(30) for h in range(50))
    f = rng.integers(-5, 50, 50)
    wantc = oz.integer_cols(A, f)
    gotc = oz.integer_cols_int64(A, f)
    assert all(int(gotc[i, h]) == wantc[i, h] for i in range(30) for h in range(50))
    with pytest.raises(ValueError):
        oz.integer_rows_int64(np.array([[1.0]]), np.array([62]))


# ----------------------------------------------------------------- FP32 log2


def log2_f32_reference(x32):
    """Correctly rounded FP32 log2 from an 80-digit decimal logarithm (no oracle code)."""
    decimal.getcontext().prec = 80
    d = decimal.Decimal(float(x32)).ln() / decimal.Decimal(2).ln()
    lo = np.float32(float(d))
    while decimal.Decimal(float(lo)) > d:
        lo = np.nextafter(lo, np.float32(-np.inf))
    while decimal.Decimal(float(np.nextafter(lo, np.float32(np.inf)))) <= d:
        lo = np.nextafter(lo, np.float32(np.inf))
    if decimal.Decimal(float(lo)) == d:
        return lo
    hi = np.nextafter(lo, np.float32(np.inf))
    return lo if d - decimal.Decimal(float(lo)) < decimal.Decimal(float(hi)) - d else hi


def near_midpoint_values(count, seed):
    """float32 x whose log2 lies close to a midpoint between two float32 values: for a
    random float32 y and its midpoint with the next float32, the float32 neighbours of
    2^mid are scanned and the one whose log2 is nearest a midpoint is kept."""
    decimal.getcontext().prec = 80
    rng = np.random.default_rng(seed)
    ln2 = decimal.Decimal(2).ln()
    out = []
    for _ in range(count):
        y = np.float32(rng.uniform(-120, 120))
        mid = (decimal.Decimal(float(y)) + decimal.Decimal(float(np.nextafter(y, np.float32(np.inf))))) / 2
        x0 = np.float32(float((mid * ln2).exp()))
        best, best_d = None, None
        x = x0
        for _ in range(40):
            x = np.nextafter(x, np.float32(-np.inf))
        for _ in range(81):
            d = decimal.Decimal(float(x)).ln() / ln2
            f = np.float32(float(d))
            g = np.nextafter(f, np.float32(np.inf)) if decimal.Decimal(float(f)) < d else \
                np.nextafter(f, np.float32(-np.inf))
            gap = abs(d - (decimal.Decimal(float(f)) + decimal.Decimal(float(g))) / 2) / abs(d)
            if best_d is None or gap < best_d:
                best, best_d = x, gap
            x = np.nextafter(x, np.float32(np.inf))
        out.append(best)
    return out


def log2_failures(fn, xs):
    return [(float(x), fn(x), log2_f32_reference(x)) for x in xs
            if np.float32(fn(x)).view(np.uint32) != np.float32(log2_f32_reference(x)).view(np.uint32)]


def log2_cases():
    rng = np.random.default_rng(21)
    pows = [np.float32(2.0**t) for t in range(-149, 128, 7)] + [np.float32(1.0), np.float32(2.0**127)]
    rand = [np.float32(v) for v in np.exp(rng.uniform(-80, 80, 300))]
    sub = [np.float32(1e-40), np.float32(3e-45), np.float32(1.1754942e-38)]
    return pows, rand + sub, near_midpoint_values(12, 22)


def test_log2_f32_powers_of_two_are_exact():
    for t in range(-149, 128):
        x = np.float32(2.0**t)
        assert oz.log2_f32(x) == np.float32(t), t


def test_log2_f32_matches_decimal_reference():
    pows, rand, near = log2_cases()
    assert log2_failures(oz.log2_f32, pows + rand + near) == []


def test_planted_one_ulp_log2_is_caught():
    pows, rand, near = log2_cases()

    def one_ulp_up(x):
        return np.nextafter(oz.log2_f32(x), np.float32(np.inf))

    def truncating(x):  # the float32 below the double log2 (round toward -inf)
        d = math.log2(float(np.float32(x)))
        r = np.float32(d)
        return np.nextafter(r, np.float32(-np.inf)) if float(r) > d else r

    assert log2_failures(one_ulp_up, pows)
    assert log2_failures(truncating, rand)


# ----------------------------------------------------------------- emulated_entry


def entry_failures(fn, N, seed, shape=(6, 5, 40), phi=1.0):
    m, n, k = shape
    rng = np.random.default_rng(seed)
    A = (rng.random((m, k)) - 0.5) * np.exp(phi * rng.standard_normal((m, k)))
    B = (rng.random((k, n)) - 0.5) * np.exp(phi * rng.standard_normal((k, n)))
    r = oz.ozk2_dgemm(A, B, N)
    moduli = oz.hybrid_moduli(N)
    bad = []
    for i in range(m):
        for j in range(n):
            v, cond = fn(A[i], B[:, j], r["e"][i], r["f"][j], moduli)
            if not cond or np.float64(v).view(np.uint64) != np.float64(r["C"][i, j]).view(np.uint64):
                bad.append((i, j))
    return bad


@pytest.mark.parametrize("N,seed,phi", [(6, 0, 0.5), (12, 1, 1.0), (16, 2, 2.0), (12, 3, 2.0)])
def test_emulated_entry_equals_the_method(N, seed, phi):
    """The per-entry route (exact A'B' then one rounding) equals the oracle's step-by-step
    method (digit planes, residue products, CRT) entry for entry."""
    assert entry_failures(oz.emulated_entry, N, seed, phi=phi) == []


def test_planted_entry_mistakes_are_caught():
    def dropped_sign(a_row, b_col, e_i, f_j, moduli):
        P = oz.product_P(moduli)
        ai = [abs(oz.trunc_scaled(x, int(e_i))) for x in a_row]
        bj = [oz.trunc_scaled(x, int(f_j)) for x in b_col]
        c = sum(x * y for x, y in zip(ai, bj))
        return oz.round_scaled_to_double(c, int(e_i) + int(f_j)), True

    def swapped_exponents(a_row, b_col, e_i, f_j, moduli):
        return oz.emulated_entry(a_row, b_col, f_j, e_i, moduli)

    assert entry_failures(dropped_sign, 12, 1)
    assert entry_failures(swapped_exponents, 12, 1)


def _residue_cases():
    rng = np.random.default_rng(31)
    A = (rng.random((12, 40)) - 0.5) * np.exp(rng.normal(0, 6, (12, 40)))
    A[0, :6] = [-2.5, 2.5, -0.75, 5e-324, -3 * 5e-324, -1.0]
    A[1, 0] = np.nan
    A[1, 1] = -np.inf
    A[2, :] = 0.0
    e = np.array([0, 5, 40, 80, 120, -3, 1, 200, 1074, 30, 60, 63])
    return A, e


@pytest.mark.parametrize("p", [1089, 1024, 961, 529, 513, 511, 509, 503, 499])
def test_scaled_residues_match_python_integers(p):
    """The residue route that never forms a' equals smod of the exact integers, also
    where a' exceeds 64 bits (e up to 1074)."""
    A, e = _residue_cases()
    got = oz.scaled_residues_rows(A, e, p)
    want = oz.smod(oz.integer_rows(A, e), p)
    assert all(int(got[i, h]) == want[i, h] for i in range(A.shape[0]) for h in range(A.shape[1]))


def test_planted_floor_shift_in_residues_is_caught():
    """A floor (arithmetic) shift instead of truncation for the scaled-down entries."""
    A, e = _residue_cases()
    p = 513

    def floor_shift(A, e, p):
        x = np.where(np.isfinite(A), A, 0.0)
        frac, E = np.frexp(x)
        M = np.ldexp(frac, 53).astype(np.int64)
        s = E.astype(np.int64) - 53 + np.asarray(e).reshape(-1, 1)
        pow2 = np.array([pow(2, t, p) for t in range(max(int(s.max()), 0) + 1)], dtype=np.int64)
        up = s >= 0
        return np.where(up, oz.smod(oz.smod(M, p) * pow2[np.where(up, s, 0)], p),
                        oz.smod(M >> np.minimum(np.where(up, 0, -s), 63), p))

    want = oz.smod(oz.integer_rows(A, e), p)
    got = floor_shift(A, e, p)
    assert any(int(got[i, h]) != want[i, h] for i in range(A.shape[0]) for h in range(A.shape[1]))
