"""Plain CPU oracle of FP8 Ozaki-II DGEMM emulation (arXiv:2603.10634).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` are the only callers.  The CUDA
library never imports, links or calls anything here, and this module imports
nothing from the library: it regenerates its own moduli, constants and CRT
weights from the paper's definitions.

What is computed (paper section / equation in brackets):

  1. preliminary scales  e'_i = 7 - floor(log2 max_h |a_ih|)       [Sec. III-E, Eq. def:mu'nu']
     and the bound operands Abar = RU_E4M3(2^e' |A|)                [Sec. III-E]
  2. the bound product  Cbar' = Abar Bbar  (FP32), Cbar = RU((1+k 2^-24) Cbar')
                                                                    [Sec. III-E, Eq. barCupper]
  3. final exponents  e_i = e'_i + int(P' + delta log2 max_j cbar_ij)  [Eq. mu-computation]
  4. integer matrices  A' = trunc(diag(2^e) A),  B' = trunc(B diag(2^f))  [Eqs. def:A', def:B']
  5. residues A'_l = mod(A', p_l) and their FP8 digits              [Sec. III-B, III-C, III-D]
  6. residue products C'_l = mod(A'_l B'_l, p_l) from three digit products
                                                 [Eqs. 3matmult-notKaratsuba, C'-Karatsuba]
  7. CRT  C' = mod(sum_l q_l P/p_l C'_l, P)                          [Eq. CRT_finalreduction]
  8. inverse scaling  C = diag(2^-e) C' diag(2^-f), rounded once to FP64  [Eq. inversescaling]

Integers are exact Python ints (numpy object arrays) or int64 where the
magnitude bound is stated.  Floating point appears only where the paper fixes
FP32 (steps 2-3); there each rounding is done from the exact rational value with
an explicit direction, so nothing depends on the host's rounding mode.

Readings taken where the paper is silent or ambiguous:
  R1  Abar uses |A| (the bound derivation needs absolute values).
  R2  The exponent rule of Eq. mu-computation is followed literally; the garbled
      inequality printed just before it is not used.
  R3  "int(.)" is floor (its argument is positive for every non-degenerate row).
  R4  log2 in step 3 is the correctly rounded FP32 log2 of the FP32 value; P' +
      delta*log2 is evaluated as RD(P' + RD(delta*log2)) (two round-down ops).
  R5  Cbar' (computed on the GPU with some FP32 accumulation order) is taken here
      as RN_fp32 of the exact product, which is one admissible FP32 result; the
      factor is RU_fp32(1 + k 2^-24) and the scaling of Cbar' is rounded up.
  R6  A zero row (column) gets e' = 0 and e = 0.  A nonzero row whose bound row
      maximum is 0 gets e = e' + floor(P').
  R7  RU to E4M3 maps every positive value below 2^-9 to 2^-9; zero stays zero.
  R8  smod(x, p) returns the representative in [-floor(p/2), p - 1 - floor(p/2)]
      (for even p the interval is [-p/2, p/2 - 1]).
  R9  round() in the square-modulus split rounds half to even.
  R10 Non-finite entries are treated as 0 for scaling and residues; every output
      in a row of A or a column of B holding one is NaN.
  R11 The final value is RN-even of the exact rational C' 2^-(e_i+f_j), with
      gradual underflow and overflow to +-inf.
  R15 Fast mode (Sec. III-E gives no formula): the bound of a row is the FP32 round-up
      of sum_h RU_fp32(2^e' |a_ih|)^2, an upper bound of ||2^e' a_i||^2, and the
      exponent rule of Eq. mu-computation is applied to it in place of max_j cbar_ij;
      then 2 mu_i nu_j ||a_i|| ||b_j|| <= P - 1 as in accurate mode.
"""

from __future__ import annotations

import math
from bisect import bisect_left
from fractions import Fraction
from math import gcd

import numpy as np

# --------------------------------------------------------------------------
# Moduli  [Sec. II Eq. p_list; Sec. III-B Eq. p_list_karatsuba; Sec. III-D Eq. p_list_hybrid]
# --------------------------------------------------------------------------


def _greedy_coprime_descending(start, chosen, count):
    """Scan integers downward from ``start`` and keep each one that is coprime
    to everything kept so far, until ``count`` numbers are held."""
    out = list(chosen)
    c = start
    while len(out) < count and c >= 2:
        if all(gcd(c, q) == 1 for q in out):
            out.append(c)
        c -= 1
    return out


def int8_moduli(N):
    """INT8 Ozaki-II list: greedy pairwise-coprime integers from 256 down [Sec. II]."""
    return _greedy_coprime_descending(256, [], N)


def karatsuba_moduli(N):
    """Karatsuba-only FP8 list: greedy pairwise-coprime integers from 513 down [Sec. III-B]."""
    return _greedy_coprime_descending(513, [], N)


def direct_fp8_moduli():
    """Candidates p <= 32 for a direct FP8 encoding [Sec. III-A]: greedy coprime from 32."""
    return _greedy_coprime_descending(32, [], 10**9)


def hybrid_squares():
    """Pairwise-coprime squares taken in descending order from 33^2 = 1089 [Sec. III-D]."""
    out = []
    s = 33
    while s >= 2:
        if all(gcd(s * s, q) == 1 for q in out):
            out.append(s * s)
        s -= 1
    return out


def hybrid_moduli(N):
    """Hybrid list [Sec. III-D]: the squares 1089, 1024, 961, 841, 625, 529 first, then
    greedy pairwise-coprime integers downward from 513.  For N < 34 (the range used
    by the method) the squares are exactly the first six entries."""
    squares = hybrid_squares()[:6]
    if N <= 6:
        return squares[:N]
    return _greedy_coprime_descending(513, squares, N)


def hybrid_moduli_full():
    """The whole hybrid list (all entries down to 2), for the bound printed in Sec. III-D."""
    return _greedy_coprime_descending(513, hybrid_squares()[:6], 10**9)


def modulus_kind(p):
    """('square', s) when p = s^2 is one of the hybrid squares, else ('karatsuba', 16)
    [Sec. III-D: squares use the reduction of Sec. III-C, the rest use Sec. III-B]."""
    s = math.isqrt(p)
    if s * s == p and p in hybrid_squares()[:6]:
        return "square", s
    return "karatsuba", 16


def num_digit_planes(N):
    """M_N, the number of FP8 planes per operand [Sec. IV-B Eq. M]."""
    return 2 * N if N <= 6 else 3 * N - 6


def num_fp8_gemms(N, mode="accurate"):
    """FP8 matrix products per emulated DGEMM [Sec. IV-A Table 2]: 3N (+1 bound product)."""
    return 3 * N + (1 if mode == "accurate" else 0)


def product_P(moduli):
    P = 1
    for p in moduli:
        P *= p
    return P


# --------------------------------------------------------------------------
# Symmetric modulo and digit splits  [Sec. II; Sec. III-B; Sec. III-D]
# --------------------------------------------------------------------------


def smod(x, p):
    """Symmetric remainder (reading R8): the y = x (mod p) with -floor(p/2) <= y < p - floor(p/2).
    Works on Python ints, int64 arrays and object arrays."""
    h = p // 2
    return (x + h) % p - h


def split_square(r, s):
    """Square modulus p = s^2 [Sec. III-D]: d1 = round(r/s) (half to even, R9), d2 = r - s d1."""
    d1 = round(Fraction(int(r), int(s)))
    return d1, int(r) - s * d1


def split_karatsuba(r, s=16):
    """Karatsuba split [Sec. III-B]: d1 = sign(r) ceil(|r|/s), d2 = r - s d1, d3 = d1 + d2."""
    r = int(r)
    sign = (r > 0) - (r < 0)
    d1 = sign * (-(-abs(r) // s))
    d2 = r - s * d1
    return d1, d2, d1 + d2


def split_digits(r, p):
    kind, s = modulus_kind(p)
    return split_square(r, s) if kind == "square" else split_karatsuba(r, s)


# --------------------------------------------------------------------------
# FP8 E4M3  (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; 0x7F/0xFF are NaN)
# --------------------------------------------------------------------------


def e4m3_value(code):
    """Exact value of an E4M3 code as a Fraction (None for NaN)."""
    code = int(code) & 0xFF
    sign = -1 if code & 0x80 else 1
    ex = (code >> 3) & 0xF
    man = code & 0x7
    if ex == 0xF and man == 0x7:
        return None
    if ex == 0:
        return sign * Fraction(man, 1 << 9)  # subnormal: man * 2^-9
    return sign * Fraction(8 + man, 8) * Fraction(2) ** (ex - 7)


# the 127 finite non-negative values with their codes, sorted by value
_E4M3_POS = [(e4m3_value(c), c) for c in range(0x7F)]
_E4M3_POS_VALUES = [v for v, _ in _E4M3_POS]


def e4m3_round_up_code(x):
    """RU_E4M3(x) for a finite x >= 0: the code of the least E4M3 value >= x.  Values
    above 0 and below 2^-9 go to 2^-9 (reading R7).  x may be a float or Fraction."""
    fx = Fraction(x)
    if fx < 0:
        raise ValueError("e4m3_round_up_code expects x >= 0")
    i = bisect_left(_E4M3_POS_VALUES, fx)
    if i == len(_E4M3_POS_VALUES):
        raise OverflowError("value above the E4M3 maximum 448")
    return _E4M3_POS[i][1]


def e4m3_code_of_integer(d):
    """Code of an integer |d| <= 16 (exactly representable) [Sec. III-A]."""
    d = int(d)
    for v, c in _E4M3_POS:
        if v == abs(d):
            return c | (0x80 if d < 0 else 0)
    raise ValueError(f"{d} is not an E4M3 integer")


# --------------------------------------------------------------------------
# FP32 rounding from exact rationals (for the FP32 steps the paper prescribes)
# --------------------------------------------------------------------------


def _f32_neighbors(q):
    """The two float32 values bracketing the rational q: (lo, hi) with lo <= q <= hi."""
    f = np.float32(float(q))  # some nearby float32
    while Fraction(float(f)) > q:
        f = np.nextafter(f, np.float32(-np.inf))
    lo = f
    while Fraction(float(lo)) < q:
        nxt = np.nextafter(lo, np.float32(np.inf))
        if Fraction(float(nxt)) > q:
            break
        lo = nxt
    hi = lo if Fraction(float(lo)) == q else np.nextafter(lo, np.float32(np.inf))
    return lo, hi


def f32_round_down(q):
    return _f32_neighbors(Fraction(q))[0]


def f32_round_up(q):
    return _f32_neighbors(Fraction(q))[1]


def f32_round_nearest(q):
    q = Fraction(q)
    lo, hi = _f32_neighbors(q)
    if lo == hi:
        return lo
    dlo, dhi = q - Fraction(float(lo)), Fraction(float(hi)) - q
    if dlo < dhi:
        return lo
    if dhi < dlo:
        return hi
    return lo if (int(np.float32(lo).view(np.uint32)) & 1) == 0 else hi


# --------------------------------------------------------------------------
# Accurate-mode scaling  [Sec. III-E]
# --------------------------------------------------------------------------


def ufp_exponent(x):
    """floor(log2 |x|) for a finite nonzero double, exactly (ufp(x) = 2^that) [Sec. III-E]."""
    m, ex = math.frexp(abs(float(x)))  # |x| = m 2^ex, 0.5 <= m < 1
    return ex - 1


def delta_constant():
    """delta = RD_fp32(-1/(2 - 2^-21))  [Sec. III-E]."""
    return f32_round_down(Fraction(-1) / (2 - Fraction(1, 1 << 21)))


def _log2_int_high_precision(n, bits=200):
    """log2 of a positive int to about ``bits`` bits: bit_length plus a binary expansion
    of the log of the leading part computed by repeated squaring (exact rationals)."""
    L = n.bit_length() - 1
    # mantissa y in [1, 2) as an exact fraction
    y = Fraction(n, 1 << L)
    frac = Fraction(0)
    step = Fraction(1, 2)
    for _ in range(bits):
        y = y * y
        # keep y bounded in size: truncate to 400 bits of precision (error << 2^-200)
        if y.denominator.bit_length() > 420:
            num = (y.numerator << 400) // y.denominator
            y = Fraction(num, 1 << 400)
        if y >= 2:
            y /= 2
            frac += step
        step /= 2
    return Fraction(L) + frac


def p_prime_constant(moduli):
    """P' = RD_fp32((log2(P-1) - 1)/2)  [Sec. III-E]; log2(P-1) is evaluated to ~200 bits."""
    P = product_P(moduli)
    return f32_round_down((_log2_int_high_precision(P - 1) - 1) / 2)


def prelim_exponent_rows(A):
    """e'_i = 7 - floor(log2 max_h |a_ih|) [Eq. def:mu'nu']; 0 for a zero row (R6).
    Non-finite entries count as 0 (R10).  Returns an int64 array."""
    m = A.shape[0]
    out = np.zeros(m, dtype=np.int64)
    for i in range(m):
        row = A[i]
        row = np.where(np.isfinite(row), np.abs(row), 0.0)
        mx = float(row.max()) if row.size else 0.0
        out[i] = 0 if mx == 0.0 else 7 - ufp_exponent(mx)
    return out


def bound_operand(A, eprime):
    """Abar_ih = RU_E4M3(2^e'_i |a_ih|) as uint8 codes (m x k) [Sec. III-E, R1, R7].

    v = ldexp(|a|, e') is exact whenever v >= 2^-1022 and never overflows (v < 2^8
    because e' comes from the row maximum).  A v that ldexp rounds lies far below
    2^-9 and maps to code 1 like every other positive value there.  The code is the
    index of the least E4M3 value >= v in the sorted list of non-negative values."""
    A = np.asarray(A, dtype=np.float64)
    a = np.where(np.isfinite(A), np.abs(A), 0.0)
    v = np.ldexp(a, np.asarray(eprime, dtype=np.int64)[:, None].astype(np.int32))
    table = np.array([float(x) for x in _E4M3_POS_VALUES], dtype=np.float64)
    idx = np.searchsorted(table, v, side="left")
    codes = np.array([c for _, c in _E4M3_POS], dtype=np.uint8)[np.minimum(idx, len(table) - 1)]
    if np.any(idx >= len(table)):
        raise OverflowError("scaled value above the E4M3 maximum")
    codes = np.where(a > 0, np.maximum(codes, 1), 0).astype(np.uint8)
    return codes


def e4m3_decode_array(codes):
    """float64 values of an array of non-negative E4M3 codes (exact)."""
    lut = np.array([float(e4m3_value(c)) if e4m3_value(c) is not None else np.nan
                    for c in range(256)], dtype=np.float64)
    return lut[np.asarray(codes, dtype=np.int64)]


def bound_product(Abar, Bbar, k):
    """cbar = RU_fp32(RU_fp32(1 + k 2^-24) * Cbar'), Cbar' = RN_fp32(Abar Bbar)  [Eq. barCupper, R5].

    Abar is m x k and Bbar is k x n (codes).  The float64 matmul is exact: every
    product is a multiple of 2^-18 below 2^16, so each partial sum of k <= 2^19
    terms is a multiple of 2^-18 below 2^35 and fits in 53 bits.  numpy's float64 ->
    float32 cast rounds to nearest even.  The product of two float32 values is exact
    in float64 (48 significant bits), and its round-up to float32 is the RN result
    moved one step up whenever RN fell below the exact value."""
    if k > (1 << 19):
        raise ValueError("bound_product exactness argument needs k <= 2^19")
    exact = e4m3_decode_array(Abar) @ e4m3_decode_array(Bbar)
    c1 = exact.astype(np.float32)
    factor = f32_round_up(1 + Fraction(k, 1 << 24))
    prod = np.float64(factor) * c1.astype(np.float64)
    r = prod.astype(np.float32)
    below = r.astype(np.float64) < prod
    r[below] = np.nextafter(r[below], np.float32(np.inf))
    return r


def log2_f32(x):
    """Correctly rounded FP32 log2 of a positive float32 (reading R4).

    math.log2 is within one double ulp of log2(x); rounding it to float32 is then the
    correctly rounded result unless it sits within 2^-40 (relative) of the midpoint
    between two float32 neighbours, in which case the midpoint is decided exactly."""
    x = float(np.float32(x))
    d = math.log2(x)
    r = np.float32(d)
    lo, hi = _f32_neighbors(Fraction(d))
    if lo == hi:
        return lo
    mid = (Fraction(float(lo)) + Fraction(float(hi))) / 2
    if abs(Fraction(d) - mid) > abs(mid) * Fraction(1, 1 << 40) + Fraction(1, 1 << 80):
        return r
    # exact decision: log2 x < mid  <=>  x < 2^mid, compared via a high-precision log
    return lo if _log2_fraction(Fraction(x), 120) < mid else hi


def _log2_fraction(q, bits=80):
    q = Fraction(q)
    num = q.numerator << 256
    return _log2_int_high_precision(num // q.denominator, bits) - 256


def final_exponent(eprime, rmax, pprime, delta, row_is_zero):
    """e = e' + floor(RD(P' + RD(delta * log2 rmax)))  [Eq. mu-computation, R2-R4, R6]."""
    if row_is_zero:
        return 0
    if rmax == 0:
        return int(eprime) + math.floor(float(pprime))
    L = log2_f32(rmax)
    t1 = f32_round_down(Fraction(float(delta)) * Fraction(float(L)))
    t2 = f32_round_down(Fraction(float(pprime)) + Fraction(float(t1)))
    return int(eprime) + math.floor(float(t2))


def sum_of_squares_bound(X, eprime):
    """Fast-mode line norms (reading R15): s_i = RU_fp32(sum_h v_ih^2) with
    v_ih = RU_fp32(2^e'_i |x_ih|), computed exactly (v^2 as an exact rational, the sum in
    Python integers) and rounded up once.  ||2^e'_i x_i||_2^2 <= s_i."""
    m, k = X.shape
    out = np.zeros(m, dtype=np.float32)
    for i in range(m):
        sc = Fraction(2) ** int(eprime[i])
        total = Fraction(0)
        for h in range(k):
            a = float(X[i, h])
            if a == 0.0 or not math.isfinite(a):
                continue
            v = Fraction(float(f32_round_up(Fraction(abs(a)) * sc)))
            total += v * v
        out[i] = f32_round_up(total) if total else np.float32(0.0)
    return out


def scaling_exponents(A, B, N, moduli=None, mode="accurate"):
    """Exponents (e for the rows of A, f for the columns of B) and the intermediate
    quantities.  accurate: the FP8 bound product of Sec. III-E (workflow steps 1-3 of
    Sec. IV-B).  fast: the Cauchy-Schwarz bound of Sec. III-E, 2 sum |a'||b'| <=
    2 mu nu ||a_i|| ||b_j||, with the same exponent rule applied to the squared norms
    (reading R15)."""
    moduli = hybrid_moduli(N) if moduli is None else moduli
    k = A.shape[1]
    Af = np.where(np.isfinite(A), A, 0.0)
    Bf = np.where(np.isfinite(B), B, 0.0)
    ep = prelim_exponent_rows(Af)
    fp = prelim_exponent_rows(Bf.T)
    pprime = p_prime_constant(moduli)
    delta = delta_constant()
    m, n = A.shape[0], B.shape[1]
    if mode == "fast":
        Abar = Bbar = cbar = None
        R = sum_of_squares_bound(Af, ep)
        S = sum_of_squares_bound(Bf.T, fp)
    else:
        Abar = bound_operand(Af, ep)
        Bbar = bound_operand(Bf.T, fp).T  # k x n
        cbar = bound_product(Abar, Bbar, k)
        R = cbar.max(axis=1) if n else np.zeros(m, np.float32)
        S = cbar.max(axis=0) if m else np.zeros(n, np.float32)
    zero_row = ~np.any(Af != 0, axis=1)
    zero_col = ~np.any(Bf != 0, axis=0)
    e = np.array([final_exponent(ep[i], R[i], pprime, delta, zero_row[i]) for i in range(m)],
                 dtype=np.int64)
    f = np.array([final_exponent(fp[j], S[j], pprime, delta, zero_col[j]) for j in range(n)],
                 dtype=np.int64)
    ep = np.where(zero_row, 0, ep)
    fp = np.where(zero_col, 0, fp)
    return dict(e=e, f=f, eprime=ep, fprime=fp, Abar=Abar, Bbar=Bbar, cbar=cbar, R=R, S=S,
                pprime=pprime, delta=delta)


# --------------------------------------------------------------------------
# Integer conversion  [Eqs. def:A', def:B']
# --------------------------------------------------------------------------


def trunc_scaled(x, e):
    """trunc(2^e x) as an exact Python int for a finite double x (0 for non-finite, R10)."""
    x = float(x)
    if not math.isfinite(x) or x == 0.0:
        return 0
    num, den = x.as_integer_ratio()  # x = num/den exactly, den a power of two
    if e >= 0:
        num <<= e
    else:
        den <<= -e
    q = abs(num) // den
    return q if num > 0 else -q


def integer_rows(A, e):
    """A' = trunc(diag(2^e) A) as an object array of Python ints [Eq. def:A']."""
    m, k = A.shape
    out = np.empty((m, k), dtype=object)
    for i in range(m):
        ei = int(e[i])
        for h in range(k):
            out[i, h] = trunc_scaled(A[i, h], ei)
    return out


def integer_cols(B, f):
    """B' = trunc(B diag(2^f)) as an object array of Python ints [Eq. def:B']."""
    return integer_rows(B.T, f).T


INT64_SAFE = float(2**62)


def integer_rows_int64(A, e):
    """A' = trunc(diag(2^e) A) [Eq. def:A'] as an int64 array, for inputs whose scaled
    entries all stay below 2^62 in magnitude (raises ValueError otherwise; integer_rows
    has no such limit).  Non-finite entries give 0 (R10).

    For a finite double a, ldexp(a, e) = 2^e a exactly whenever the result is at least 1
    in magnitude (it is then a normal double and only the exponent changes); a result
    below 1 in magnitude, rounded or not, truncates to 0.  np.trunc is exact, and values
    below 2^62 convert to int64 exactly."""
    A = np.asarray(A, dtype=np.float64)
    x = np.where(np.isfinite(A), A, 0.0)
    ex = np.asarray(e, dtype=np.int64).reshape(-1, 1)
    v = np.ldexp(x, ex.astype(np.int32))
    if v.size and not np.all(np.abs(v) < INT64_SAFE):
        raise ValueError("a scaled entry reaches 2^62: use integer_rows")
    return np.trunc(v).astype(np.int64)


def integer_cols_int64(B, f):
    """B' = trunc(B diag(2^f)) [Eq. def:B'] as int64 (see integer_rows_int64)."""
    return integer_rows_int64(np.asarray(B, dtype=np.float64).T, f).T


# --------------------------------------------------------------------------
# Residues, digit planes and residue products
# [Sec. II Eq. CRTmatmul; Sec. III-B Eqs. Karatsuba, C'-Karatsuba; Sec. III-C Eq. 3matmult]
# --------------------------------------------------------------------------


def residue_matrix(Xint, p):
    """mod(X', p) (symmetric, R8) as int64."""
    return np.array(smod(Xint, p), dtype=np.int64) if Xint.size else np.zeros(Xint.shape, np.int64)


def scaled_decomposition(A, e):
    """(M, s) with 2^e_i a_ih = M_ih 2^s_ih exactly, M an integer of magnitude below 2^53
    (np.frexp scaled by 2^53) and s = E + e_i; non-finite entries count as 0 (R10)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.where(np.isfinite(A), A, 0.0)
    frac, E = np.frexp(x)  # x = frac 2^E, 0.5 <= |frac| < 1 (frac = 0 for x = 0)
    M = np.ldexp(frac, 53).astype(np.int64)
    s = E.astype(np.int64) - 53 + np.asarray(e, dtype=np.int64).reshape(-1, 1)
    return M, s


def residues_of_decomposition(M, s, p):
    """smod(trunc(M 2^s), p) for the (M, s) of scaled_decomposition: for s >= 0 the value
    is the integer M 2^s and its residue is smod(smod(M, p) (2^s mod p), p); for s < 0,
    trunc(M 2^s) = sign(M) (|M| >> -s) lies below 2^53 and is reduced directly."""
    smax = int(s.max()) if s.size else 0
    pow2 = np.array([pow(2, t, p) for t in range(max(smax, 0) + 1)], dtype=np.int64)
    up = s >= 0
    r_up = smod(smod(M, p) * pow2[np.where(up, s, 0)], p)
    q = np.abs(M) >> np.minimum(np.where(up, 0, -s), 63)
    r_down = smod(np.sign(M) * q, p)
    return np.where(up, r_up, r_down).astype(np.int64)


def scaled_residues_rows(A, e, p):
    """smod(trunc(2^e_i a_ih), p) [Eqs. def:A', CRTmatmul] as int64, without forming the
    integers a' (they exceed 64 bits for large N): a finite double is M 2^E with an
    integer |M| < 2^53, so 2^e a = M 2^(E + e) and its truncation's residue follows from
    M and the power of two alone (residues_of_decomposition)."""
    return residues_of_decomposition(*scaled_decomposition(A, e), p)


def digit_split(r, p):
    """The FP8 digit planes of residues r (int64, symmetric mod p) as int64 arrays of
    integers in [-16, 16]: two planes (d1, d2) for a square modulus, three (d1, d2, d3)
    for a Karatsuba one [Sec. III-B, III-D]."""
    r = np.asarray(r, dtype=np.int64)
    kind, s = modulus_kind(p)
    if kind == "square":
        # round half to even of r/s (R9).  r/s is a half-integer only for even s (= 32),
        # where the division is exact; for odd s it is at least 1/(2s) away from any
        # half-integer, far more than the double division error, so np.rint is exact.
        d1 = np.rint(r.astype(np.float64) / s).astype(np.int64)
        return [d1, r - s * d1]
    sign = np.sign(r)
    d1 = sign * ((np.abs(r) + (s - 1)) // s)
    d2 = r - s * d1
    return [d1, d2, d1 + d2]


def digit_planes(Xint, p):
    """The FP8 digit planes of X' for modulus p (digit_split of mod(X', p))."""
    return digit_split(residue_matrix(Xint, p), p)


def _int_matmul(X, Y):
    """Exact integer product of two int64 matrices with entries in [-16, 16], through
    float64 BLAS: every partial sum is an integer of magnitude <= 256 k <= 2^53."""
    if X.shape[1] > (1 << 45):
        raise ValueError("digit products exceed the float64 exactness range")
    return np.rint(X.astype(np.float64) @ Y.astype(np.float64)).astype(np.int64)


def residue_product(planesA, planesB, p):
    """C'_l = mod(A'_l B'_l, p) from the digit planes.

    square p = s^2   : smod(s A1 B2 + s A2 B1 + A2 B2, p)          [Eq. 3matmult-notKaratsuba]
    Karatsuba (s=16) : smod(s^2 C1 + C2 + s (C3 - C1 - C2), p),  Cx = Ax Bx  [Eq. C'-Karatsuba]
    planesA are m x k, planesB are k x n."""
    kind, s = modulus_kind(p)
    if kind == "square":
        A1, A2 = planesA
        B1, B2 = planesB
        v = s * _int_matmul(A1, B2) + s * _int_matmul(A2, B1) + _int_matmul(A2, B2)
    else:
        C1 = _int_matmul(planesA[0], planesB[0])
        C2 = _int_matmul(planesA[1], planesB[1])
        C3 = _int_matmul(planesA[2], planesB[2])
        v = s * s * C1 + C2 + s * (C3 - C1 - C2)
    return smod(v, p)


# --------------------------------------------------------------------------
# CRT and inverse scaling  [Eqs. CRT_finalreduction, inversescaling]
# --------------------------------------------------------------------------


def crt_weights(moduli):
    """w_l = q_l P / p_l with q_l P/p_l = 1 (mod p_l), reduced mod P; returns (w, P)."""
    P = product_P(moduli)
    w = []
    for p in moduli:
        Pl = P // p
        q = pow(Pl % p, -1, p)
        w.append((q * Pl) % P)
    return w, P


def crt_reconstruct(residues, moduli):
    """C' = smod(sum_l w_l C'_l, P) as an object array of Python ints."""
    w, P = crt_weights(moduli)
    acc = np.zeros(residues[0].shape, dtype=object)
    acc[...] = 0
    for wl, r in zip(w, residues):
        acc = acc + wl * r.astype(object)
    return smod(acc, P)


def round_scaled_to_double(c, s):
    """RN-even of the exact rational c * 2^-s as a Python float (R11).  Python's int/int
    true division and float(int) are correctly rounded, with gradual underflow."""
    c = int(c)
    if c == 0:
        return 0.0
    try:
        if s >= 0:
            return c / (1 << s)
        return float(c << (-s))
    except OverflowError:
        return math.copysign(math.inf, c)


def unscale(Cint, e, f):
    """C = diag(2^-e) C' diag(2^-f), each entry rounded once to FP64 [Eq. inversescaling, R11]."""
    m, n = Cint.shape
    out = np.empty((m, n), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            out[i, j] = round_scaled_to_double(Cint[i, j], int(e[i]) + int(f[j]))
    return out


# --------------------------------------------------------------------------
# The whole method
# --------------------------------------------------------------------------


def nonfinite_masks(A, B):
    return ~np.all(np.isfinite(A), axis=1), ~np.all(np.isfinite(B), axis=0)


def ozk2_dgemm(A, B, N, e=None, f=None, keep=False, mode="accurate"):
    """Emulated C = A B with N hybrid moduli in accurate mode.

    A is m x k, B is k x n (float64).  ``e``/``f`` inject row/column exponents (for
    parity against a GPU that made its own FP32 rounding choices in step 2); when
    omitted they are computed by ``scaling_exponents``.  Returns a dict with C and,
    with keep=True, every intermediate."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    moduli = hybrid_moduli(N)
    out = {"moduli": moduli}
    if e is None or f is None:
        sc = scaling_exponents(A, B, N, moduli, mode=mode)
        e = sc["e"] if e is None else e
        f = sc["f"] if f is None else f
        if keep:
            out.update(sc)
    e = np.asarray(e, dtype=np.int64)
    f = np.asarray(f, dtype=np.int64)
    Aint = integer_rows(A, e)
    Bint = integer_cols(B, f)
    residues, planesA, planesB = [], [], []
    for p in moduli:
        pa = digit_planes(Aint, p)
        pb = [x.T for x in digit_planes(Bint.T, p)]
        residues.append(np.asarray(residue_product(pa, pb, p), dtype=np.int64))
        if keep:
            planesA.append(pa)
            planesB.append(pb)
    Cint = crt_reconstruct(residues, moduli)
    C = unscale(Cint, e, f)
    badr, badc = nonfinite_masks(A, B)
    C[badr, :] = np.nan
    C[:, badc] = np.nan
    out.update(C=C, e=e, f=f, residues=residues)
    if keep:
        out.update(Aint=Aint, Bint=Bint, Cint=Cint, planesA=planesA, planesB=planesB)
    return out


# --------------------------------------------------------------------------
# Exact references (definitions of the plain matrix product)
# --------------------------------------------------------------------------


def exact_integer_product_entry(Aint, Bint, i, j):
    """(A'B')_ij with Python ints."""
    return sum(int(Aint[i, h]) * int(Bint[h, j]) for h in range(Aint.shape[1]))


def condition_lhs_entry(Aint, Bint, i, j):
    """2 sum_h |a'_ih| |b'_hj|, the left side of the Ozaki-II condition [Sec. II Eq. condition]."""
    return 2 * sum(abs(int(Aint[i, h])) * abs(int(Bint[h, j])) for h in range(Aint.shape[1]))


def exact_dot(a, b):
    """Exact sum_h a_h b_h of two float64 vectors as a Fraction."""
    terms = []
    for x, y in zip(a, b):
        x, y = float(x), float(y)
        if x == 0.0 or y == 0.0:
            continue
        nx, dx = x.as_integer_ratio()
        ny, dy = y.as_integer_ratio()
        terms.append((nx * ny, dx * dy))
    if not terms:
        return Fraction(0)
    den = max(d for _, d in terms)  # all denominators are powers of two
    return Fraction(sum(nm * (den // d) for nm, d in terms), den)


def exact_abs_dot(a, b):
    """Exact sum_h |a_h| |b_h| as a Fraction ((|A||B|)_ij for the error bound)."""
    return exact_dot(np.abs(a), np.abs(b))


def emulated_entry(a_row, b_col, e_i, f_j, moduli):
    """One output entry of the method for given exponents, through the plain
    definition: C'_ij = (A'B')_ij exactly (what the CRT returns when Eq. condition
    holds), then RN(C'_ij 2^-(e_i+f_j)).  Returns (value, condition_holds)."""
    P = product_P(moduli)
    ai = [trunc_scaled(x, int(e_i)) for x in a_row]
    bj = [trunc_scaled(x, int(f_j)) for x in b_col]
    c = sum(x * y for x, y in zip(ai, bj))
    lhs = 2 * sum(abs(x) * abs(y) for x, y in zip(ai, bj))
    return round_scaled_to_double(c, int(e_i) + int(f_j)), lhs < P


# --------------------------------------------------------------------------
# Gradients of C = A B that reuse the forward's integer matrices A', B'
# (the paper covers only the product itself; this follows its construction:
#  Eqs. def:A', def:B', condition, CRTmatmul, CRT_finalreduction, inversescaling)
#
#   dA = dC B^T:  B'_hj = trunc(2^f_j b_hj) is the forward's.  With G'_ij =
#                 trunc(2^(g_i - f_j) dC_ij),  (G' B'^T)_ih ~ 2^g_i dA_ih.
#   dB = A^T dC:  A'_ih = trunc(2^e_i a_ih) is the forward's.  With H'_ij =
#                 trunc(2^(h_j - e_i) dC_ij),  (A'^T H')_hj ~ 2^h_j dB_hj.
# Since |G'_ij| |B'_hj| <= 2^g_i |dC_ij| |b_hj|, the Ozaki-II condition
# 2 sum_j |G'_ij| |B'_hj| < P holds once 2 2^g_i max_h (|dC| |B|^T)_ih <= P - 1; the
# whole budget goes to dC's side (B' is fixed).  The bound comes from an FP8 bound
# product as in accurate mode (Sec. III-E, Eq. barCupper), with the lines of B (and the
# columns of A) scaled to FP8 by their own prelim exponents t_h, which the maximum then
# removes again: R_i = max_h RU(cbar_ih 2^-t_h) >= 2^g'_i max_h (|dC||B|^T)_ih.
# --------------------------------------------------------------------------

DELTA_REUSE_POS = np.float32(-(1 + 2.0**-21))  # exact in FP32
DELTA_REUSE_NEG = np.float32(-(1 - 2.0**-21))  # exact in FP32


def reuse_budget_constant(moduli):
    """Q = RD_fp32(log2(P - 1) - 1): log2 of (P - 1)/2, the whole budget of one side."""
    P = product_P(moduli)
    return f32_round_down(_log2_int_high_precision(P - 1) - 1)


def reuse_exponent(gprime, rmax, Q, line_is_zero):
    """g = g' + floor(RD(Q + RD(d log2_f32(R)))), d = -(1 + 2^-21) for log2 R >= 0 and
    -(1 - 2^-21) below, so that d log2_f32(R) <= -log2 R whatever the FP32 rounding of
    the logarithm: then 2 2^(g - g') R <= P - 1.  Zero line: 0.  R = 0 (the other
    operand vanishes on this line's support): g' + floor(Q)."""
    if line_is_zero:
        return 0
    if rmax == 0:
        return int(gprime) + math.floor(float(Q))
    L = log2_f32(rmax)
    d = DELTA_REUSE_POS if float(L) >= 0 else DELTA_REUSE_NEG
    t1 = f32_round_down(Fraction(float(d)) * Fraction(float(L)))
    t2 = f32_round_down(Fraction(float(Q)) + Fraction(float(t1)))
    return int(gprime) + math.floor(float(t2))


def shifted_row_maxima(cbar, shift):
    """max_h RU_fp32(cbar_ih 2^-s_h), s_h = min(shift_h, 126) (an upper bound of
    max_h cbar_ih 2^-shift_h for every shift_h >= -126)."""
    s = np.minimum(np.asarray(shift, dtype=np.int64), 126)
    m, k = cbar.shape
    out = np.zeros(m, dtype=np.float32)
    for i in range(m):
        best = np.float32(0.0)
        for h in range(k):
            c = cbar[i, h]
            if c == 0:
                continue
            v = f32_round_up(Fraction(float(c)) * Fraction(2) ** int(-s[h]))
            best = max(best, v)
        out[i] = best
    return out


def reuse_side_exponents(X, Y, moduli):
    """Exponents of the rows of X for a product X Y^T whose other operand's integers are
    fixed: (g, g', R) with R_i >= 2^g'_i max_h sum_j |x_ij| |y_hj| from the FP8 bound
    product of RU_E4M3(2^g' |X|) and RU_E4M3(2^t |Y|) (t: prelim exponents of Y's rows)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Xf = np.where(np.isfinite(X), X, 0.0)
    Yf = np.where(np.isfinite(Y), Y, 0.0)
    gp = prelim_exponent_rows(Xf)
    t = prelim_exponent_rows(Yf)
    n = X.shape[1]
    cbar = bound_product(bound_operand(Xf, gp), bound_operand(Yf, t).T, n)
    R = shifted_row_maxima(cbar, t) if Y.shape[0] else np.zeros(X.shape[0], np.float32)
    Q = reuse_budget_constant(moduli)
    zero = ~np.any(Xf != 0, axis=1)
    g = np.array([reuse_exponent(gp[i], R[i], Q, zero[i]) for i in range(X.shape[0])], dtype=np.int64)
    return g, np.where(zero, 0, gp), R


def dc_integers_for_dA(dC, g, f):
    """G'_ij = trunc(2^(g_i - f_j) dC_ij) as Python ints."""
    m, n = dC.shape
    out = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            out[i, j] = trunc_scaled(dC[i, j], int(g[i]) - int(f[j]))
    return out


def dc_integers_for_dB(dC, h, e):
    """H'_ij = trunc(2^(h_j - e_i) dC_ij) as Python ints."""
    m, n = dC.shape
    out = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            out[i, j] = trunc_scaled(dC[i, j], int(h[j]) - int(e[i]))
    return out


def _residue_products_of_integers(Xint, YintT, moduli):
    """C'_l = mod(X' Y'^T, p_l) from digit planes (X' is r x c, Y'^T is s x c)."""
    out = []
    for p in moduli:
        px = digit_planes(Xint, p)
        py = [z.T for z in digit_planes(YintT, p)]
        out.append(np.asarray(residue_product(px, py, p), dtype=np.int64))
    return out


def reuse_gradients(A, B, dC, N, e=None, f=None, g=None, h=None):
    """dA = dC B^T and dB = A^T dC by the method, reusing the forward's A' and B'.

    e, f: the forward's exponents (default: the oracle's own accurate-mode scaling of
    A, B); g, h: the exponents of dC's rows and columns (default: reuse_side_exponents).
    Returns dict(dA, dB, g, h, residues_dA, residues_dB).  Non-finite entries: a row of
    dC or a row of B holding one gives NaN in dA's row / column, a column of dC or of A
    NaN in dB's column / row (R10)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    dC = np.asarray(dC, dtype=np.float64)
    moduli = hybrid_moduli(N)
    if e is None or f is None:
        sc = scaling_exponents(A, B, N, moduli)
        e = sc["e"] if e is None else e
        f = sc["f"] if f is None else f
    e = np.asarray(e, dtype=np.int64)
    f = np.asarray(f, dtype=np.int64)
    if g is None:
        g = reuse_side_exponents(dC, B, moduli)[0]
    if h is None:
        h = reuse_side_exponents(dC.T, A.T, moduli)[0]
    g = np.asarray(g, dtype=np.int64)
    h = np.asarray(h, dtype=np.int64)
    Aint = integer_rows(A, e)          # the forward's A' (m x k)
    BintT = integer_rows(B.T, f)       # the forward's B'^T (n x k): columns of B' as rows
    Gint = dc_integers_for_dA(dC, g, f)        # m x n
    Hint = dc_integers_for_dB(dC, h, e)        # m x n
    # dA = G' B'^T: contraction over j; B'^T's lines are the rows h of B' (k x n)
    res_a = _residue_products_of_integers(Gint, BintT.T, moduli)
    # dB = A'^T H': contraction over i; lines of A'^T are the columns of A' (k x m),
    # lines of H' for the output columns are the columns of H' (n x m)
    res_b = _residue_products_of_integers(Aint.T, Hint.T, moduli)
    k = A.shape[1]
    dA = unscale(crt_reconstruct(res_a, moduli), g, np.zeros(k, np.int64))
    dB = unscale(crt_reconstruct(res_b, moduli), np.zeros(k, np.int64), h)
    dA[~np.all(np.isfinite(dC), axis=1), :] = np.nan
    dA[:, ~np.all(np.isfinite(B), axis=1)] = np.nan
    dB[:, ~np.all(np.isfinite(dC), axis=0)] = np.nan
    dB[~np.all(np.isfinite(A), axis=0), :] = np.nan
    return dict(dA=dA, dB=dB, g=g, h=h, residues_dA=res_a, residues_dB=res_b)


def reuse_gradient_entry_dA(dC_row, b_row, f, g_i, moduli):
    """One entry of dA by the plain definition: C'_ih = sum_j G'_ij B'_hj exactly, then
    RN(C' 2^-g_i).  Returns (value, condition_holds)."""
    P = product_P(moduli)
    G = [trunc_scaled(x, int(g_i) - int(fj)) for x, fj in zip(dC_row, f)]
    Bh = [trunc_scaled(x, int(fj)) for x, fj in zip(b_row, f)]
    c = sum(x * y for x, y in zip(G, Bh))
    lhs = 2 * sum(abs(x) * abs(y) for x, y in zip(G, Bh))
    return round_scaled_to_double(c, int(g_i)), lhs < P


def reuse_gradient_entry_dB(a_col, dC_col, e, h_j, moduli):
    """One entry of dB: C'_hj = sum_i A'_ih H'_ij exactly, then RN(C' 2^-h_j)."""
    P = product_P(moduli)
    Ah = [trunc_scaled(x, int(ei)) for x, ei in zip(a_col, e)]
    H = [trunc_scaled(x, int(h_j) - int(ei)) for x, ei in zip(dC_col, e)]
    c = sum(x * y for x, y in zip(Ah, H))
    lhs = 2 * sum(abs(x) * abs(y) for x, y in zip(Ah, H))
    return round_scaled_to_double(c, int(h_j)), lhs < P
