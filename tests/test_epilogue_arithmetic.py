"""Arithmetic facts the digit-plane kernels and the residue-product epilogue rely on,
checked on the CPU in exact arithmetic (the GPU parity tests check the kernels).

* Karatsuba moduli (Sec. III-B): with r = 16 d1 + d2 and d3 = d1 + d2 for both operands
  and Dx = dx_a dx_b, 240 D1 - 15 D2 + 16 D3 = r_a r_b exactly (Eq. C'-Karatsuba
  rearranged), so the second pass may park v = mod(240 d1 - 15 D2, p) and the third
  finish with mod(v + 16 D3, p).
* The FP32 reduction: for an exact-integer float |x| <= 2^24 and every modulus p of the
  hybrid list (N <= 20), q = RN(x RN(1/p) + 1.5 2^23) - 1.5 2^23 gives r = x - p q with
  r = x (mod p) and |r| < 0.51 p, and the sums formed from such remainders stay below
  2^24 (exact in FP32).
* The digit-plane kernels' quotient: one rounded product gives the nearest integer to
  x / p for odd p (|x| < 2^23), and the floor form for p = 1024.
* The CRT kernel's quotient estimate from 16-bit weight fractions (Eq. CRT_finalreduction):
  within 0.17 of V / P, in a 32-bit accumulator that cannot overflow (N <= 20).
"""
import os
import random
import sys
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ozaki2 as oz  # noqa: E402

MAGIC = Fraction(3 * 2**22)  # 1.5 * 2^23


def _residues(p):
    h = p // 2
    return np.arange(-h, p - h, dtype=np.int64)


def test_karatsuba_parking_identity():
    for p in oz.hybrid_moduli(20):
        kind, s = oz.modulus_kind(p)
        if kind == "square":
            continue
        r = _residues(p)
        d = np.array([oz.split_karatsuba(int(x), s) for x in r], dtype=np.int64)  # (p, 3)
        d1, d2, d3 = d[:, 0], d[:, 1], d[:, 2]
        D1, D2, D3 = np.outer(d1, d1), np.outer(d2, d2), np.outer(d3, d3)
        assert np.array_equal(240 * D1 - 15 * D2 + 16 * D3, np.outer(r, r)), p


def _mod_near(x, p, inv_p):
    """The kernel's steps in exact arithmetic: one FMA rounded to FP32, one exact
    subtraction, one exact FMA."""
    t = oz.f32_round_nearest(Fraction(x) * Fraction(float(inv_p)) + MAGIC)
    q = Fraction(float(t)) - MAGIC
    assert q.denominator == 1
    return x - p * int(q)


def test_fp32_reduction_exact_and_bounded():
    rng = random.Random(7)
    top = 2**24
    for p in oz.hybrid_moduli(20):
        inv_p = oz.f32_round_nearest(Fraction(1, p))
        xs = [0, 1, -1, top, -top, top - 1, -(top - 1), p // 2, -(p // 2), p // 2 + 1]
        base = (top // p) * p
        xs += [base + p // 2 + t for t in (-1, 0, 1)] + [-(base + p // 2 + t) for t in (-1, 0, 1)]
        xs += [rng.randint(-top, top) for _ in range(150)]
        for x in xs:
            r = _mod_near(x, p, inv_p)
            assert (x - r) % p == 0, (p, x)
            assert abs(r) < 0.51 * p, (p, x, r)


def test_fp32_reduction_sums_stay_exact():
    bound = 0.51
    for p in oz.hybrid_moduli(20):
        kind, s = oz.modulus_kind(p)
        if kind == "square":
            # s (X mod p) + Z with |Z| <= 2^15 * 16 * 16 = 2^23; in the two-pass form
            # X mod p is parked as int16 between the passes
            assert s * bound * p + 2**23 < 2**24, p
            assert bound * p < 2**15, p
        else:
            # 240 d1 - 15 (D2 mod p) with |d1| <= p/2, and v + 16 (D3 mod p) with |v| <= p/2
            assert 240 * (p // 2) + 15 * bound * p < 2**24, p
            assert (p // 2) + 16 * bound * p < 2**24, p


def test_residue_kernel_quotient_is_the_nearest_integer():
    # The digit-plane kernels form x = sum_j c_j w_j (|x| <= 5 (2^11 - 1) 544 < 2^23) and
    # take q from one rounded product x RN(1/p) + 1.5 2^23; for odd p this is the
    # nearest integer to x / p (never a tie), so r = x - p q is the symmetric remainder
    # without a correction.  p = 1024 uses q = RN(x 2^-10 + 2^-11 + 1.5 2^23) - 1.5 2^23
    # = floor((x + 512) / 1024).
    rng = random.Random(11)
    top = 5 * (2**11 - 1) * 544
    assert top < 2**23
    for p in oz.hybrid_moduli(20):
        h = p // 2
        xs = [0, 1, -1, top, -top] + [rng.randint(-top, top) for _ in range(150)]
        xs += [k * p + d for k in (1, 7, 1000, -3, -1000) for d in (h, h + 1, -h, -h - 1)]
        for x in xs:
            if p == 1024:
                t = oz.f32_round_nearest(Fraction(x, 1024) + Fraction(1, 2048) + MAGIC)
                q = Fraction(float(t)) - MAGIC
                assert q == (x + 512) // 1024, x
            else:
                inv_p = oz.f32_round_nearest(Fraction(1, p))
                t = oz.f32_round_nearest(Fraction(x) * Fraction(float(inv_p)) + MAGIC)
                q = Fraction(float(t)) - MAGIC
                assert q == round(Fraction(x, p)), (p, x)
            r = x - p * int(q)
            assert r == oz.smod(x, p), (p, x)


def test_crt_quotient_estimate_bound():
    # The CRT kernel estimates Q = round(V / P), V = sum_l c_l w_l with the signed residues
    # c_l in [-h_l, p_l - 1 - h_l], from est = sum_l c_l round(2^16 w_l / P) in a signed
    # 32-bit integer: the estimate is within 0.05 of V / P (so a fractional part at least
    # 0.3 from one half decides the rounding, and the rarer cases take the exact
    # comparison), est never overflows, and V - Q P stays inside the kernel's limbs.
    for N in range(1, 21):
        moduli = oz.hybrid_moduli(N)
        w, P = oz.crt_weights(moduli)
        err = Fraction(0)
        est_max = 0
        for p, wl in zip(moduli, w):
            exact = Fraction(2**16 * wl, P)
            f16 = round(exact)
            err += (p // 2) * abs(f16 - exact) / 2**16
            est_max += (p // 2) * f16
        assert err < Fraction(5, 100), (N, float(err))
        assert est_max + 0x8000 < 2**31, N
        # V = sum c_l w_l changes by q_l P when c_l < 0 is replaced by c_l + p_l: the same mod P
        for p, wl in zip(moduli, w):
            assert (p * wl) % P == 0


def test_crt_balanced_weight_limbs():
    # w_l = sum_t b_t 2^(32 t) with every b_t in [-2^31, 2^31) in the kernel's limb count,
    # and the 64-bit limb sums of at most 20 terms |c_l b_t| < 2^46 cannot overflow
    for N in range(1, 21):
        moduli = oz.hybrid_moduli(N)
        w, P = oz.crt_weights(moduli)
        L = (P.bit_length() + 1 + 31) // 32
        for wl in w:
            b, carry = [], 0
            for t in range(L):
                u = ((wl >> (32 * t)) & 0xFFFFFFFF) + carry
                carry = 1 if u >= 2**31 else 0
                b.append(u - (carry << 32))
            assert carry == 0 and all(-2**31 <= x < 2**31 for x in b)
            assert sum(x << (32 * t) for t, x in enumerate(b)) == wl
        assert 20 * 2**15 * 2**31 < 2**63


def test_library_reciprocals_are_correctly_rounded():
    # The library stores 1/p and 1/s as float(1.0 / p) (a double quotient rounded to
    # float); the quotient bounds above assume the correctly rounded RN(1/p), and the two
    # agree for every modulus and digit base of the list.
    for p in oz.hybrid_moduli(20):
        _, s = oz.modulus_kind(p)
        for v in (p, s):
            assert np.float32(1.0 / v) == oz.f32_round_nearest(Fraction(1, v)), v


def _smod_small_step(y, p, inv_p):
    """The epilogue's exact final reduction of an exact integer |y| < 2^23: one rounded
    product for odd p, q = RN((y + 1/2) / 1024) for p = 1024 (|y| < 2^12 there)."""
    if p == 1024:
        t = oz.f32_round_nearest(Fraction(y, 1024) + Fraction(1, 2048))
        assert Fraction(float(t)) == Fraction(y, 1024) + Fraction(1, 2048)  # the FMA is exact
        q = Fraction(float(oz.f32_round_nearest(Fraction(float(t)) + MAGIC))) - MAGIC
        return y - 1024 * int(q)
    return _mod_near(y, p, inv_p)


def test_epilogue_two_step_reduction_is_the_symmetric_remainder():
    # smod2: a first reduction of |x| <= 2^24 to |r| < 0.51 p, then the exact step
    rng = random.Random(13)
    top = 2**24
    for p in oz.hybrid_moduli(20):
        inv_p = oz.f32_round_nearest(Fraction(1, p))
        h = p // 2
        xs = [0, 1, -1, top, -top, h, -h, h + 1, -h - 1]
        xs += [k * p + d for k in (1, 9, 15000, -7, -15000) for d in (h, h + 1, -h, -h - 1, p - 1 - h)]
        xs += [rng.randint(-top, top) for _ in range(300)]
        for x in xs:
            r1 = _mod_near(x, p, inv_p)
            assert abs(r1) < 2**12
            assert _smod_small_step(r1, p, inv_p) == oz.smod(x, p), (p, x)


def test_epilogue_karatsuba_steps_are_exact():
    # pass 2: y = 240 d1 - 15 (D2 mod_near) with |d1| <= h; pass 3: y = v + 16 (D3 mod_near);
    # both below 2^23, so the single final step gives the symmetric remainder
    rng = random.Random(17)
    for p in oz.hybrid_moduli(20):
        kind, _ = oz.modulus_kind(p)
        if kind == "square":
            continue
        inv_p = oz.f32_round_nearest(Fraction(1, p))
        h = p // 2
        for _ in range(300):
            d1 = rng.randint(-h, p - 1 - h)
            D2 = rng.randint(-2**24, 2**24)
            d2 = _mod_near(D2, p, inv_p)
            y = 240 * d1 - 15 * d2
            assert abs(y) < 2**17
            assert _smod_small_step(y, p, inv_p) == oz.smod(240 * d1 - 15 * D2, p)
            D3 = rng.randint(-2**24, 2**24)
            y3 = d1 + 16 * _mod_near(D3, p, inv_p)
            assert abs(y3) < 2**14
            assert _smod_small_step(y3, p, inv_p) == oz.smod(d1 + 16 * D3, p)


def test_epilogue_int16_packing_by_magic_bias():
    # r + 1.5 2^23 is exact for |r| < 2^22; its low 16 bits are r in two's complement
    for r in [0, 1, -1, 511, -512, 544, -544, 2**15 - 1, -2**15] + list(range(-600, 600, 37)):
        b = np.array([np.float32(r) + np.float32(1.5 * 2**23)], dtype=np.float32).view(np.uint32)[0]
        assert np.float32(r) + np.float32(1.5 * 2**23) == np.float32(r + 1.5 * 2**23)
        assert np.int16(np.uint16(int(b) & 0xFFFF)) == r


def test_karatsuba_high_digit_one_rounding():
    # the digit kernels form d1 = sign(r) ceil(|r| / 16) as RN(r / 16 + sign(r) 15/32) through
    # 1.5 2^23: r / 16 + 15/32 is exact in FP32 and never a half-integer for integer r
    for p in oz.hybrid_moduli(20):
        kind, s = oz.modulus_kind(p)
        if kind == "square":
            continue
        for r in _residues(p):
            r = int(r)
            off = Fraction(15, 32) if r >= 0 else Fraction(-15, 32)
            t = Fraction(r, 16) + off
            assert oz.f32_round_nearest(t) == t  # exact
            q = Fraction(float(oz.f32_round_nearest(t + MAGIC))) - MAGIC
            assert int(q) == oz.split_karatsuba(r, s)[0], (p, r)
