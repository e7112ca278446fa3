"""Pins for symmetric residues, digit splits and the FP8 E4M3 encoding.

Digit bounds |d| <= 16 and E4M3 representability: Sec. III-B (Karatsuba split,
s = 16) and Sec. III-D (square split, s = sqrt(p)).  E4M3 codes are checked
against torch's float8_e4m3fn decoder (an independent library routine).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import ozaki2 as oz

MODULI = oz.hybrid_moduli(20)


def torch_e4m3_values():
    return torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()


def test_e4m3_value_matches_torch():
    ref = torch_e4m3_values()
    for c in range(256):
        v = oz.e4m3_value(c)
        if v is None:
            assert np.isnan(ref[c])
        else:
            assert float(v) == ref[c], hex(c)


def test_e4m3_landmarks():
    assert oz.e4m3_value(0x01) == Fraction(1, 512)  # smallest subnormal 2^-9
    assert oz.e4m3_value(0x08) == Fraction(1, 64)  # smallest normal 2^-6
    assert oz.e4m3_value(0x7E) == 448
    assert oz.e4m3_value(0x78) == 256
    # every integer in [-16, 16] is representable (Sec. III-A)
    for d in range(-16, 17):
        assert oz.e4m3_value(oz.e4m3_code_of_integer(d)) == d
    with pytest.raises(ValueError):
        oz.e4m3_code_of_integer(17)


@pytest.mark.parametrize("seed", [0, 1])
def test_round_up_is_least_upper_value(seed):
    rng = np.random.default_rng(seed)
    xs = np.concatenate([rng.uniform(0, 448, 3000), 2.0 ** rng.uniform(-14, 8.8, 3000),
                         np.array([0.0, 2.0**-9, 2.0**-10, 1e-300, 5e-324, 256.0, 255.999, 448.0])])
    vals = torch_e4m3_values()
    for x in xs:
        c = oz.e4m3_round_up_code(float(x))
        v = vals[c]
        assert v >= x
        if x == 0:
            assert c == 0
            continue
        # the previous finite code is strictly below x, except that x < 2^-9 maps to 2^-9
        if c > 1:
            assert vals[c - 1] < x
        else:
            assert c == 1 and x <= 2.0**-9


def test_round_up_vectorised_matches_scalar():
    rng = np.random.default_rng(3)
    A = (rng.random((17, 33)) - 0.5) * np.exp(2.0 * rng.standard_normal((17, 33)))
    A[3, :] = 0.0
    A[4, 5] = 5e-324
    A[5, 7] = -1e-310
    ep = oz.prelim_exponent_rows(A)
    codes = oz.bound_operand(A, ep)
    for i in range(A.shape[0]):
        for h in range(A.shape[1]):
            a = A[i, h]
            want = 0 if a == 0 else oz.e4m3_round_up_code(Fraction(abs(float(a))) * Fraction(2) ** int(ep[i]))
            assert codes[i, h] == want


def test_scaled_row_fits_below_256():
    # Sec. III-E: 2^e' |a| < 2^8, so RU to E4M3 never overflows and stays <= 256
    rng = np.random.default_rng(5)
    A = (rng.random((50, 40)) - 0.5) * np.exp(3.0 * rng.standard_normal((50, 40)))
    ep = oz.prelim_exponent_rows(A)
    for i in range(50):
        mx = np.abs(A[i]).max()
        assert 2.0**7 <= mx * 2.0 ** ep[i] < 2.0**8
    vals = torch_e4m3_values()
    assert vals[oz.bound_operand(A, ep)].max() <= 256


@pytest.mark.parametrize("p", MODULI)
def test_smod_range_and_congruence(p):
    xs = np.arange(-3 * p, 3 * p + 1, dtype=np.int64)
    r = oz.smod(xs, p)
    assert np.all((r - xs) % p == 0)
    assert r.min() == -(p // 2) and r.max() == p - 1 - p // 2
    # object arrays of big ints too
    big = np.array([2**100 + 7, -(2**90) - 3], dtype=object)
    rb = oz.smod(big, p)
    for x, y in zip(big, rb):
        assert (x - y) % p == 0 and -(p // 2) <= y < p - p // 2


@pytest.mark.parametrize("p", MODULI)
def test_digit_split_exhaustive(p):
    """Every residue of every modulus splits into digits |d| <= 16 that recompose exactly."""
    kind, s = oz.modulus_kind(p)
    for r in range(-(p // 2), p - p // 2):
        ds = oz.split_digits(r, p)
        assert all(abs(d) <= 16 for d in ds), (p, r, ds)
        if kind == "square":
            d1, d2 = ds
            assert s * d1 + d2 == r
        else:
            d1, d2, d3 = ds
            assert s * d1 + d2 == r and d3 == d1 + d2
            assert abs(r) <= 256  # Eq. limit1
    # the vectorised plane builder gives the same digits
    X = np.arange(-(p // 2), p - p // 2, dtype=object).reshape(1, -1)
    planes = oz.digit_planes(X, p)
    for idx, r in enumerate(range(-(p // 2), p - p // 2)):
        assert tuple(int(pl[0, idx]) for pl in planes) == tuple(oz.split_digits(r, p))


def test_square_split_ties_go_to_even():
    # s = 32 (p = 1024) is the only even s; r = 32 d + 16 is a tie
    assert oz.split_square(16, 32) == (0, 16)
    assert oz.split_square(48, 32) == (2, -16)
    assert oz.split_square(-16, 32) == (0, -16)
    assert oz.split_square(-48, 32) == (-2, 16)


def test_karatsuba_split_examples():
    # sign(r) * ceil(|r| / 16) [Sec. III-B]
    assert oz.split_karatsuba(0) == (0, 0, 0)
    assert oz.split_karatsuba(1) == (1, -15, -14)
    assert oz.split_karatsuba(16) == (1, 0, 1)
    assert oz.split_karatsuba(17) == (2, -15, -13)
    assert oz.split_karatsuba(-255) == (-16, 1, -15)
    assert oz.split_karatsuba(256) == (16, 0, 16)
