"""Pins for the oracle's moduli, P and counts against values printed in the paper.

Moduli lists: Sec. II Eq. p_list, Sec. III-B Eq. p_list_karatsuba, Sec. III-D
Eq. p_list_hybrid, Sec. III-A.  Bounds on P/2: same sections.  GEMM counts and
effective bits: Sec. IV-A Table 2.  M_N: Sec. IV-B Eq. M.
"""
import math
from math import gcd

import pytest

from oracle import ozaki2 as oz

LISTS = {
    "int8": lambda N: oz.int8_moduli(N),
    "karatsuba": lambda N: oz.karatsuba_moduli(N),
    "hybrid": lambda N: oz.hybrid_moduli(N),
    "direct": lambda N: oz.direct_fp8_moduli()[:N],
}
FULL = {
    "int8": lambda: oz._greedy_coprime_descending(256, [], 10**9),
    "karatsuba": lambda: oz._greedy_coprime_descending(513, [], 10**9),
    "hybrid": oz.hybrid_moduli_full,
    "direct": oz.direct_fp8_moduli,
}


def test_printed_lists(golden):
    rows = golden("paper_moduli_lists.txt")
    assert {r[0] for r in rows} == set(LISTS)
    for name, _src, vals in rows:
        printed = [int(v) for v in vals.split()]
        assert LISTS[name](len(printed)) == printed, name


def test_direct_list_is_complete():
    # Sec. III-A lists exactly eleven candidates <= 32
    assert oz.direct_fp8_moduli() == [32, 31, 29, 27, 25, 23, 19, 17, 13, 11, 7]


@pytest.mark.parametrize("name", ["int8", "karatsuba", "hybrid"])
def test_pairwise_coprime(name):
    ms = FULL[name]()
    for i in range(len(ms)):
        for j in range(i):
            assert gcd(ms[i], ms[j]) == 1


def test_printed_bounds(golden):
    for name, N, rel, power, _src in golden("paper_bounds.txt"):
        ms = FULL[name]() if N == "all" else LISTS[name](int(N))
        half = oz.product_P(ms) / 2  # Python float of an exact int ratio is fine for these
        lhs = math.log2(oz.product_P(ms)) - 1
        p = int(power)
        if rel == ">":
            assert lhs > p and half > 2**p, (name, N)
        elif rel == ">=":
            assert oz.product_P(ms) >= 2 ** (p + 1), (name, N)
        else:
            assert oz.product_P(ms) < 2 ** (p + 1), (name, N)


def test_hybrid_fp64_threshold():
    # Sec. III-D: N >= 12 is what reaches P/2 > 2^(53+53); N = 11 does not.
    assert oz.product_P(oz.hybrid_moduli(11)) < 2 ** 107
    assert oz.product_P(oz.hybrid_moduli(12)) > 2 ** 111


def test_squares_lead_the_hybrid_list():
    # Sec. III-D and Sec. IV-B: for N < 34 the square moduli are p_1..p_6.
    full = oz.hybrid_moduli_full()
    assert full[:6] == [1089, 1024, 961, 841, 625, 529]
    squares_later = [i for i, p in enumerate(full) if i >= 6 and math.isqrt(p) ** 2 == p]
    assert min(squares_later) == 33  # 361 = 19^2 is the 34th entry
    for N in range(1, 34):
        kinds = [oz.modulus_kind(p)[0] for p in oz.hybrid_moduli(N)]
        assert kinds == ["square"] * min(N, 6) + ["karatsuba"] * max(0, N - 6)


def test_table2_counts_and_bits(golden):
    for method, N, fast, acc, bits in golden("paper_table2.txt"):
        N = int(N)
        if method == "fp8_ozaki2":
            assert oz.num_fp8_gemms(N, "fast") == int(fast)
            assert oz.num_fp8_gemms(N, "accurate") == int(acc)
            P = oz.product_P(oz.hybrid_moduli(N))
        else:
            assert (N, N + 1) == (int(fast), int(acc))
            P = oz.product_P(oz.int8_moduli(N))
        # effective bits <~ log2 sqrt(P/2), printed as its integer part
        assert math.floor((math.log2(P) - 1) / 2) == int(bits), (method, N)


def test_num_digit_planes():
    # Eq. M: 2N for N <= 6, else 3N - 6; equals the planes each modulus contributes
    for N in range(1, 34):
        per = sum(2 if oz.modulus_kind(p)[0] == "square" else 3 for p in oz.hybrid_moduli(N))
        assert oz.num_digit_planes(N) == per


def test_paper_workspace_figure():
    # Sec. IV-C: W_f8 at m = n = k = 16384, N = 12 is quoted as 55 GB
    m = n = k = 16384
    N = 12
    M = oz.num_digit_planes(N)
    W = (m * k + k * n + 4 * m * n) * M + 2 * N * m * n + 2 * (m + n)
    assert round(W / 1e9) == 55
