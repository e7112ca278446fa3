"""CPU-side checks of the C-ABI boundary (no GPU needed).

* libozk2.so builds for sm_103a, loads, and exports every function declared in
  include/ozk2.h.
* Host-side argument validation returns synchronously and touches no memory.
* The library's own moduli table (C++, independent of the oracle) equals the
  oracle's hybrid list, and its workspace size follows its documented layout.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ozk2.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ozk2_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_10634_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ozk2_dgemm", "ozk2_workspace_size", "ozk2_dgemm_ws", "ozk2_status_string",
                     "ozk2_device_status", "ozk2_moduli", "ozk2_debug_fp8_gemm", "ozk2_debug_scales",
                     "ozk2_debug_residue_planes", "ozk2_debug_residue_products", "ozk2_debug_crt"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_10634_gb300 import _lib

    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    for code, name in [(0, b"OZK2_OK"), (1, b"OZK2_ERR_INVALID_VALUE"), (6, b"OZK2_ERR_TIMEOUT")]:
        assert lib.ozk2_status_string(code) == name


def test_argument_validation_is_synchronous(lib):
    null = ctypes.c_void_p(0)
    bogus = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    # negative sizes, bad N, bad leading dimensions, missing pointers
    assert lib.ozk2_dgemm(-1, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, null) == 1
    assert lib.ozk2_dgemm(4, 4, 4, bogus, 4, bogus, 4, bogus, 4, 0, null) == 1
    assert lib.ozk2_dgemm(4, 4, 4, bogus, 4, bogus, 4, bogus, 4, 21, null) == 1
    assert lib.ozk2_dgemm(4, 4, 8, bogus, 4, bogus, 4, bogus, 4, 12, null) == 1  # lda < k
    assert lib.ozk2_dgemm(4, 4, 4, bogus, 4, bogus, 3, bogus, 4, 12, null) == 1  # ldb < n
    assert lib.ozk2_dgemm(4, 4, 4, bogus, 4, bogus, 4, bogus, 3, 12, null) == 1  # ldc < n
    assert lib.ozk2_dgemm(4, 4, 4, null, 4, bogus, 4, bogus, 4, 12, null) == 1
    assert lib.ozk2_dgemm(2**21, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, null) == 2
    # empty products are complete without touching memory
    assert lib.ozk2_dgemm(0, 4, 4, null, 4, null, 4, null, 4, 12, null) == 0
    assert lib.ozk2_dgemm(4, 0, 4, null, 4, null, 1, null, 1, 12, null) == 0
    assert lib.ozk2_dgemm_ws(4, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, null, 0, null) == 1
    assert lib.ozk2_debug_fp8_gemm(-1, 1, 1, bogus, 16, bogus, 16, bogus, 1, null) == 1


def test_library_moduli_match_oracle(lib):
    from oracle import ozaki2 as oz

    for N in range(1, 21):
        buf = (ctypes.c_int32 * N)()
        assert lib.ozk2_moduli(N, buf) == N
        assert list(buf) == oz.hybrid_moduli(N)
    buf = (ctypes.c_int32 * 21)()
    assert lib.ozk2_moduli(21, buf) == -1
    assert lib.ozk2_moduli(0, buf) == -1


def test_workspace_size(lib):
    from oracle import ozaki2 as oz

    assert lib.ozk2_workspace_size(-1, 1, 1, 12) == 0
    assert lib.ozk2_workspace_size(1, 1, 1, 0) == 0
    for (m, n, k, N) in [(256, 256, 256, 12), (16384, 16384, 16384, 12), (100, 37, 999, 7), (64, 64, 64, 3)]:
        ws = lib.ozk2_workspace_size(m, n, k, N)
        kp = 32 * ((k + 31) // 32)
        ldr = 8 * ((n + 7) // 8)
        M = oz.num_digit_planes(N)
        dominant = (1 + M) * (m + n) * kp + 2 * N * m * ldr
        gemm_scratch = 192 * 128 * 256 * 4  # per-CTA tile scratch of the residue products
        assert dominant + gemm_scratch <= ws <= dominant + gemm_scratch + 64 * 1024 + 40 * (m + n)
    # the paper's layout needs 55 GB at 16384^3, N = 12 (Sec. IV-C); this one about 23 GB
    assert lib.ozk2_workspace_size(16384, 16384, 16384, 12) < 24e9
