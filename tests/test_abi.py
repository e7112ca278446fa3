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
                     "ozk2_debug_residue_planes", "ozk2_debug_residue_products", "ozk2_debug_crt",
                     "ozk2_dgemm_ex", "ozk2_workspace_size_ex", "ozk2_debug_scales_ex", "ozk2_dgemm_noalloc",
                     "ozk2_dgemm_host", "ozk2_dgemm_host_ex", "ozk2_workspace_size_host", "ozk2_dgemm_batched",
                     "ozk2_batch_plan_create", "ozk2_batch_plan_execute", "ozk2_batch_plan_destroy",
                     "ozk2_workspace_size_batched"]:
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


def test_extended_entry_validation(lib):
    null = ctypes.c_void_p(0)
    bogus = ctypes.c_void_p(0x1000)

    def ex(ta, tb, m, n, k, lda, ldb, ldc, N=12, mode=0, bm=0, bn=0, A=bogus, B=bogus, C=bogus):
        return lib.ozk2_dgemm_ex(ta, tb, m, n, k, A, lda, B, ldb, C, ldc, N, mode, bm, bn, null, 0, null)

    assert ex(2, 0, 4, 4, 4, 4, 4, 4) == 1  # bad op
    assert ex(0, 7, 4, 4, 4, 4, 4, 4) == 1
    assert ex(0, 0, 4, 4, 4, 4, 4, 4, mode=2) == 1  # bad mode
    assert ex(0, 0, 4, 4, 4, 4, 4, 4, bm=-1) == 1  # bad block
    # op(A) = A^T: A stored k x m, lda >= m;  op(B) = B^T: B stored n x k, ldb >= k
    assert ex(1, 0, 6, 4, 3, 5, 4, 4) == 1  # lda 5 < m 6
    assert ex(0, 1, 4, 6, 3, 3, 2, 6) == 1  # ldb 2 < k 3
    assert ex(1, 1, 4, 6, 3, 4, 3, 5) == 1  # ldc 5 < n 6
    assert ex(1, 1, 0, 6, 3, 4, 3, 6, A=null, B=null, C=null) == 0  # empty: nothing touched
    assert ex(0, 0, 4, 4, 4, 4, 4, 4, N=21) == 1


def test_workspace_size_ex(lib):
    # the transposes do not enter; fast mode drops the two bound operands; blocking
    # sizes the workspace for one block
    m, n, k, N = 3000, 2000, 1000, 12
    acc = lib.ozk2_workspace_size_ex(m, n, k, N, 0, 0, 0)
    assert acc == lib.ozk2_workspace_size(m, n, k, N)
    fast = lib.ozk2_workspace_size_ex(m, n, k, N, 1, 0, 0)
    assert acc - fast >= (m + n) * 1024 - (m + n) * 4 * 32 - 4096
    assert fast < acc
    blk = lib.ozk2_workspace_size_ex(m, n, k, N, 0, 1024, 512)
    assert blk == lib.ozk2_workspace_size(1024, 512, k, N)
    assert lib.ozk2_workspace_size_ex(m, n, k, N, 0, 5000, 5000) == acc
    assert lib.ozk2_workspace_size_ex(m, n, k, N, 3, 0, 0) == 0
    assert lib.ozk2_workspace_size_ex(m, n, k, N, 0, -2, 0) == 0


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
        # the residue products park their partial residues in registers: no GEMM scratch
        assert dominant <= ws <= dominant + 64 * 1024 + 40 * (m + n)
    # the paper's layout needs 55 GB at 16384^3, N = 12 (Sec. IV-C); this one about 23 GB
    assert lib.ozk2_workspace_size(16384, 16384, 16384, 12) < 24e9


def test_host_entry_validation_and_size(lib):
    null = ctypes.c_void_p(0)
    bogus = ctypes.c_void_p(0x1000)
    host = lib.ozk2_dgemm_host
    assert host(0, 0, -1, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, 0, null, 0, null) == 1
    assert host(3, 0, 4, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, 0, null, 0, null) == 1  # bad op
    assert host(0, 0, 4, 4, 4, bogus, 4, bogus, 4, bogus, 4, 12, 5, null, 0, null) == 1  # bad mode
    assert host(0, 0, 4, 4, 8, bogus, 4, bogus, 4, bogus, 4, 12, 0, null, 0, null) == 1  # lda < k
    assert host(0, 0, 4, 4, 4, null, 4, bogus, 4, bogus, 4, 12, 0, null, 0, null) == 1
    assert host(0, 0, 0, 4, 4, null, 4, null, 4, null, 4, 12, 0, null, 0, null) == 0  # empty
    hx = lib.ozk2_dgemm_host_ex
    assert hx(0, 0, 0, 4, 4, null, 4, null, 4, null, 4, 12, 0, 1, null, 0, null) == 0  # inputs-ready flag
    assert hx(0, 0, 0, 4, 4, null, 4, null, 4, null, 4, 12, 0, 2, null, 0, null) == 1  # unknown flag
    assert hx(0, 0, 4, 4, 8, bogus, 4, bogus, 4, bogus, 4, 12, 0, 1, null, 0, null) == 1  # lda < k
    m, n, k, N = 1000, 700, 300, 12
    for mode in (0, 1):
        staged = 8 * (m * k + k * n + m * n)
        ws = lib.ozk2_workspace_size_host(m, n, k, N, mode)
        base = lib.ozk2_workspace_size_ex(m, n, k, N, mode, 0, 0)
        assert base + staged <= ws <= base + staged + 3 * 256
    assert lib.ozk2_workspace_size_host(m, n, k, N, 2) == 0


def test_batch_validation_and_size(lib):
    null = ctypes.c_void_p(0)
    I64 = ctypes.c_int64 * 3
    P = ctypes.c_void_p * 3
    m, n, k = I64(10, 20, 30), I64(5, 6, 7), I64(8, 9, 10)
    ld_ok_a, ld_ok_b = I64(8, 9, 10), I64(5, 6, 7)
    ptr = P(0x1000, 0x2000, 0x3000)
    batched = lib.ozk2_dgemm_batched
    assert batched(-1, m, n, k, ptr, ld_ok_a, ptr, ld_ok_b, ptr, ld_ok_b, 12, 0, null, 0, null) == 1
    assert batched(3, null, n, k, ptr, ld_ok_a, ptr, ld_ok_b, ptr, ld_ok_b, 12, 0, null, 0, null) == 1
    assert batched(3, m, n, k, ptr, I64(8, 8, 10), ptr, ld_ok_b, ptr, ld_ok_b, 12, 0, null, 0, null) == 1
    assert batched(3, m, n, k, ptr, ld_ok_a, ptr, ld_ok_b, P(0x1000, 0, 0x3000), ld_ok_b, 12, 0, null, 0,
                   null) == 1
    assert batched(3, m, n, k, ptr, ld_ok_a, ptr, ld_ok_b, ptr, ld_ok_b, 21, 0, null, 0, null) == 1
    assert batched(0, null, null, null, null, null, null, null, null, null, 12, 0, null, 0, null) == 0
    # the batch layout: the per-problem arrays of single calls plus descriptors
    single = sum(lib.ozk2_workspace_size(int(m[i]), int(n[i]), int(k[i]), 12) for i in range(3))
    ws = lib.ozk2_workspace_size_batched(3, m, n, k, 12, 0)
    assert single - 3 * 64 * 1024 <= ws <= single + 64 * 1024
    assert lib.ozk2_workspace_size_batched(3, m, n, k, 12, 0) > lib.ozk2_workspace_size_batched(3, m, n, k, 12, 1)
    assert lib.ozk2_workspace_size_batched(3, m, I64(5, -6, 7), k, 12, 0) == 0


def test_fault_injection_arming(lib):
    """ozk2_debug_inject_fault arms one fault kind, reports the previous one, rejects
    unknown kinds; argument and device checks come before any injected fault."""
    assert lib.ozk2_debug_inject_fault(-1) == 0  # nothing armed
    assert lib.ozk2_debug_inject_fault(1) == 0  # arm alloc
    assert lib.ozk2_debug_inject_fault(-1) == 1
    assert lib.ozk2_debug_inject_fault(7) == -1  # unknown kind: unchanged
    assert lib.ozk2_debug_inject_fault(-1) == 1
    bogus = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    # an argument error returns before the workspace is taken: the fault stays armed
    assert lib.ozk2_dgemm(4, 4, 8, bogus, 4, bogus, 4, bogus, 4, 12, null) == 1
    assert lib.ozk2_debug_inject_fault(-1) == 1
    assert lib.ozk2_debug_inject_fault(0) == 1  # disarm
    assert lib.ozk2_debug_inject_fault(-1) == 0


def test_fault_injection_from_environment():
    """OZK2_FAULT arms a fault when the library first needs the setting."""
    import subprocess
    import sys

    code = ("from paper_2603_10634_gb300 import _lib; lib = _lib.load(); "
            "print(lib.ozk2_debug_inject_fault(-1))")
    for spec, want in [("stall", 3), ("launch", 2), ("alloc", 1), ("bogus", 0)]:
        env = dict(os.environ, OZK2_FAULT=spec)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0, out.stderr
        assert int(out.stdout.strip().splitlines()[-1]) == want, spec


def test_wait_limit_setting(lib):
    """ozk2_set_wait_limit returns the previous setting; 0 is the default."""
    assert lib.ozk2_set_wait_limit(1000) == 0
    assert lib.ozk2_set_wait_limit(0) == 1000
    assert lib.ozk2_set_wait_limit(0) == 0


def test_tile_setting(lib):
    """ozk2_set_tile_n takes 0, 128 or 256 and returns the previous value."""
    assert lib.ozk2_set_tile_n(64) == -1
    assert lib.ozk2_set_tile_n(128) == 0
    assert lib.ozk2_set_tile_n(256) == 128
    assert lib.ozk2_set_tile_n(0) == 256
    assert lib.ozk2_batch_plan_tile_n(None) == -1


def test_square_split_setting(lib):
    prev = lib.ozk2_set_square_split(-1)
    assert prev == 0
    assert lib.ozk2_set_square_split(4096) == 0
    assert lib.ozk2_set_square_split(8192) == 4096
    assert lib.ozk2_set_square_split(prev) == 8192
