"""ozk2_dgemm_noalloc, the entry point for callers that may not allocate device memory.

It must give exactly what ozk2_dgemm gives on the same inputs, on two calls in a row
(the second call reuses the static workspace left by the first, with another shape),
and refuse a problem that does not fit its static workspace.  Called through the C
ABI.  This file is named so that pytest collects it after every other test file."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from paper_2603_10634_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, B, N):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), float("nan"), dtype=torch.float64, device=A.device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.ozk2_dgemm_noalloc(m, n, k, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                               B.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(0), N, st)
    return s, C


def _noalloc_status(lib):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.STATUS.get(lib.ozk2_noalloc_device_status(st))


def test_noalloc_matches_dgemm_on_two_calls(cuda):
    lib = _lib.load()
    cases = [((300, 200, 700), 12, 1.0, 0), ((512, 384, 1000), 14, 2.0, 5)]
    for (m, n, k), N, phi, seed in cases:
        A, B = workloads.problem(m, n, k, phi, seed=seed, device=cuda)
        s, C = _noalloc(lib, A, B, N)
        assert s == 0, _lib.STATUS.get(s, s)
        want = ozk.dgemm(A, B, num_moduli=N)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().view(np.uint64), want.cpu().numpy().view(np.uint64))


def test_noalloc_smaller_call_after_a_larger_one_with_a_flag(cuda):
    """A larger call whose input has a NaN row (it sets the non-finite flag, fills bound
    maxima and column reductions over its whole layout) followed by a smaller call: the
    smaller call ignores what the larger one left in the shared array.  The flag word of
    each call is read by ozk2_noalloc_device_status; ozk2_device_status, which reads the
    library-owned workspace, reports nothing about these calls."""
    lib = _lib.load()
    A, B = workloads.problem(520, 400, 1100, 1.0, seed=9, device=cuda)
    A[17, 5] = float("nan")
    ozk.device_status()  # clear the library-owned workspace's flag word
    s, C = _noalloc(lib, A, B, 12)
    assert s == 0
    assert _noalloc_status(lib) == "OZK2_ERR_NONFINITE"
    assert ozk.device_status() == "OZK2_OK"
    want = ozk.dgemm(A, B, num_moduli=12)
    torch.cuda.synchronize()
    assert torch.isnan(C[17]).all().item()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), want.cpu().numpy().view(np.uint64))
    ozk.device_status()
    A2, B2 = workloads.problem(100, 90, 50, 0.5, seed=10, device=cuda)
    s, C2 = _noalloc(lib, A2, B2, 12)
    assert s == 0
    assert _noalloc_status(lib) == "OZK2_OK"
    want2 = ozk.dgemm(A2, B2, num_moduli=12)
    torch.cuda.synchronize()
    assert np.array_equal(C2.cpu().numpy().view(np.uint64), want2.cpu().numpy().view(np.uint64))


def test_noalloc_trivial_shapes_as_dgemm(cuda):
    """m or n = 0 and k = 0 need no workspace: they behave as ozk2_dgemm even where the
    other dimensions are far beyond the static array; out-of-range sizes are refused as
    ozk2_dgemm refuses them."""
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    buf = torch.full((3400, 3400), 4.0, dtype=torch.float64, device=cuda)
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.ozk2_dgemm_noalloc(0, 50000, 50000, p, 50000, p, 50000, p, 50000, 12, st) == 0
    assert lib.ozk2_dgemm_noalloc(50000, 0, 50000, p, 50000, p, 1, p, 1, 12, st) == 0
    torch.cuda.synchronize()
    assert (buf == 4.0).all().item()
    # k = 0 with a 3400 x 3400 output: C = 0 (its workspace would exceed the array)
    assert ozk.workspace_size(3400, 3400, 1, 12) > 256 * 1024 * 1024
    assert lib.ozk2_dgemm_noalloc(3400, 3400, 0, p, 1, p, 3400, p, 3400, 12, st) == 0
    torch.cuda.synchronize()
    assert (buf == 0.0).all().item()
    big = 2**21
    assert lib.ozk2_dgemm_noalloc(big, 4, 4, p, 4, p, 4, p, 4, 12, st) == 2  # as ozk2_dgemm
    assert lib.ozk2_dgemm(big, 4, 4, p, 4, p, 4, p, 4, 12, st) == 2
    assert lib.ozk2_dgemm_noalloc(4, 4, 4, p, 4, p, 4, p, 4, 21, st) == 1


def test_noalloc_rejects_problems_beyond_its_workspace(cuda):
    lib = _lib.load()
    m = n = k = 4096
    assert ozk.workspace_size(m, n, k, 12) > 256 * 1024 * 1024
    A = torch.zeros((8, 8), dtype=torch.float64, device=cuda)  # never touched
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.ozk2_dgemm_noalloc(m, n, k, ctypes.c_void_p(A.data_ptr()), k, ctypes.c_void_p(A.data_ptr()), n,
                               ctypes.c_void_p(A.data_ptr()), n, 12, st)
    assert s == 2  # OZK2_ERR_UNSUPPORTED
    assert torch.count_nonzero(A).item() == 0
