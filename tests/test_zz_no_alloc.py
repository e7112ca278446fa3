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
