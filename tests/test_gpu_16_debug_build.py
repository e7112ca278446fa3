"""The debug build (libozk2_debug.so, -DOZK2_DEBUG): the kernels check that every FP8
digit written is |d| <= 16 (Sec. III-B: digits are exact E4M3 integers) and every residue
product lies in its symmetric range; a failed check sets a flag that ozk2_device_status
reports as OZK2_ERR_INTERNAL (no trap).  On ordinary, long-reduction, large-N and
extreme-exponent inputs it must run clean and give the release build's results bit for
bit."""
import ctypes

import pytest
import torch

from paper_2603_10634_gb300 import _lib, build, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib(cuda):
    return _lib.load(build.build(debug=True))


def _call(lib, A, B, N, C):
    m, k = A.shape
    n = B.shape[1]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ozk2_dgemm(m, n, k, ctypes.c_void_p(A.data_ptr()), k, ctypes.c_void_p(B.data_ptr()), n,
                          ctypes.c_void_p(C.data_ptr()), n, N, st)


@pytest.mark.parametrize("m,n,k,N,phi", [(300, 260, 500, 12, 1.0), (129, 300, 70000, 14, 1.0),
                                         (64, 100, 300, 20, 2.0), (257, 64, 33, 6, 4.0)])
def test_debug_build_runs_clean(cuda, debug_lib, m, n, k, N, phi):
    release = _lib.load()
    A, B = workloads.problem(m, n, k, phi, seed=m + k, device=cuda)
    A[0] *= 2.0**-900  # a row of tiny entries: large exponents, the 2^t mod p path
    Cd = torch.empty((m, n), dtype=torch.float64, device=cuda)
    Cr = torch.empty_like(Cd)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _call(debug_lib, A, B, N, Cd) == 0
    assert debug_lib.ozk2_device_status(None, st) == 0
    assert _call(release, A, B, N, Cr) == 0
    assert release.ozk2_device_status(None, st) == 0
    torch.cuda.synchronize()
    assert torch.equal(Cd, Cr)
