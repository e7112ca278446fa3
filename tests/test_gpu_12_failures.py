"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the injected stall makes the FP8 product kernel
  wait on a barrier that nothing signals; with a short wait limit the wait gives up, the
  kernel returns (no hang, no fault), the device status reads OZK2_ERR_TIMEOUT, the
  output is not written, and the next call is OZK2_OK and correct.  Single-CTA raw
  product (ozk2_debug_fp8_gemm).
* Host-injected failures: a workspace allocation that fails (OZK2_ERR_ALLOC) and a launch
  that fails (OZK2_ERR_CUDA) leave C untouched, and the next call is bit-identical to an
  undisturbed one.
* Caller workspaces that are not device memory of this GPU are refused before anything
  is enqueued (the TMA tensor maps are only ever built over this GPU's own memory)."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from paper_2603_10634_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

ALLOC, LAUNCH, STALL = 1, 2, 3


@pytest.fixture
def lib(cuda):
    lib = _lib.load()
    lib.ozk2_debug_inject_fault(0)
    lib.ozk2_set_wait_limit(0)
    ozk.device_status()  # clear the flag word of the library-owned workspace
    yield lib
    lib.ozk2_debug_inject_fault(0)
    lib.ozk2_set_wait_limit(0)


def _fp8_operands(m, n, k, dev, seed=0):
    g = torch.Generator().manual_seed(seed)
    a = torch.randint(-16, 17, (m, k), generator=g).to(torch.float32)
    b = torch.randint(-16, 17, (n, k), generator=g).to(torch.float32)
    a8 = a.to(torch.float8_e4m3fn).view(torch.uint8).to(dev)
    b8 = b.to(torch.float8_e4m3fn).view(torch.uint8).to(dev)
    return a, b, a8, b8


def test_bounded_wait_runs_out_and_the_next_call_works(lib, cuda):
    m, n, k = 128, 256, 4096
    a, b, a8, b8 = _fp8_operands(m, n, k, cuda)
    D = torch.full((m, n), float("nan"), dtype=torch.float32, device=cuda)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        return lib.ozk2_debug_fp8_gemm(m, n, k, ctypes.c_void_p(a8.data_ptr()), k, ctypes.c_void_p(b8.data_ptr()),
                                       k, ctypes.c_void_p(D.data_ptr()), n, st)

    assert lib.ozk2_set_wait_limit(2_000_000) == 0  # 2 ms
    assert lib.ozk2_debug_inject_fault(STALL) == 0
    assert call() == 0  # the launch itself succeeds
    assert lib.ozk2_debug_inject_fault(-1) == 0  # the stall fired (one-shot)
    torch.cuda.synchronize()  # the kernel returned by itself
    assert ozk.device_status() == "OZK2_ERR_TIMEOUT"
    assert torch.isnan(D).all().item()  # the aborted epilogue wrote nothing
    lib.ozk2_set_wait_limit(0)
    assert call() == 0
    torch.cuda.synchronize()
    assert ozk.device_status() == "OZK2_OK"
    assert torch.equal(D.cpu(), a @ b.T)  # exact: |entries| <= k 16 16 < 2^24


def test_injected_allocation_failure(lib, cuda):
    A, B = workloads.problem(300, 200, 500, 1.0, seed=3, device=cuda)
    want = ozk.dgemm(A, B, num_moduli=12)
    C = torch.full_like(want, 7.0)
    assert lib.ozk2_debug_inject_fault(ALLOC) == 0
    with pytest.raises(_lib.Ozk2Error) as ei:
        ozk.dgemm(A, B, num_moduli=12, out=C)
    assert ei.value.status == 3  # OZK2_ERR_ALLOC
    torch.cuda.synchronize()
    assert (C == 7.0).all().item()
    assert ozk.device_status() == "OZK2_OK"
    ozk.dgemm(A, B, num_moduli=12, out=C)
    assert torch.equal(C, want)
    # a batch plan that allocates its own workspace reports the same
    assert lib.ozk2_debug_inject_fault(ALLOC) == 0
    with pytest.raises(_lib.Ozk2Error) as ei:
        ozk.BatchPlan([A], [B], num_moduli=12)
    assert ei.value.status == 3
    plan = ozk.BatchPlan([A], [B], num_moduli=12)
    out = plan.execute()
    assert torch.equal(out[0], want)
    plan.close()


def test_injected_launch_failure(lib, cuda):
    A, B = workloads.problem(260, 300, 700, 1.0, seed=4, device=cuda)
    want = ozk.dgemm(A, B, num_moduli=13)
    C = torch.full_like(want, 5.0)
    assert lib.ozk2_debug_inject_fault(LAUNCH) == 0
    with pytest.raises(_lib.Ozk2Error) as ei:
        ozk.dgemm(A, B, num_moduli=13, out=C)
    assert ei.value.status == 4  # OZK2_ERR_CUDA
    torch.cuda.synchronize()
    assert (C == 5.0).all().item()
    ozk.dgemm(A, B, num_moduli=13, out=C)
    assert torch.equal(C, want)
    assert ozk.device_status() == "OZK2_OK"


def test_host_memory_workspace_is_refused(lib, cuda):
    m, n, k, N = 200, 150, 300, 12
    A, B = workloads.problem(m, n, k, 1.0, seed=5, device=cuda)
    need = ozk.workspace_size(m, n, k, N)
    ws = torch.full((need + 256,), 0xA5, dtype=torch.uint8).pin_memory()
    off = (-ws.data_ptr()) % 256
    C = torch.full((m, n), 3.0, dtype=torch.float64, device=cuda)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.ozk2_dgemm_ws(m, n, k, ctypes.c_void_p(A.data_ptr()), k, ctypes.c_void_p(B.data_ptr()), n,
                          ctypes.c_void_p(C.data_ptr()), n, N, ctypes.c_void_p(ws.data_ptr() + off), need,
                          st)
    assert s == 1  # OZK2_ERR_INVALID_VALUE
    torch.cuda.synchronize()
    assert (C == 3.0).all().item()
    assert (ws == 0xA5).all().item()
    # the same for a batch plan and for the host-buffer call
    I64 = ctypes.c_int64 * 1
    P = ctypes.c_void_p * 1
    plan = ctypes.c_void_p(0)
    bneed = ozk.workspace_size_batched([(m, n, k)], N)
    wsb = torch.full((bneed + 256,), 0xA5, dtype=torch.uint8).pin_memory()
    offb = (-wsb.data_ptr()) % 256
    s = lib.ozk2_batch_plan_create(ctypes.byref(plan), 1, I64(m), I64(n), I64(k), P(A.data_ptr()), I64(k),
                                   P(B.data_ptr()), I64(n), P(C.data_ptr()), I64(n), N, 0,
                                   ctypes.c_void_p(wsb.data_ptr() + offb), bneed, st)
    assert s == 1 and not plan.value
    assert (wsb == 0xA5).all().item()
    hA, hB = A.cpu(), B.cpu()
    hC = torch.full((m, n), 3.0, dtype=torch.float64)
    hneed = ozk.workspace_size_host(m, n, k, N)
    wsh = torch.full((hneed + 256,), 0xA5, dtype=torch.uint8).pin_memory()
    offh = (-wsh.data_ptr()) % 256
    s = lib.ozk2_dgemm_host_ex(0, 0, m, n, k, ctypes.c_void_p(hA.data_ptr()), k, ctypes.c_void_p(hB.data_ptr()), n,
                               ctypes.c_void_p(hC.data_ptr()), n, N, 0, 0, ctypes.c_void_p(wsh.data_ptr() + offh),
                               hneed, st)
    assert s == 1
    torch.cuda.synchronize()
    assert (hC == 3.0).all().item() and (wsh == 0xA5).all().item()
    # and device memory of this GPU still works
    wsd = torch.empty(need + 256, dtype=torch.uint8, device=cuda)
    offd = (-wsd.data_ptr()) % 256
    s = lib.ozk2_dgemm_ws(m, n, k, ctypes.c_void_p(A.data_ptr()), k, ctypes.c_void_p(B.data_ptr()), n,
                          ctypes.c_void_p(C.data_ptr()), n, N, ctypes.c_void_p(wsd.data_ptr() + offd), need, st)
    assert s == 0
    assert torch.equal(C, ozk.dgemm(A, B, num_moduli=N))
