"""ozk2_dgemm_host: host buffers in and out, copies pipelined with the kernels.

The device arithmetic is that of the device-buffer call, so every result must be
bit-identical to ozk2_dgemm / ozk2_dgemm_ex on the same inputs: square and ragged
shapes, shapes that split into several output row blocks, transposed host views,
pinned and pageable memory, fast mode, caller workspace, back-to-back asynchronous
calls, non-finite inputs and the empty cases.
"""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _host(X, pinned):
    return X.pin_memory() if pinned else X.clone()


@pytest.mark.parametrize("m,n,k,N,mode,pinned", [
    (300, 260, 200, 12, "accurate", True),
    (17, 5, 3, 12, "accurate", False),
    (4096, 4096, 512, 12, "accurate", True),   # four output row blocks
    (4000, 3000, 700, 13, "fast", True),       # three ragged row blocks
    (2048, 4096, 300, 12, "accurate", False),  # two blocks, pageable memory
    (3, 40, 70, 12, "accurate", True),         # fewer rows than upload chunks
    (515, 300, 260, 14, "fast", True),         # ragged chunks of A, fast mode
])
def test_bit_identical_to_device_call(cuda, m, n, k, N, mode, pinned):
    A, B = workloads.problem(m, n, k, 1.0, seed=30)
    C = ozk.dgemm_host(_host(A, pinned), _host(B, pinned), num_moduli=N, mode=mode)
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N, mode=mode).cpu()
    assert torch.equal(C.view(torch.int64), ref.view(torch.int64))
    assert ozk.device_status() == "OZK2_OK"


def test_column_maxima_from_the_last_chunk(cuda):
    # A's chunks are bounded and converted while later chunks upload; the column
    # exponents must still see every chunk: here the largest rows sit in the last one,
    # and a zero row sits in the first.
    m, n, k = 1000, 700, 300
    A, B = workloads.problem(m, n, k, 1.0, seed=31)
    A = A * torch.exp2(torch.linspace(-30, 30, m, dtype=torch.float64)).unsqueeze(1)
    A[5] = 0
    for mode in ("accurate", "fast"):
        C = ozk.dgemm_host(A.pin_memory(), B.pin_memory(), num_moduli=12, mode=mode)
        ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12, mode=mode).cpu()
        assert torch.equal(C.view(torch.int64), ref.view(torch.int64))
    assert ozk.device_status() == "OZK2_OK"


def test_pipelined_calls_with_inputs_ready(cuda):
    # Back-to-back calls with OZK2_HOST_INPUTS_READY upload while the previous call
    # computes; a device-buffer call, a change of shape or of mode in between must fall
    # back to waiting for the stream.  Every result must equal its device-buffer call.
    s1, s2 = (1500, 1300, 700), (900, 1100, 500)
    shapes = [s1, s1, s1, s1, s2, s2, s2, s2]
    modes = ["accurate"] * 6 + ["fast"] * 2
    probs = [workloads.problem(m, n, k, 1.0, seed=40 + i) for i, (m, n, k) in enumerate(shapes)]
    outs = [torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64).pin_memory() for A, B in probs]
    hosts = [(A.pin_memory(), B.pin_memory()) for A, B in probs]
    mid = None
    for i, ((hA, hB), o) in enumerate(zip(hosts, outs)):
        ozk.dgemm_host(hA, hB, num_moduli=12, out=o, sync=False, inputs_ready=True, mode=modes[i])
        if i == 1:  # a device-buffer call in the same owned workspace
            A, B = probs[0]
            mid = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12)
    torch.cuda.current_stream().synchronize()
    for i, ((A, B), o) in enumerate(zip(probs, outs)):
        ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12, mode=modes[i]).cpu()
        assert torch.equal(o.view(torch.int64), ref.view(torch.int64)), i
    assert torch.equal(mid.cpu().view(torch.int64), outs[0].view(torch.int64))
    assert ozk.device_status() == "OZK2_OK"


def test_inputs_ready_with_caller_workspace(cuda):
    # a caller workspace never takes the early start: the flag only asserts the inputs
    m, n, k = 700, 500, 900
    ws = torch.empty(ozk.workspace_size_host(m, n, k, 12), dtype=torch.uint8, device=cuda)
    probs = [workloads.problem(m, n, k, 1.0, seed=60 + i) for i in range(3)]
    # the host inputs must outlive the asynchronous calls (a freed pinned block could be
    # handed to the next pin_memory() while its upload is still pending)
    hosts = [(A.pin_memory(), B.pin_memory()) for A, B in probs]
    outs = []
    for hA, hB in hosts:
        outs.append(ozk.dgemm_host(hA, hB, num_moduli=12, workspace=ws, sync=False, inputs_ready=True))
    torch.cuda.current_stream().synchronize()
    for (A, B), o in zip(probs, outs):
        ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=12).cpu()
        assert torch.equal(o.view(torch.int64), ref.view(torch.int64))


@pytest.mark.parametrize("ta,tb", [(True, False), (False, True), (True, True)])
def test_transposed_host_views(cuda, ta, tb):
    m, n, k, N = 600, 520, 333, 12
    A, B = workloads.problem(m, n, k, 0.5, seed=31)
    hA = A.T.contiguous().pin_memory().T if ta else A.pin_memory()
    hB = B.T.contiguous().pin_memory().T if tb else B.pin_memory()
    C = ozk.dgemm_host(hA, hB, num_moduli=N)
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N).cpu()
    assert torch.equal(C, ref)
    sc = ozk.scales(A.to(cuda), B.to(cuda), num_moduli=N)
    r = oz.ozk2_dgemm(A.numpy(), B.numpy(), N, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy())
    assert np.array_equal(C.numpy().view(np.uint64), r["C"].view(np.uint64))


def test_strided_host_output_and_workspace(cuda):
    m, n, k, N = 250, 190, 140, 14
    A, B = workloads.problem(m, n, k, 1.0, seed=32)
    big = torch.full((m, n + 9), 7.0, dtype=torch.float64).pin_memory()
    out = big[:, :n]
    need = ozk.workspace_size_host(m, n, k, N)
    assert need >= ozk.workspace_size(m, n, k, N) + 8 * (m * k + k * n + m * n)
    ws = torch.empty(need, dtype=torch.uint8, device=cuda)
    ozk.dgemm_host(A.pin_memory(), B.pin_memory(), num_moduli=N, out=out, workspace=ws)
    ref = ozk.dgemm(A.to(cuda), B.to(cuda), num_moduli=N).cpu()
    assert torch.equal(out, ref)
    assert torch.all(big[:, n:] == 7.0)  # the padding columns are untouched
    assert ozk.device_status(workspace=ws) == "OZK2_OK"
    with pytest.raises(ozk.Ozk2Error):
        ozk.dgemm_host(A, B, num_moduli=N, workspace=ws[: need - 256])


def test_back_to_back_asynchronous_calls(cuda):
    m, n, k, N = 1024, 768, 640, 12
    A1, B1 = workloads.problem(m, n, k, 1.0, seed=33)
    A2, B2 = workloads.problem(m, n, k, 2.0, seed=35)
    h = [(A1.pin_memory(), B1.pin_memory()), (A2.pin_memory(), B2.pin_memory())]
    outs = [torch.empty((m, n), dtype=torch.float64).pin_memory() for _ in range(3)]
    ozk.dgemm_host(*h[0], num_moduli=N, out=outs[0], sync=False)
    ozk.dgemm_host(*h[1], num_moduli=N, out=outs[1], sync=False)
    ozk.dgemm_host(*h[0], num_moduli=N, out=outs[2], sync=False)
    torch.cuda.current_stream().synchronize()
    r1 = ozk.dgemm(A1.to(cuda), B1.to(cuda), num_moduli=N).cpu()
    r2 = ozk.dgemm(A2.to(cuda), B2.to(cuda), num_moduli=N).cpu()
    assert torch.equal(outs[0], r1) and torch.equal(outs[1], r2) and torch.equal(outs[2], r1)


def test_nonfinite_and_empty(cuda):
    A, B = workloads.problem(300, 200, 100, 1.0, seed=36)
    A[250, 3] = float("inf")
    C = ozk.dgemm_host(A.pin_memory(), B.pin_memory(), num_moduli=12)
    assert ozk.device_status() == "OZK2_ERR_NONFINITE"
    assert torch.all(torch.isnan(C[250])) and not torch.any(torch.isnan(C[:250]))
    Z = ozk.dgemm_host(torch.ones(4, 0, dtype=torch.float64), torch.ones(0, 3, dtype=torch.float64))
    assert Z.shape == (4, 3) and torch.all(Z == 0)
    E = ozk.dgemm_host(torch.ones(0, 5, dtype=torch.float64), torch.ones(5, 3, dtype=torch.float64))
    assert E.shape == (0, 3)
