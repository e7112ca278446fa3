"""Batched products (one launch per phase for a whole batch) through the C ABI.

Every C_i of a batch must be bit-identical to the single-problem call on the same
operands (which the other parity tests tie to the oracle); a few small problems are
also checked against the oracle directly.  Covered: an uneven batch of 512 products
with sizes log-uniform on [64, 2048], a mixed batch with ragged, tiny, k = 0 and
m = 0 problems in both scaling modes, plan reuse with new operand contents, CUDA graph
capture of the plan, non-finite inputs in one problem, the caller workspace.
"""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _device(As, Bs, cuda):
    return [A.to(cuda) for A in As], [B.to(cuda) for B in Bs]


def _same(x, y):
    return torch.equal(x.view(torch.int64), y.view(torch.int64))


@pytest.mark.parametrize("mode", ["accurate", "fast"])
def test_mixed_batch_matches_single_calls(cuda, mode):
    shapes = [(300, 260, 200), (1, 1, 1), (17, 5, 3), (128, 256, 128), (129, 257, 129), (5, 7, 0),
              (0, 9, 4), (640, 100, 1500), (64, 64, 64), (33, 700, 70), (2, 3, 40000)]
    As, Bs = _device(*workloads.batch_problems(shapes, 1.0, seed=40), cuda)
    Cs = ozk.dgemm_batched(As, Bs, num_moduli=13, mode=mode)
    assert ozk.device_status() == "OZK2_OK"
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        ref = ozk.dgemm(A, B, num_moduli=13, mode=mode)
        assert _same(C, ref), (i, shapes[i])
    # two small problems straight against the oracle
    for i in (2, 4):
        A, B = As[i].cpu().numpy(), Bs[i].cpu().numpy()
        sc = ozk.scales(As[i], Bs[i], num_moduli=13, mode=mode)
        r = oz.ozk2_dgemm(A, B, 13, e=sc["e"].cpu().numpy(), f=sc["f"].cpu().numpy(), mode=mode)
        assert np.array_equal(Cs[i].cpu().numpy().view(np.uint64), r["C"].view(np.uint64))


def test_uneven_batch_of_512(cuda):
    shapes = workloads.batch_shapes(512, 64, 2048, seed=0)
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=0, device=cuda)
    plan = ozk.BatchPlan(As, Bs, num_moduli=12)
    Cs = plan.execute()
    assert plan.status() == "OZK2_OK"
    for i in range(512):
        ref = ozk.dgemm(As[i], Bs[i], num_moduli=12)
        assert _same(Cs[i], ref), (i, shapes[i])
    plan.close()


def test_plan_reuse_and_graph_capture(cuda):
    shapes = [(200, 150, 300), (64, 700, 90), (1000, 64, 64)]
    As, Bs = _device(*workloads.batch_problems(shapes, 0.5, seed=50), cuda)
    plan = ozk.BatchPlan(As, Bs, num_moduli=12)
    plan.execute()
    first = [C.clone() for C in plan.outs]
    # new contents at the same addresses
    As2, Bs2 = workloads.batch_problems(shapes, 2.0, seed=60, device=cuda)
    for X, Y in zip(As + Bs, As2 + Bs2):
        X.copy_(Y)
    plan.execute()
    for A, B, C, C0 in zip(As, Bs, plan.outs, first):
        assert _same(C, ozk.dgemm(A, B, num_moduli=12))
        assert not torch.equal(C, C0)
    # capture one execution and replay it on restored inputs
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.execute()  # warm-up on the capture stream (kernel attributes are set once)
        with torch.cuda.graph(graph, stream=s):
            plan.execute()
    torch.cuda.current_stream().wait_stream(s)
    for C in plan.outs:
        C.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for A, B, C in zip(As, Bs, plan.outs):
        assert _same(C, ozk.dgemm(A, B, num_moduli=12))
    plan.close()


def test_nonfinite_and_caller_workspace(cuda):
    shapes = [(100, 80, 60), (50, 40, 30), (70, 90, 110)]
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=70)
    As[1][7, 3] = float("nan")
    As, Bs = _device(As, Bs, cuda)
    need = ozk.workspace_size_batched(shapes, num_moduli=12)
    ws = torch.empty(need, dtype=torch.uint8, device=cuda)
    Cs = ozk.dgemm_batched(As, Bs, num_moduli=12, workspace=ws)
    assert ozk.device_status(workspace=ws) == "OZK2_ERR_NONFINITE"
    assert torch.all(torch.isnan(Cs[1][7])) and torch.isnan(Cs[1]).sum() == Cs[1].shape[1]
    assert not torch.any(torch.isnan(Cs[0])) and not torch.any(torch.isnan(Cs[2]))
    for i in (0, 2):
        assert _same(Cs[i], ozk.dgemm(As[i], Bs[i], num_moduli=12))
    with pytest.raises(ozk.Ozk2Error):
        ozk.dgemm_batched(As, Bs, num_moduli=12, workspace=ws[: need - 256])


def test_single_call_graph_capture(cuda):
    """One ozk2_dgemm call captured into a CUDA graph (after a warm-up call of the same
    size, which sizes the workspace) replays the method on new operand contents."""
    A, B = workloads.problem(300, 200, 500, 1.0, seed=80, device=cuda)
    C = torch.empty((300, 200), dtype=torch.float64, device=cuda)
    ozk.dgemm(A, B, num_moduli=12, out=C)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            ozk.dgemm(A, B, num_moduli=12, out=C)
    torch.cuda.current_stream().wait_stream(s)
    A2, B2 = workloads.problem(300, 200, 500, 2.0, seed=82, device=cuda)
    A.copy_(A2)
    B.copy_(B2)
    C.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert _same(C, ozk.dgemm(A2, B2, num_moduli=12))
