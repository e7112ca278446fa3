"""The two tile widths of the FP8 products (128 x 256 and 128 x 128 output tiles): the
residue products (Eq. CRTmatmul) are bit-exact against the oracle with either width, the
full emulated product is bit-identical between them, the raw FP8 product is exact, a
batch plan runs with the width it was created with, and the tuner's measured choices are
valid settings."""
import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,N", [(200, 100, 300, 12), (129, 300, 700, 13), (64, 64, 64, 12),
                                     (300, 520, 257, 16), (7, 130, 33000, 12)])
def test_narrow_tile_residue_products_bit_exact(cuda, m, n, k, N):
    A, B = workloads.problem(m, n, k, 1.0, seed=m + n)
    Ad, Bd = A.to(cuda), B.to(cuda)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    with ozk.tile_width(128):
        res = ozk.residue_products(Ad, Bd, sc["e"], sc["f"], num_moduli=N).cpu().numpy()
        C128 = ozk.dgemm(Ad, Bd, num_moduli=N)
    with ozk.tile_width(256):
        C256 = ozk.dgemm(Ad, Bd, num_moduli=N)
    assert ozk.device_status() == "OZK2_OK"
    e, f = sc["e"].cpu().numpy().astype(np.int64), sc["f"].cpu().numpy().astype(np.int64)
    da = oz.scaled_decomposition(A.numpy(), e)
    db = oz.scaled_decomposition(B.numpy().T, f)
    for l, p in enumerate(oz.hybrid_moduli(N)):
        pa = oz.digit_split(oz.residues_of_decomposition(*da, p), p)
        pb = [x.T for x in oz.digit_split(oz.residues_of_decomposition(*db, p), p)]
        assert np.array_equal(res[l].astype(np.int64), np.asarray(oz.residue_product(pa, pb, p), dtype=np.int64)), p
    assert torch.equal(C128, C256)


def test_narrow_tile_raw_product_exact(cuda):
    m, n, k = 300, 200, 1024  # row strides of the raw hook are multiples of 16 bytes
    g = torch.Generator().manual_seed(3)
    a = torch.randint(-16, 17, (m, k), generator=g).to(torch.float32)
    b = torch.randint(-16, 17, (n, k), generator=g).to(torch.float32)
    a8 = a.to(torch.float8_e4m3fn).view(torch.uint8).to(cuda)
    b8 = b.to(torch.float8_e4m3fn).view(torch.uint8).to(cuda)
    with ozk.tile_width(128):
        D = ozk.fp8_gemm(a8, b8)
    assert torch.equal(D.cpu(), a @ b.T)


def test_tile_setting_and_plans(cuda):
    lib = _lib.load()
    assert lib.ozk2_set_tile_n(100) == -1
    prev = lib.ozk2_set_tile_n(0)
    assert lib.ozk2_set_tile_n(prev) == 0
    shapes = [(100, 70, 300), (300, 100, 64), (64, 60, 1000), (257, 120, 65)]
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=4, device=cuda)
    singles = [ozk.dgemm(A, B, num_moduli=12) for A, B in zip(As, Bs)]
    for t in (128, 256):
        plan = ozk.BatchPlan(As, Bs, num_moduli=12, tile_n=t)
        assert plan.tile_n() == t
        outs = plan.execute()
        assert plan.status() == "OZK2_OK"
        assert all(torch.equal(C, D) for C, D in zip(outs, singles))
        plan.close()
    auto = ozk.BatchPlan(As, Bs, num_moduli=12)
    assert auto.tile_n() == 128  # these narrow shapes pad a 256-wide tile by far more than a quarter
    auto.close()


def test_plan_with_both_tile_widths(cuda):
    """By default a plan gives each problem the tile width of a single call: narrow or
    ragged problems 128, the rest 256, in one grouped launch per width (the plan reports
    0).  Outputs are bit-identical to single calls, also inside a CUDA graph and with the
    tile setting fixed afterwards."""
    shapes = [(300, 100, 500), (200, 512, 700), (130, 1000, 64), (64, 256, 2000), (257, 384, 129)]
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=8, device=cuda)
    singles = [ozk.dgemm(A, B, num_moduli=12) for A, B in zip(As, Bs)]
    plan = ozk.BatchPlan(As, Bs, num_moduli=12, tile_n=0)
    assert plan.tile_n() == 0
    outs = plan.execute()
    assert plan.status() == "OZK2_OK"
    assert all(torch.equal(C, D) for C, D in zip(outs, singles))
    assert ozk.last_launch_count() == 10  # the residue products in two launches
    for C in outs:
        C.fill_(float("nan"))
    side = torch.cuda.Stream(cuda)
    side.wait_stream(torch.cuda.current_stream(cuda))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute()
    torch.cuda.current_stream(cuda).wait_stream(side)
    graph.replay()
    torch.cuda.synchronize(cuda)
    assert all(torch.equal(C, D) for C, D in zip(outs, singles))
    plan.close()


def test_tuner_choices(cuda):
    A, B = workloads.problem(512, 200, 700, 1.0, seed=5, device=cuda)
    t, times = ozk.choose_tile(A, B, 12, reps=2)
    assert t in (128, 256) and set(times) == {128, 256}
    shapes = workloads.batch_shapes(12, 64, 512, seed=1)
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=6, device=cuda)
    N, tile, rep = ozk.choose_plan(As, Bs, "fp64", probes=2, reps=2)
    assert 8 <= N <= 20 and tile in (0, 128, 256) and set(rep["plan_ms"]) == {0, 128, 256}


@pytest.mark.parametrize("m,n,k,N,kmax", [(200, 300, 500, 12, 4096), (130, 260, 33000, 13, 1 << 20),
                                          (300, 128, 129, 6, 4096), (64, 70, 2048, 16, 4096)])
def test_split_square_passes_bit_exact(cuda, m, n, k, N, kmax):
    """Square moduli as two single-slot passes (X parked, then Z) give the residues of the
    one-pass form, also across exactness blocks (k > 2^15 with the split forced on)."""
    lib = _lib.load()
    A, B = workloads.problem(m, n, k, 1.0, seed=k + 7)
    Ad, Bd = A.to(cuda), B.to(cuda)
    sc = ozk.scales(Ad, Bd, num_moduli=N)
    prev = lib.ozk2_set_square_split(kmax)
    try:
        split = ozk.residue_products(Ad, Bd, sc["e"], sc["f"], num_moduli=N)
        C_split = ozk.dgemm(Ad, Bd, num_moduli=N)
        lib.ozk2_set_square_split(0)
        whole = ozk.residue_products(Ad, Bd, sc["e"], sc["f"], num_moduli=N)
        C_whole = ozk.dgemm(Ad, Bd, num_moduli=N)
    finally:
        lib.ozk2_set_square_split(prev)
    assert torch.equal(split, whole)
    assert torch.equal(C_split, C_whole)
    res = split.cpu().numpy()
    e, f = sc["e"].cpu().numpy().astype(np.int64), sc["f"].cpu().numpy().astype(np.int64)
    da = oz.scaled_decomposition(A.numpy(), e)
    db = oz.scaled_decomposition(B.numpy().T, f)
    for l, p in enumerate(oz.hybrid_moduli(N)[:6]):
        pa = oz.digit_split(oz.residues_of_decomposition(*da, p), p)
        pb = [x.T for x in oz.digit_split(oz.residues_of_decomposition(*db, p), p)]
        assert np.array_equal(res[l].astype(np.int64), np.asarray(oz.residue_product(pa, pb, p), dtype=np.int64)), p
