"""Moduli-count autotuner: the smallest N that meets a requested accuracy.

The accuracy of the emulation is set by the scaling exponents (Sec. III-E): adding a
modulus raises P, hence e_i and f_j by about half its bit length, and the truncation
error 2^-e_i, 2^-f_j falls accordingly.  How many moduli a problem needs depends on its
data (phi, k, the spread of its rows and columns), so the tuner measures it: for each
candidate N it takes the exponents of the WHOLE problem (the real scaling, computed by
the library's scaling kernels), emulates a sampled block of rows and columns of C with
them, and compares the block with the same block emulated at N = 20 (whose error is the
final FP64 rounding alone).

The tile width of the FP8 products (128 x 256 or 128 x 128 output tiles) does not change
any result bit, only the time: choose_tile times a problem with both widths and
choose_plan times a whole batch plan with both (after choose_moduli_batch has fixed N).
The k-block is not a tunable: it is set by exactness (2^15 terms for the square moduli'
shared accumulator, 2^16 for the Karatsuba moduli; Eq. error-free-FP8-matmult).

Every step runs in libozk2's kernels; torch.matmul appears only as the native-FP64
yardstick of target="fp64" and for the |A||B| normaliser of the sampled block.
"""
from __future__ import annotations

import torch

from . import ozk2

REFERENCE_MODULI = 20


def _sample_indices(count, size, generator, device):
    if size <= count:
        return torch.arange(size, device=device)
    return torch.randperm(size, generator=generator)[:count].sort().values.to(device)


def _block(A, B, e, f, rows, cols, N):
    """The sampled block of C emulated with the given exponents of the whole problem."""
    Ab = A.index_select(0, rows).contiguous()
    Bb = B.index_select(1, cols).contiguous()
    eb = e.index_select(0, rows).contiguous()
    fb = f.index_select(0, cols).contiguous()
    return ozk2.crt(ozk2.residue_products(Ab, Bb, eb, fb, N), eb, fb, N)


def sampled_errors(A, B, candidates, mode="accurate", rows=128, cols=128, seed=0):
    """{N: max_ij |C_ij - C*_ij| / (|A||B|)_ij} over a sampled block, C* the N = 20
    emulation; plus the native FP64 error of the same block under the key "native"."""
    dev = A.device
    g = torch.Generator()
    g.manual_seed(int(seed))
    r = _sample_indices(rows, A.shape[0], g, dev)
    c = _sample_indices(cols, B.shape[1], g, dev)
    sc = ozk2.scales(A, B, num_moduli=REFERENCE_MODULI, mode=mode)
    ref = _block(A, B, sc["e"], sc["f"], r, c, REFERENCE_MODULI)
    Ab, Bb = A.index_select(0, r), B.index_select(1, c)
    absab = torch.matmul(Ab.abs(), Bb.abs())
    scale = torch.where(absab > 0, absab, torch.ones_like(absab))
    out = {"native": float(((torch.matmul(Ab, Bb) - ref).abs() / scale).max())}
    for N in candidates:
        sc = ozk2.scales(A, B, num_moduli=N, mode=mode)
        blk = _block(A, B, sc["e"], sc["f"], r, c, N)
        out[N] = float(((blk - ref).abs() / scale).max())
    return out


def choose_moduli(A, B, target="fp64", mode="accurate", candidates=range(8, 21), margin=1.0, rows=128, cols=128,
                  seed=0):
    """Smallest N in `candidates` whose sampled error is within the target.

    target: "fp64" (within 2x of native FP64 GEMM's error on the same block) or a float
    tau (relative to |A||B|).  margin < 1 asks for headroom (error <= margin * bound).
    Returns (N, report) where report holds the sampled errors."""
    cands = sorted(int(x) for x in candidates)
    if not cands or cands[0] < 1 or cands[-1] > REFERENCE_MODULI:
        raise ValueError("candidates must lie in 1..20")
    errs = sampled_errors(A, B, cands, mode, rows, cols, seed)
    if target == "fp64":
        bound = 2.0 * max(errs["native"], 2.0**-53)
    else:
        bound = float(target)
    bound *= margin
    for N in cands:
        if errs[N] <= bound:
            return N, {"bound": bound, "errors": errs}
    return cands[-1], {"bound": bound, "errors": errs}


def choose_moduli_batch(As, Bs, target="fp64", mode="accurate", probes=4, **kw):
    """One N for a batch: the largest choice over the `probes` problems with the longest
    reductions (then the largest outputs), where truncation errors accumulate most."""
    order = sorted(range(len(As)), key=lambda i: (As[i].shape[1], As[i].shape[0] * Bs[i].shape[1]), reverse=True)
    best, reports = 1, []
    for i in order[:max(1, probes)]:
        N, rep = choose_moduli(As[i], Bs[i], target, mode, **kw)
        reports.append((i, N, rep))
        best = max(best, N)
    return best, reports


def _time(fn, reps, warmup=1):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(reps):
        fn()
    s1.record()
    torch.cuda.synchronize()
    return s0.elapsed_time(s1) / reps


def choose_tile(A, B, num_moduli=12, mode="accurate", reps=3):
    """The faster tile width for this problem, measured: (tile_n, {tile_n: ms})."""
    out = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=A.device)
    times = {}
    for t in (256, 128):
        with ozk2.tile_width(t):
            times[t] = _time(lambda: ozk2.dgemm(A, B, num_moduli=num_moduli, out=out, mode=mode), reps)
    return min(times, key=times.get), times


def choose_plan(As, Bs, target="fp64", mode="accurate", probes=4, reps=3, **kw):
    """Moduli count for the requested accuracy (choose_moduli_batch) and the fastest tile
    setting of the batch plan, measured: 256 or 128 for every problem, or 0 for the
    library's per-problem widths (narrow and ragged problems in 128-wide tiles, the rest
    in 256-wide ones): (N, tile_n, report)."""
    N, reports = choose_moduli_batch(As, Bs, target, mode, probes, **kw)
    times = {}
    for t in (0, 256, 128):
        plan = ozk2.BatchPlan(As, Bs, num_moduli=N, mode=mode, tile_n=t)
        times[t] = _time(plan.execute, reps)
        plan.close()
    return N, min(times, key=times.get), {"moduli": reports, "plan_ms": times}

