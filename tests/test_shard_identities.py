"""The two ways the method shards over GPUs, checked on CPU ranks (gloo, world size 2)
with the oracle's steps: the library itself runs one problem on one GPU and has no
exchange step, so the identities a sharded run relies on are tested here.

* Rows of A (output rows) per rank: the row exponents e_i need only rank-local data;
  the column exponents f_j need max_i cbar_ij over ALL rows, one all-reduce(max) of S.
  With it, every rank's C rows are bit-identical to the single-process result.
* k split: each rank holds A[:, K_r], B[K_r, :]. Given the exponents, the residue
  products are additive: mod(sum_r C'_l,r, p) (one all-reduce(sum) of the N int planes,
  then mod p) equals the single-process C'_l, and so does C. Without the global bound
  product, summing the per-rank bound maxima (an upper bound of the global maxima) gives
  conservative exponents for which the Ozaki-II condition still holds exactly.
"""
import os
import sys

import numpy as np
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 12
M_, N_, K_ = 12, 10, 40


def _problem():
    rng = np.random.default_rng(123)
    A = (rng.random((M_, K_)) - 0.5) * np.exp(rng.standard_normal((M_, K_)))
    B = (rng.random((K_, N_)) - 0.5) * np.exp(rng.standard_normal((K_, N_)))
    return A, B


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _rows_worker(rank, world, port, out):
    from oracle import ozaki2 as oz

    dist = _init(rank, world, port)
    A, B = _problem()
    rows = np.array_split(np.arange(M_), world)[rank]
    Ar = A[rows]
    moduli = oz.hybrid_moduli(N)
    pprime, delta = oz.p_prime_constant(moduli), oz.delta_constant()
    ep = oz.prelim_exponent_rows(Ar)
    fp = oz.prelim_exponent_rows(B.T)
    cbar = oz.bound_product(oz.bound_operand(Ar, ep), oz.bound_operand(B.T, fp).T, K_)
    R = cbar.max(axis=1)
    S = torch.from_numpy(cbar.max(axis=0).astype(np.float32))
    dist.all_reduce(S, op=dist.ReduceOp.MAX)  # the one exchange of the row sharding
    S = S.numpy()
    zr, zc = ~np.any(Ar != 0, axis=1), ~np.any(B != 0, axis=0)
    e = np.array([oz.final_exponent(ep[i], R[i], pprime, delta, zr[i]) for i in range(len(rows))])
    f = np.array([oz.final_exponent(fp[j], S[j], pprime, delta, zc[j]) for j in range(N_)])
    C = oz.ozk2_dgemm(Ar, B, N, e=e, f=f)["C"]
    out.put((rank, rows.tolist(), e.tolist(), f.tolist(), C))
    dist.destroy_process_group()


def _ksplit_worker(rank, world, port, out):
    from oracle import ozaki2 as oz

    dist = _init(rank, world, port)
    A, B = _problem()
    ks = np.array_split(np.arange(K_), world)[rank]
    Ak, Bk = A[:, ks], B[ks]
    full = oz.scaling_exponents(A, B, N)  # exponents as the exchange would give them
    e, f = full["e"], full["f"]
    moduli = oz.hybrid_moduli(N)
    Aint, Bint = oz.integer_rows(Ak, e), oz.integer_cols(Bk, f)
    planes = []
    for p in moduli:
        pa = oz.digit_planes(Aint, p)
        pb = [x.T for x in oz.digit_planes(Bint.T, p)]
        planes.append(np.asarray(oz.residue_product(pa, pb, p), dtype=np.int64))
    R = torch.from_numpy(np.stack(planes))
    dist.all_reduce(R, op=dist.ReduceOp.SUM)  # the one exchange of the k split
    residues = [np.asarray(oz.smod(R[l].numpy().astype(object), p), dtype=np.int64) for l, p in enumerate(moduli)]
    C = oz.unscale(oz.crt_reconstruct(residues, moduli), e, f)
    # conservative exponents without the global bound product: global row/column maxima
    # (all-reduce max) and the per-rank bound maxima summed (all-reduce sum, exact in fp64)
    rowmax = torch.from_numpy(np.abs(Ak).max(axis=1))
    colmax = torch.from_numpy(np.abs(Bk).max(axis=0))
    dist.all_reduce(rowmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(colmax, op=dist.ReduceOp.MAX)
    ep = oz.prelim_exponent_rows(rowmax.numpy()[:, None])
    fp = oz.prelim_exponent_rows(colmax.numpy()[:, None])
    cbar = oz.bound_product(oz.bound_operand(Ak, ep), oz.bound_operand(Bk.T, fp).T, K_)
    Rs = torch.from_numpy(cbar.max(axis=1).astype(np.float64))
    Ss = torch.from_numpy(cbar.max(axis=0).astype(np.float64))
    dist.all_reduce(Rs, op=dist.ReduceOp.SUM)
    dist.all_reduce(Ss, op=dist.ReduceOp.SUM)
    pprime, delta = oz.p_prime_constant(moduli), oz.delta_constant()
    Rs32 = np.array([oz.f32_round_up(oz.Fraction(float(x))) for x in Rs.numpy()], dtype=np.float32)
    Ss32 = np.array([oz.f32_round_up(oz.Fraction(float(x))) for x in Ss.numpy()], dtype=np.float32)
    ec = np.array([oz.final_exponent(ep[i], Rs32[i], pprime, delta, rowmax[i] == 0) for i in range(M_)])
    fc = np.array([oz.final_exponent(fp[j], Ss32[j], pprime, delta, colmax[j] == 0) for j in range(N_)])
    out.put((rank, C, residues, e.tolist(), f.tolist(), ec.tolist(), fc.tolist()))
    dist.destroy_process_group()


def _run(worker, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() % 1000)
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


def test_row_sharding_matches_single_process():
    from oracle import ozaki2 as oz

    A, B = _problem()
    ref = oz.ozk2_dgemm(A, B, N, keep=True)
    res = _run(_rows_worker)
    C = np.zeros((M_, N_))
    for rank, rows, e, f, Cr in res:
        assert e == ref["e"][rows].tolist()
        assert f == ref["f"].tolist()  # identical column exponents on every rank
        C[rows] = Cr
    assert np.array_equal(C.view(np.uint64), ref["C"].view(np.uint64))


def test_k_split_residues_add_mod_p():
    from oracle import ozaki2 as oz

    A, B = _problem()
    ref = oz.ozk2_dgemm(A, B, N, keep=True)
    res = _run(_ksplit_worker)
    for rank, C, residues, e, f, ec, fc in res:
        for got, want in zip(residues, ref["residues"]):
            assert np.array_equal(got, want)
        assert np.array_equal(C.view(np.uint64), ref["C"].view(np.uint64))
    # the conservative exponents: never larger than the global ones, condition exact
    _, _, _, e, f, ec, fc = res[0]
    assert all(a <= b for a, b in zip(ec, e)) and all(a <= b for a, b in zip(fc, f))
    r = oz.ozk2_dgemm(A, B, N, e=np.array(ec), f=np.array(fc), keep=True)
    P = oz.product_P(r["moduli"])
    lhs = 2 * np.abs(r["Aint"]).astype(object).dot(np.abs(r["Bint"]).astype(object))
    assert max(int(v) for v in lhs.flat) < P
