"""Benchmark: emulated DGEMM throughput (2mnk / t) of the FP8 Ozaki-II path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--size 16384] [--moduli 12] [--phi 1.0]

One step is one ozk2_dgemm call: scaling pass, FP8 bound product, exponents,
residues and digit planes, 3N FP8 residue products with mod-reduce, CRT and inverse
scaling, on m = n = k = 16384 float64 inputs generated on the device from the
paper's distribution (U - 0.5) exp(phi N(0,1)) (seed 0 for A, 1 for B).  Inputs
(2 GiB each) are larger than the 129 MB L2, so no flush is needed between steps.

Under torchrun (--gpus N > 1) every rank runs the same problem on its own GPU
(replicas: the method has no exchange step), ranks are fenced by barriers and
the slowest rank's time defines the step time.

--impl reference times the CPU oracle (the plain Python/numpy implementation of
the method) on the host cores, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "emulated DGEMM TFLOP/s (2mnk/t) at FP64-level error vs native FP64, 16384³"
NOMINAL_FP8_TFLOPS = 4500.0  # dense FP8 per GPU, the FP8-count roofline of the method
NOMINAL_HBM_GBS = 7700.0
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--moduli", type=int, default=12)
    ap.add_argument("--phi", type=float, default=1.0)
    ap.add_argument("--no-native", action="store_true", help="skip the native FP64 reference timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--samples", type=int, default=32, help="entries checked against the exact product")
    ap.add_argument("--mode", default="accurate", choices=["accurate", "fast"], help="scaling mode")
    ap.add_argument("--sizes", default="1024,4096,8192,16384", help="sweep: square sizes")
    ap.add_argument("--phis", default="0.5,1,2", help="sweep: phi values")
    ap.add_argument("--moduli-list", default="8,9,10,11,12,13,14,16,18,20", help="sweep: N values")
    ap.add_argument("--tile", type=int, default=None, choices=[0, 128, 256],
                    help="output tile width of the FP8 products (0: the library's rule; default: leave it)")
    ap.add_argument("--square-split", type=int, default=None,
                    help="square moduli as two passes for k up to this (0: never; default: the library's)")
    ap.add_argument("--shapes", default="4096x4096x65536,65536x1024x1024",
                    help="rect: comma-separated m x n x k shapes")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: plan with --moduli and --tile (default 0: the library's per-problem "
                         "widths) instead of the autotuner")
    ap.add_argument("--workload", default="dgemm", choices=["dgemm", "autograd", "batched", "sweep", "rect"],
                    help="dgemm: the square product above; autograd: forward + backward of "
                         "C = A B with A 8192 x 4096, B 4096 x 4096 and upstream gradient W ~ N(0, 1); "
                         "batched: 512 products with m, n, k log-uniform on [64, 2048]; "
                         "sweep: error and TFLOP/s over sizes x phi x N (one JSON line each); "
                         "rect: 4096 x 4096 x 65536 and 65536 x 1024 x 1024 (or --shapes)")
    return ap.parse_args()


def workload_config(a):
    return {
        "workload": f"square DGEMM m=n=k={a.size}, phi={a.phi}, N={a.moduli} moduli, {a.mode} mode",
        "m": a.size, "n": a.size, "k": a.size, "phi": a.phi, "num_moduli": a.moduli, "seed": 0, "mode": a.mode,
        "l2": "inputs larger than L2 (2 x 8 k^2 bytes), no flush",
        "parallelism": f"replicas x{a.gpus}" if a.gpus > 1 else "single GPU",
        "settings": {"tile_n": a.tile, "square_split_kmax": a.square_split},
    }


# ------------------------------------------------------------------ distributed
def dist_init(a):
    rank, world = 0, 1
    if a.gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist

        rank = int(os.environ.get("RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        backend = "nccl" if a.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ peaks, traffic
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_source_hash():
    """Hash of the residue-product kernel's own sources (its translation unit and the
    PTX helpers it includes)."""
    h = hashlib.sha256()
    for f in ["gemm.cu", "device.cuh"]:
        with open(os.path.join(ROOT, "paper_2603_10634_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(size, moduli):
    """DRAM bytes per residue-product launch from the committed ncu summary and how they
    were obtained, if the summary was taken on the current kernel source for this
    workload; (None, None) otherwise."""
    p = os.path.join(PROFILES, "residue_gemm_traffic.txt")
    try:
        kv = {}
        with open(p) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    key, v = line.split(":", 1)
                    kv[key.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return None, None
        if int(kv.get("size", -1)) != size or int(kv.get("num_moduli", -1)) != moduli:
            return None, None
        return float(kv["dram_bytes_per_launch"]), kv.get("traffic_method", "ncu capture")
    except (OSError, KeyError, ValueError):
        return None, None


# ------------------------------------------------------------------ exact error samples
def _exact_dot(a, b):
    """Exact sum a_h b_h of two float64 sequences, as (numerator, denominator)."""
    num, den = 0, 1
    for x, y in zip(a, b):
        x, y = float(x), float(y)
        if x == 0.0 or y == 0.0:
            continue
        nx, dx = x.as_integer_ratio()
        ny, dy = y.as_integer_ratio()
        d = dx * dy
        if d > den:
            num *= d // den
            den = d
        num += nx * ny * (den // d)
    return num, den


def error_samples(A, B, C, Cnat, samples, seed=7):
    import numpy as np
    import torch

    m, n = C.shape
    rng = np.random.default_rng(seed)
    rows = torch.as_tensor(rng.integers(0, m, samples), device=A.device)
    cols = torch.as_tensor(rng.integers(0, n, samples), device=A.device)
    Ar = A[rows].cpu().numpy()
    Bc = B[:, cols].cpu().numpy()
    Cs = C[rows, cols].cpu().numpy()
    Cn = Cnat[rows, cols].cpu().numpy() if Cnat is not None else None
    emu, nat, bound_ok = [], [], True
    k = A.shape[1]
    for t in range(samples):
        num, den = _exact_dot(Ar[t], Bc[:, t])
        anum, aden = _exact_dot(abs(Ar[t]), abs(Bc[:, t]))
        ab = anum / aden
        cn, cd = float(Cs[t]).as_integer_ratio()
        err = abs(num * cd - cn * den) / (den * cd)
        emu.append(err / ab)
        bound_ok &= err <= k * 2.0**-52 * ab
        if Cn is not None:
            nn, nd = float(Cn[t]).as_integer_ratio()
            nat.append(abs(num * nd - nn * den) / (den * nd) / ab)
    out = {"samples": samples, "max_rel_err_vs_absAB": max(emu), "bound_k_2^-52_holds": bool(bound_ok)}
    if nat:
        out["native_fp64_max_rel_err_vs_absAB"] = max(nat)
        out["within_2x_native"] = bool(max(emu) <= 2 * max(max(nat), 2.0**-53))
    return out


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(size, phi, moduli):
    """Time the oracle once on a size^3 instance of the same generator; returns seconds."""
    import numpy as np

    from oracle import ozaki2 as oz
    from paper_2603_10634_gb300 import workloads

    A, B = workloads.problem(size, size, size, phi, seed=0, device="cpu")
    A, B = A.numpy(), B.numpy()
    t0 = time.perf_counter()
    oz.ozk2_dgemm(A, B, moduli)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# The oracle runs with every BLAS / OpenMP pool pinned to one thread, so that the
# core count stated beside its time is the one it used.
ONE_THREAD_ENV = {"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                  "BLIS_NUM_THREADS": "1", "VECLIB_MAXIMUM_THREADS": "1"}


def oracle_times(sizes, phi, moduli):
    """Seconds of one oracle run per size, in a child process with one thread."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps([bench.oracle_sample(s, %r, %d) for s in %r]))" % (ROOT, phi, moduli, list(sizes)))
    env = dict(os.environ, **ONE_THREAD_ENV)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def extrapolate_seconds(t_small, t_large, s_small, s_large, target):
    """Fit t(s) = a s^2 + b s^3 (conversions and CRT grow as s^2, the digit products as
    s^3) through two timed sizes and evaluate it at `target`."""
    r = s_large / s_small
    b = (t_large - r**2 * t_small) / (s_large**3 - r**2 * s_small**3)
    a = (t_small - b * s_small**3) / s_small**2
    if a < 0 or b < 0:  # noisy small samples: fall back to pure cubic scaling of the larger one
        return t_large * (target / s_large) ** 3
    return a * target**2 + b * target**3


def cpu_baseline(a, sizes=(256, 512)):
    t = oracle_times(sizes, a.phi, a.moduli)
    s = sizes[-1]
    t_ext = extrapolate_seconds(t[0], t[1], sizes[0], sizes[1], a.size)
    return {"value": 2.0 * s**3 / t[-1] / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"full oracle pipeline on one m=n=k={s} instance of the workload's generator "
                      f"(phi={a.phi}, N={a.moduli}), {t[-1]:.2f} s, one thread (BLAS pinned to 1)",
            "extrapolated_to_workload": {"m=n=k": a.size, "seconds": t_ext,
                                         "tflops": 2.0 * a.size**3 / t_ext / 1e12,
                                         "how": f"t = a s^2 + b s^3 fitted to the oracle's times at "
                                                f"s = {sizes[0]} ({t[0]:.2f} s) and {sizes[1]} ({t[1]:.2f} s); "
                                                f"extrapolated, not measured"}}


def run_reference(a, rank, world):
    """--impl reference: the CPU oracle as it stands, one bounded sample of the workload
    per step, on one host thread."""
    if rank != 0:
        return
    os.environ.update(ONE_THREAD_ENV)  # before numpy is first imported in this process
    size = int(os.environ.get("OZK2_REFERENCE_SAMPLE", "512"))
    for _ in range(a.warmup):
        oracle_sample(size, a.phi, a.moduli)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle_sample(size, a.phi, a.moduli)
    dt = (time.perf_counter() - t0) / a.steps
    val = 2.0 * size**3 / dt / 1e12
    cfg = workload_config(a)
    cfg["workload"] += f" (reference arm: each step times the oracle on one m=n=k={size} sample of this workload)"
    cfg["reference_sample"] = {"m": size, "n": size, "k": size}
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+int", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: full oracle pipeline on one m=n=k={size} instance of the "
                                   f"workload's generator (2 {size}^3 flop per step), one thread "
                                   f"(BLAS pinned to 1)"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(a, rank, world):
    import torch

    import paper_2603_10634_gb300 as ozk
    from paper_2603_10634_gb300 import _lib, workloads

    _lib.load()  # fails loudly without the built library
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m = n = k = a.size
    N = a.moduli
    flops = 2.0 * m * n * k
    A, B = workloads.problem(m, n, k, a.phi, seed=0, device=dev)
    C = torch.empty((m, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(a.warmup):
        ozk.dgemm(A, B, num_moduli=N, out=C, mode=a.mode)
    torch.cuda.synchronize(dev)
    assert ozk.device_status() == "OZK2_OK"
    launches_per_call = ozk.last_launch_count()

    # ---- timed region: K back-to-back calls, device inputs
    ozk.set_timing(True)
    phase_sum = {p: 0.0 for p in ozk.PHASES}
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(a.steps):
            ozk.dgemm(A, B, num_moduli=N, out=C, mode=a.mode)
            ph = ozk.get_timing()  # waits for this call's last event (host-side, ~us)
            for p in ozk.PHASES:
                phase_sum[p] += ph[p]
        end.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    ozk.set_timing(False)
    ms = start.elapsed_time(end) / a.steps
    ms = max_over_ranks(ms, world, dev)
    status = ozk.device_status()
    phases = {p: v / a.steps for p, v in phase_sum.items()}
    value = world * flops / (ms * 1e-3) / 1e12

    # ---- end to end: host buffers in and out, through the public API
    e2e = None
    if not a.no_e2e:
        Cdev = C.cpu()
        hA = A.cpu().pin_memory()
        hB = B.cpu().pin_memory()
        hC = torch.empty((m, n), dtype=torch.float64).pin_memory()

        def e2e_step(ready):
            ozk.dgemm_host(hA, hB, num_moduli=N, out=hC, mode=a.mode, sync=False, inputs_ready=ready)

        # back-to-back calls, as a stream of host-resident problems would issue them:
        # each call's upload overlaps the previous call's residue products
        for _ in range(max(1, a.warmup)):
            e2e_step(True)
        torch.cuda.synchronize(dev)
        barrier(world)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(a.steps):
            e2e_step(True)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        ems = max_over_ranks(s0.elapsed_time(s1) / a.steps, world, dev)
        matches = bool(torch.equal(hC, Cdev))
        # one call at a time (nothing overlaps it): its latency and its phase ends
        ozk.set_timing(True)
        ends, lat = {}, []
        for _ in range(2):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            e2e_step(False)
            t1.record(stream)
            tl = ozk.timeline()  # waits for this call's last event (host-side)
            torch.cuda.synchronize(dev)
            lat.append(t0.elapsed_time(t1))
            for key, v in (tl or {}).items():
                ends[key] = ends.get(key, 0.0) + v / 2
        ozk.set_timing(False)
        single = sum(lat) / len(lat)
        e2e = {"value": world * flops / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": hA.numel() * 8 + hB.numel() * 8, "d2h_bytes_per_step": hC.numel() * 8,
               "ms_per_step": ems,
               "path": "ozk2_dgemm_host_ex with OZK2_HOST_INPUTS_READY, pinned host A, B, C, calls back to back: "
                       "each call's upload overlaps the previous call's residue products, its download its own",
               "single_call": {"ms": single, "tflops": flops / (single * 1e-3) / 1e12,
                               "phase_ends_ms": {"uploads done, last chunk of A scaled": ends.get("scale"),
                                                 "last chunk bounded": ends.get("bound_gemm"),
                                                 "last chunk converted": ends.get("exponents"),
                                                 "B converted": ends.get("residues"),
                                                 "last CRT": ends.get("residue_gemm"),
                                                 "last block back": ends.get("crt")}}}
        e2e["matches_device_call"] = matches and bool(torch.equal(hC, Cdev))
        # the link itself on this machine: one plain pinned copy each way
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        dA = torch.empty_like(A)
        c0.record(stream)
        dA.copy_(hA, non_blocking=True)
        c1.record(stream)
        hA.copy_(dA, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize(dev)
        nb = hA.numel() * 8
        e2e["link_h2d_gbs"] = nb / c0.elapsed_time(c1) / 1e6
        e2e["link_d2h_gbs"] = nb / c1.elapsed_time(c2) / 1e6
        e2e["copy_floor_ms"] = (hA.numel() * 8 + hB.numel() * 8) / e2e["link_h2d_gbs"] / 1e6 + \
            hC.numel() * 8 / e2e["link_d2h_gbs"] / 1e6
        del dA
        del hA, hB, hC, Cdev

    # ---- roofline of the dominant kernel (the residue-product GEMM)
    peaks, src = measured_peaks()
    fp8_peak = 2.0 * float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    gemm_flops = 3 * N * flops  # residue products only; the bound product is its own phase
    achieved = gemm_flops / (phases["residue_gemm"] * 1e-3) / 1e12
    traffic, traffic_method = recorded_traffic(a.size, N)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": fp8_peak, "unit": "TFLOP/s",
                "frac": achieved / fp8_peak, "traffic": traffic, "traffic_method": traffic_method,
                "kernel": "fp8_gemm_kernel<residue> (3N FP8 products + mod-reduce)",
                "peak_source": f"{src} bf16_tflops_sustained x 2 (dense FP8 / BF16 nominal ratio)"}
    conv_bytes = (16 + 1 + (2 * N if N <= 6 else 3 * N - 6)) * (m * k + k * n) + 8 * m * n
    t_roof = (3 * N + 1) * flops / (NOMINAL_FP8_TFLOPS * 1e12) + conv_bytes / (NOMINAL_HBM_GBS * 1e9)
    roof_tflops = flops / t_roof / 1e12
    fp8_count = {"roofline_tflops": roof_tflops, "frac": value / world / roof_tflops,
                 "definition": "(3N+1) 2mnk at 4.5 PF/s + conversion bytes at 7.7 TB/s (nominal)"}

    # ---- native FP64 reference point and error samples
    Cnat, native = None, None
    if not a.no_native:
        Cnat = torch.empty_like(C)
        torch.matmul(A, B, out=Cnat)
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        torch.matmul(A, B, out=Cnat)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        native = {"tflops": flops / (s0.elapsed_time(s1) * 1e-3) / 1e12, "impl": "torch.matmul float64 (cuBLAS)"}
    err = error_samples(A, B, C, Cnat, a.samples) if rank == 0 else None

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline(a)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f8e4m3", "emulates": "f64", "data": "synthetic",
            "config": workload_config(a), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_call * a.steps, "clocks": clk.summary(), "phases_ms": phases,
            "fp8_count_roofline": fp8_count, "native_fp64": native, "error": err, "device_status": status,
        }
        print(json.dumps(line), flush=True)


def run_autograd(a, rank, world):
    """Forward + backward of the differentiable product: C = A B, then dA = W B^T and
    dB = A^T W for the upstream gradient W; three emulated products per step.  The
    default backward reuses the forward's exponents and digit planes (one conversion of
    W for both gradients); the same step with fresh emulations of both gradients is
    timed beside it, and sampled entries of dA and dB of both are compared with the
    exact products next to native FP64."""
    import torch

    import paper_2603_10634_gb300 as ozk
    from paper_2603_10634_gb300 import _lib, workloads

    _lib.load()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, k, n, N = 8192, 4096, 4096, a.moduli
    A = workloads.phi_matrix(m, k, a.phi, 0, device=dev).requires_grad_(True)
    B = workloads.phi_matrix(k, n, a.phi, 1, device=dev).requires_grad_(True)
    W = workloads.normal_matrix(m, n, 2, device=dev)
    flops = 3 * 2.0 * m * n * k
    stream = torch.cuda.current_stream(dev)

    def make_step(reuse):
        def step():
            A.grad = None
            B.grad = None
            ozk.matmul(A, B, N, a.mode, reuse=reuse).backward(W)
        return step

    def timed(step):
        for _ in range(a.warmup):
            step()
        torch.cuda.synchronize(dev)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(a.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        return max_over_ranks(start.elapsed_time(end) / a.steps, world, dev)

    def grad_errors(samples=16, seed=9):
        import numpy as np

        rng = np.random.default_rng(seed)
        An, Bn, Wn = A.detach().cpu().numpy(), B.detach().cpu().numpy(), W.cpu().numpy()
        gA, gB = A.grad.cpu().numpy(), B.grad.cpu().numpy()
        nA, nB = (W @ B.detach().T).cpu().numpy(), (A.detach().T @ W).cpu().numpy()
        worst = {"dA": 0.0, "dA_native": 0.0, "dB": 0.0, "dB_native": 0.0}
        for _ in range(samples):
            i, j, h = int(rng.integers(0, m)), int(rng.integers(0, n)), int(rng.integers(0, k))
            for key, got, nat, x, y in (("dA", gA[i, h], nA[i, h], Wn[i], Bn[h]),
                                        ("dB", gB[h, j], nB[h, j], An[:, h], Wn[:, j])):
                num, den = _exact_dot(x, y)
                anum, aden = _exact_dot(abs(x), abs(y))
                for tag, v in ((key, got), (key + "_native", nat)):
                    cn, cd = float(v).as_integer_ratio()
                    worst[tag] = max(worst[tag], abs(num * cd - cn * den) / (den * cd) / (anum / aden))
        worst["within_2x_native"] = bool(worst["dA"] <= 2 * max(worst["dA_native"], 2.0**-53) and
                                         worst["dB"] <= 2 * max(worst["dB_native"], 2.0**-53))
        return worst

    step = make_step(True)
    step()
    # launches per step: the forward call and the backward call, counted on this thread
    # (autograd runs the backward on its own thread, whose count this thread cannot read)
    ws = torch.empty(ozk.workspace_size(m, n, k, N), dtype=torch.uint8, device=dev)
    ozk.dgemm(A.detach(), B.detach(), num_moduli=N, workspace=ws)
    fwd_launches = ozk.last_launch_count()
    ozk.dgemm_backward(A.detach(), B.detach(), W, ws, N)
    launches = fwd_launches + ozk.last_launch_count()
    del ws
    with ClockSampler(local) as clk:
        ms = timed(step)
    err_reuse = grad_errors() if rank == 0 else None
    status = ozk.device_status()
    ms_fresh = timed(make_step(False))
    err_fresh = grad_errors() if rank == 0 else None
    if rank == 0:
        line = {
            "metric": "emulated FP64 forward+backward TFLOP/s (3 x 2mnk / t)", "value": world * flops / ms / 1e9,
            "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f8e4m3", "emulates": "f64",
            "data": "synthetic",
            "config": {"workload": f"autograd A {m}x{k} @ B {k}x{n}, W ~ N(0,1), phi={a.phi}, N={N}, {a.mode} mode, "
                                   f"backward reusing the forward's exponents and digit planes",
                       "l2": "operands larger than L2, no flush"},
            "gpu_launches": launches * a.steps, "clocks": clk.summary(), "device_status": status,
            "gradient_error_vs_absAB": err_reuse,
            "fresh_backward": {"ms_per_step": ms_fresh, "tflops": world * flops / ms_fresh / 1e9,
                               "gradient_error_vs_absAB": err_fresh,
                               "what": "both gradients as independent emulations (own scaling of both operands)"},
        }
        print(json.dumps(line), flush=True)


def tile_label(tile):
    """Words for a batch plan's tile setting."""
    return f"tile 128x{tile}" if tile else "tiles 128x256 or 128x128 per problem"


def run_batched(a, rank, world):
    """512 uneven products as one batch plan (one launch per phase), against the same
    products issued as 512 single calls and against a CUDA graph of the plan."""
    import torch

    import paper_2603_10634_gb300 as ozk
    from paper_2603_10634_gb300 import _lib, workloads

    _lib.load()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = workloads.batch_shapes(512, 64, 2048, seed=0)
    As, Bs = workloads.batch_problems(shapes, a.phi, seed=0, device=dev)
    flops = sum(2.0 * m * n * k for (m, n, k) in shapes)
    stream = torch.cuda.current_stream(dev)
    # moduli count for FP64-level accuracy (sampled on the longest problems) and the faster
    # tile width of the plan (timed), picked by the autotuner
    t0 = time.perf_counter()
    if a.no_autotune:
        N, tile, tune_rep = a.moduli, a.tile if a.tile in (0, 128, 256) else 0, {"moduli": [], "plan_ms": {}}
    else:
        N, tile, tune_rep = ozk.choose_plan(As, Bs, "fp64", mode=a.mode, probes=4)
    reports = tune_rep["moduli"]
    tune_s = time.perf_counter() - t0
    plan = ozk.BatchPlan(As, Bs, num_moduli=N, mode=a.mode, tile_n=tile)

    def timed(fn, steps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s0.record(stream)
        for _ in range(steps):
            fn()
        s1.record(stream)
        torch.cuda.synchronize(dev)
        return s0.elapsed_time(s1) / steps

    for _ in range(a.warmup):
        plan.execute()
    torch.cuda.synchronize(dev)
    launches = ozk.last_launch_count()
    barrier(world)
    with ClockSampler(local) as clk:
        ms = timed(plan.execute, a.steps)
    barrier(world)
    ms = max_over_ranks(ms, world, dev)
    status = plan.status()

    singles = [torch.empty((m, n), dtype=torch.float64, device=dev) for (m, n, k) in shapes]

    def plain():
        for A, B, C in zip(As, Bs, singles):
            ozk.dgemm(A, B, num_moduli=N, out=C, mode=a.mode)

    plain()
    single_launches = ozk.last_launch_count()
    plain_ms = timed(plain, max(1, a.steps // 2))
    same = all(torch.equal(C, D) for C, D in zip(plan.outs, singles))

    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        plan.execute()
        with torch.cuda.graph(graph, stream=side):
            plan.execute()
    stream.wait_stream(side)
    graph_ms = timed(graph.replay, a.steps)
    if rank == 0:
        line = {
            "metric": "batched emulated DGEMM TFLOP/s (sum 2mnk / t), 512 uneven products",
            "value": world * flops / ms / 1e9, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f8e4m3", "emulates": "f64", "data": "synthetic",
            "config": {"workload": f"512 products, m, n, k log-uniform on [64, 2048] (seed 0), phi={a.phi}, "
                                   f"N={N}, {tile_label(tile)} ({'given' if a.no_autotune else 'autotuned'}), {a.mode} mode", "total_flop": flops,
                       "l2": "operands (2.7 GB) larger than L2, no flush"},
            "gpu_launches": launches * a.steps, "clocks": clk.summary(), "device_status": status,
            "plain_calls": {"ms_per_step": plain_ms, "tflops": flops / plain_ms / 1e9, "launches": 512 * single_launches,
                            "bit_identical": bool(same)},
            "cuda_graph": {"ms_per_step": graph_ms, "tflops": flops / graph_ms / 1e9},
            "autotune": {"num_moduli": N, "tile_n": tile, "plan_ms_by_tile": tune_rep["plan_ms"],
                         "target": "within 2x of native FP64 on a sampled block",
                         "probes": [{"problem": i, "shape": shapes[i], "num_moduli": n_i,
                                     "native_err": rep["errors"]["native"], "err": rep["errors"][n_i]}
                                    for (i, n_i, rep) in reports], "seconds": tune_s},
        }
        print(json.dumps(line), flush=True)
    plan.close()


def exact_samples(A, B, samples, seed=7):
    """Sampled entries (i, j) with their exact value and (|A||B|)_ij, as Python numbers."""
    import numpy as np
    import torch

    m, n = A.shape[0], B.shape[1]
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, m, samples)
    cols = rng.integers(0, n, samples)
    Ar = A[torch.as_tensor(rows, device=A.device)].cpu().numpy()
    Bc = B[:, torch.as_tensor(cols, device=A.device)].cpu().numpy()
    out = []
    for t in range(samples):
        out.append((int(rows[t]), int(cols[t]), _exact_dot(Ar[t], Bc[:, t]), _exact_dot(abs(Ar[t]), abs(Bc[:, t]))))
    return out


def sample_error(C, ex):
    """max over the samples of |C_ij - exact| / (|A||B|)_ij."""
    import torch

    idx_r = torch.as_tensor([e[0] for e in ex], device=C.device)
    idx_c = torch.as_tensor([e[1] for e in ex], device=C.device)
    vals = C[idx_r, idx_c].cpu().tolist()
    worst = 0.0
    for v, (_, _, (num, den), (anum, aden)) in zip(vals, ex):
        if v != v:  # NaN
            return float("nan")
        cn, cd = float(v).as_integer_ratio()
        err = abs(num * cd - cn * den) / (den * cd)
        worst = max(worst, err / (anum / aden) if anum else 0.0)
    return worst


def time_calls(fn, steps, warmup, dev):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(steps):
        fn()
    s1.record(stream)
    torch.cuda.synchronize(dev)
    return s0.elapsed_time(s1) / steps


def measure_shape(m, n, k, phi, Ns, mode, steps, warmup, samples, dev, seed=0):
    """TFLOP/s and sampled error of the emulated product for each N in Ns, and of native
    FP64, on one seeded instance; one dict per N plus the native figures."""
    import torch

    import paper_2603_10634_gb300 as ozk
    from paper_2603_10634_gb300 import workloads

    A, B = workloads.problem(m, n, k, phi, seed=seed, device=dev)
    flops = 2.0 * m * n * k
    ex = exact_samples(A, B, samples)
    C = torch.empty((m, n), dtype=torch.float64, device=dev)
    nat_ms = time_calls(lambda: torch.matmul(A, B, out=C), max(1, steps), 1, dev)
    nat_err = sample_error(C, ex)
    rows = []
    for N in Ns:
        ms = time_calls(lambda: ozk.dgemm(A, B, num_moduli=N, out=C, mode=mode), steps, warmup, dev)
        err = sample_error(C, ex)
        planes = 2 * N if N <= 6 else 3 * N - 6
        t_roof = ((3 * N + (0 if mode == "fast" else 1)) * flops / (NOMINAL_FP8_TFLOPS * 1e12) +
                  ((16 + (0 if mode == "fast" else 1) + planes) * (m * k + k * n) + 8 * m * n) / (NOMINAL_HBM_GBS * 1e9))
        rows.append({"m": m, "n": n, "k": k, "phi": phi, "num_moduli": N, "mode": mode, "ms": ms,
                     "tflops": flops / ms / 1e9, "fp8_count_roofline_frac": (flops / ms / 1e9) / (flops / t_roof / 1e12),
                     "max_rel_err_vs_absAB": err, "native_fp64_err": nat_err,
                     "within_2x_native": bool(err <= 2 * max(nat_err, 2.0**-53)),
                     "bound_k_2^-52_holds": bool(err <= k * 2.0**-52), "native_fp64_tflops": flops / nat_ms / 1e9,
                     "device_status": ozk.device_status()})
    del A, B, C
    torch.cuda.empty_cache()
    return rows


def run_sweep(a, rank, world):
    """Error against the exact product and TFLOP/s over sizes x phi x N (one JSON line per
    point), then the smallest N within 2x of native FP64 per (size, phi)."""
    import torch

    from paper_2603_10634_gb300 import _lib

    _lib.load()
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sizes = [int(x) for x in a.sizes.split(",")]
    phis = [float(x) for x in a.phis.split(",")]
    Ns = [int(x) for x in a.moduli_list.split(",")]
    best = {}
    for size in sizes:
        for phi in phis:
            for r in measure_shape(size, size, size, phi, Ns, a.mode, a.steps, a.warmup, a.samples, dev):
                print(json.dumps(r), flush=True)
                key = (size, phi)
                if r["within_2x_native"] and key not in best:
                    best[key] = r
    for (size, phi), r in best.items():
        print(json.dumps({"smallest_N_within_2x_native": r["num_moduli"], "size": size, "phi": phi,
                          "tflops": r["tflops"], "err": r["max_rel_err_vs_absAB"], "native_err": r["native_fp64_err"]}),
              flush=True)


def run_rect(a, rank, world):
    """The long-reduction and tall-skinny shapes at the headline accuracy."""
    import torch

    from paper_2603_10634_gb300 import _lib

    _lib.load()
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    for shape in a.shapes.split(","):
        m, n, k = (int(x) for x in shape.lower().split("x"))
        for r in measure_shape(m, n, k, a.phi, [a.moduli], a.mode, a.steps, a.warmup, a.samples, dev):
            print(json.dumps(r), flush=True)


def apply_settings(a):
    """The library's tuning settings named on the command line (recorded in config)."""
    if a.impl != "ours" or (a.tile is None and a.square_split is None):
        return
    from paper_2603_10634_gb300 import _lib

    lib = _lib.load()
    if a.tile is not None:
        lib.ozk2_set_tile_n(a.tile)
    if a.square_split is not None:
        lib.ozk2_set_square_split(a.square_split)


def main():
    a = parse()
    rank, world = dist_init(a)
    apply_settings(a)
    if a.impl == "reference":
        run_reference(a, rank, world)
    elif a.workload == "autograd":
        run_autograd(a, rank, world)
    elif a.workload == "batched":
        run_batched(a, rank, world)
    elif a.workload == "sweep":
        run_sweep(a, rank, world)
    elif a.workload == "rect":
        run_rect(a, rank, world)
    else:
        run_ours(a, rank, world)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
