"""Host-side logic of bench.py on CPU: the multi-rank path (barrier + max over ranks
with gloo, world size 2), the clock-sample parser, the exact-error helper and the
reference arm's JSON line."""
import json
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.max_over_ranks(10.0 + rank, world)
    out.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}


def test_clock_summary_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.lines = ["0, 1800, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active",
               "0, 1500, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1700, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 1700 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


def test_exact_dot_helper():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(50) * 2.0 ** rng.integers(-30, 30, 50)
    b = rng.standard_normal(50)
    num, den = bench._exact_dot(a, b)
    want = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    assert Fraction(num, den) == want


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--size", "16384"], capture_output=True, text=True, timeout=600,
                       env={**os.environ, "OZK2_REFERENCE_SAMPLE": "128"})
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "TFLOP/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
