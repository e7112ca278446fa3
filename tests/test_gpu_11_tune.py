"""The moduli-count autotuner: its choice meets the requested accuracy on the whole
problem (checked against the exact product on sampled entries), is monotone in the
target, and agrees with the measured sweep (N = 12 is the FP64-level count for the
paper's generator at phi = 1)."""
from fractions import Fraction

import numpy as np
import pytest
import torch

import paper_2603_10634_gb300 as ozk
from oracle import ozaki2 as oz
from paper_2603_10634_gb300 import workloads

pytestmark = pytest.mark.gpu


def _max_err(C, A, B, samples=24, seed=3):
    rng = np.random.default_rng(seed)
    An, Bn, Cn = A.cpu().numpy(), B.cpu().numpy(), C.cpu().numpy()
    worst = 0.0
    for i, j in zip(rng.integers(0, An.shape[0], samples), rng.integers(0, Bn.shape[1], samples)):
        ex = oz.exact_dot(An[i], Bn[:, j])
        ab = float(oz.exact_abs_dot(An[i], Bn[:, j]))
        worst = max(worst, abs(float(ex - Fraction(float(Cn[i, j])))) / ab)
    return worst


def test_fp64_target_at_phi_1(cuda):
    A, B = workloads.problem(2048, 2048, 2048, 1.0, seed=0, device=cuda)
    N, rep = ozk.choose_moduli(A, B, "fp64")
    assert N in (11, 12, 13)
    errs = rep["errors"]
    assert all(errs[a] >= errs[b] for a, b in zip(range(8, 12), range(9, 13)))  # more moduli, less error
    C = ozk.dgemm(A, B, num_moduli=N)
    native = _max_err(torch.matmul(A, B), A, B)
    assert _max_err(C, A, B) <= 2 * max(native, 2.0**-53)


def test_numeric_targets_are_monotone(cuda):
    A, B = workloads.problem(512, 384, 1500, 2.0, seed=5, device=cuda)
    picks = [ozk.choose_moduli(A, B, tau)[0] for tau in (1e-8, 1e-11, 1e-14)]
    assert picks[0] <= picks[1] <= picks[2]
    assert picks[0] < picks[2]
    for tau, N in zip((1e-8, 1e-11, 1e-14), picks):
        assert _max_err(ozk.dgemm(A, B, num_moduli=N), A, B) <= 4 * tau  # sampled block vs whole


def test_batch_choice(cuda):
    shapes = [(100, 90, 80), (300, 200, 1200), (64, 64, 64)]
    As, Bs = workloads.batch_problems(shapes, 1.0, seed=9, device=cuda)
    N, reports = ozk.choose_moduli_batch(As, Bs, "fp64", probes=2)
    assert N == max(r[1] for r in reports)
    assert reports[0][0] == 1  # the longest reduction is probed first
