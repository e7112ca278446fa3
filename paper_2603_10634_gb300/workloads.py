"""Seeded synthetic inputs shaped like the paper's workloads (Sec. V-A).

The paper's test matrices are a_ij = (rand - 0.5) exp(phi randn) with rand uniform and
randn standard normal, or plain standard normal entries.  This module only draws
random numbers; it holds none of the method's arithmetic, and both the CUDA path and
the CPU oracle take its outputs as inputs.
"""
from __future__ import annotations

import torch


def phi_matrix(rows, cols, phi, seed, device="cpu"):
    """(U - 0.5) * exp(phi * N(0, 1)), float64, from one seeded torch generator.

    U and N are drawn as two independent fields in that order.  Generating on the
    CPU and on a GPU gives different (equally distributed) matrices."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    u = torch.rand((rows, cols), generator=g, dtype=torch.float64, device=device)
    z = torch.randn((rows, cols), generator=g, dtype=torch.float64, device=device)
    return (u - 0.5) * torch.exp(phi * z)


def normal_matrix(rows, cols, seed, device="cpu"):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn((rows, cols), generator=g, dtype=torch.float64, device=device)


def problem(m, n, k, phi, seed=0, device="cpu"):
    """A (m x k) with seed `seed` and B (k x n) with seed `seed + 1`."""
    return phi_matrix(m, k, phi, seed, device), phi_matrix(k, n, phi, seed + 1, device)


def batch_shapes(count=512, lo=64, hi=2048, seed=0):
    """`count` (m, n, k) triples, each dimension log-uniform on [lo, hi] (rounded to an
    integer), from one seeded torch generator: the uneven batch of many small products
    the method's small-size behaviour is about."""
    import math

    g = torch.Generator()
    g.manual_seed(int(seed))
    u = torch.rand((count, 3), generator=g, dtype=torch.float64)
    dims = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))).round().to(torch.int64)
    return [tuple(int(x) for x in row) for row in dims.clamp(lo, hi)]


def batch_problems(shapes, phi, seed=0, device="cpu"):
    """Operands of a batch: problem i uses seeds seed + 2 i (A) and seed + 2 i + 1 (B)."""
    As, Bs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = problem(m, n, k, phi, seed=seed + 2 * i, device=device)
        As.append(A)
        Bs.append(B)
    return As, Bs
