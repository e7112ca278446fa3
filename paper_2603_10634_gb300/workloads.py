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
