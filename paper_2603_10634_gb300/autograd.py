"""Differentiable emulated FP64 matrix product.

C = A B runs through the emulated DGEMM; the backward pass needs two more products of
the same kind, dA = dC B^T and dB = A^T dC, and runs them through the same library
call with transposed operands read in place (no copy of A or B).  Each of the three
products is an independent emulation with its own scaling (Sec. III-E), so the
gradients carry the same FP64-level accuracy as the forward result.
"""
from __future__ import annotations

import torch

from . import ozk2


def _operand(x):
    """x itself when the library can read it in place (row-major or the transpose of a
    row-major matrix), else a row-major copy (e.g. the broadcast gradient of a sum)."""
    rows, cols = x.shape
    s0, s1 = x.stride()
    broadcast = (rows > 1 and s0 == 0) or (cols > 1 and s1 == 0)
    if not broadcast and (cols <= 1 or s1 == 1 or rows <= 1 or s0 == 1):
        return x
    return x.contiguous()


class OzakiMatmul(torch.autograd.Function):
    """C = A @ B for float64 CUDA matrices; forward and both gradients emulated."""

    @staticmethod
    def forward(ctx, A, B, num_moduli=12, mode="accurate"):
        ctx.num_moduli = num_moduli
        ctx.mode = mode
        ctx.save_for_backward(A, B)
        return ozk2.dgemm(_operand(A), _operand(B), num_moduli=num_moduli, mode=mode)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = _operand(dC)
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = ozk2.dgemm(dC, _operand(B).T, num_moduli=ctx.num_moduli, mode=ctx.mode)
        if ctx.needs_input_grad[1]:
            dB = ozk2.dgemm(_operand(A).T, dC, num_moduli=ctx.num_moduli, mode=ctx.mode)
        return dA, dB, None, None


def matmul(A, B, num_moduli=12, mode="accurate"):
    """Differentiable C = A @ B in emulated FP64 (see ``OzakiMatmul``)."""
    return OzakiMatmul.apply(A, B, num_moduli, mode)
