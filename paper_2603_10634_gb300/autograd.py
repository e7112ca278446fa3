"""Differentiable emulated FP64 matrix product.

C = A B runs through the emulated DGEMM.  The backward pass needs two more products,
dA = dC B^T and dB = A^T dC.  By default (``reuse=True``) they run through
ozk2_dgemm_backward, which reuses the forward call's scaling exponents and digit planes
of A' = trunc(diag(2^e) A) and B' = trunc(B diag(2^f)): the forward runs in a workspace
kept in the autograd context, only dC is scaled and converted (once, for both
gradients), and dC's exponents take the whole budget of P that A' and B' leave.  With
``reuse=False``, or where reuse does not apply (fast mode, operands that are transposed
views), each gradient is an independent emulation with its own scaling (Sec. III-E) of
operands read in place.
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


def _row_major(x):
    rows, cols = x.shape
    s0, s1 = x.stride()
    return (cols <= 1 or s1 == 1) and (rows <= 1 or s0 >= max(1, cols))


class OzakiMatmul(torch.autograd.Function):
    """C = A @ B for float64 CUDA matrices; forward and both gradients emulated."""

    @staticmethod
    def forward(ctx, A, B, num_moduli=12, mode="accurate", reuse=True):
        ctx.num_moduli = num_moduli
        ctx.mode = mode
        ctx.reuse = bool(reuse) and mode == "accurate" and _row_major(A) and _row_major(B)
        ctx.save_for_backward(A, B)
        if ctx.reuse:
            m, k = A.shape
            n = B.shape[1]
            ws = torch.empty(max(1, ozk2.workspace_size(m, n, k, num_moduli)), dtype=torch.uint8, device=A.device)
            ctx.forward_workspace = ws  # the forward's exponents and digit planes, read by backward
            return ozk2.dgemm(A, B, num_moduli=num_moduli, workspace=ws)
        return ozk2.dgemm(_operand(A), _operand(B), num_moduli=num_moduli, mode=mode)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dA = dB = None
        if ctx.reuse:
            dC = dC.contiguous()
            dA, dB = ozk2.dgemm_backward(A, B, dC, ctx.forward_workspace, ctx.num_moduli,
                                         need_dA=ctx.needs_input_grad[0], need_dB=ctx.needs_input_grad[1])
            return dA, dB, None, None, None
        dC = _operand(dC)
        if ctx.needs_input_grad[0]:
            dA = ozk2.dgemm(dC, _operand(B).T, num_moduli=ctx.num_moduli, mode=ctx.mode)
        if ctx.needs_input_grad[1]:
            dB = ozk2.dgemm(_operand(A).T, dC, num_moduli=ctx.num_moduli, mode=ctx.mode)
        return dA, dB, None, None, None


def matmul(A, B, num_moduli=12, mode="accurate", reuse=True):
    """Differentiable C = A @ B in emulated FP64 (see ``OzakiMatmul``)."""
    return OzakiMatmul.apply(A, B, num_moduli, mode, reuse)
