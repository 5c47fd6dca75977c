"""torch.autograd support for the block-sparse product.

``matmul(A, B, a_vals, b_vals)`` returns C's leaf values (a tensor
[nnzb_C, b, b] in C's Morton order) and records a backward that calls
cht_multiply_backward:
    dA = (dC B^T) on A's pattern,  dB = (A^T dC) on B's pattern.
``a_vals`` / ``b_vals`` must be the value views of A and B
(``A.values()``), e.g. made leaves with ``requires_grad_()``; their
gradients come back in the same layout.
"""

from __future__ import annotations

import torch

from . import (Matrix, Plan, cht_multiply, cht_multiply_backward,
               cht_symbolic_multiply)


class _BlockSparseMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_vals, b_vals, A, B, plan, recompute_pairs):
        C, _ = cht_multiply(plan, A, B)
        ctx.A, ctx.B, ctx.C = A, B, C
        ctx.plan = None if recompute_pairs else plan
        ctx.recompute = recompute_pairs
        return C.values()

    @staticmethod
    def backward(ctx, grad_c):
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_a or need_b):
            return None, None, None, None, None, None
        dC = ctx.C.like()
        dC.values().copy_(grad_c)
        dA, dB = cht_multiply_backward(ctx.plan, ctx.A, ctx.B, dC,
                                       recompute_pairs=ctx.recompute,
                                       want_dA=need_a, want_dB=need_b)
        return (dA.values() if dA is not None else None,
                dB.values() if dB is not None else None, None, None, None, None)


def matmul(A: Matrix, B: Matrix, a_vals: torch.Tensor | None = None,
           b_vals: torch.Tensor | None = None, plan: Plan | None = None,
           recompute_pairs: bool = False):
    """Differentiable C = A*B; returns (C values, plan)."""
    if plan is None:
        plan = cht_symbolic_multiply(A, B)
    a_vals = A.values() if a_vals is None else a_vals
    b_vals = B.values() if b_vals is None else b_vals
    c = _BlockSparseMatmul.apply(a_vals, b_vals, A, B, plan, recompute_pairs)
    return c, plan
