"""Differentiable wrappers of the projector: the gradient of a forward projection is the
adjoint computed by kct_backproject, and vice versa (A^T's adjoint is A).

    from paper_2110_09841_b300 import Projector, autograd
    A = Projector(geom)
    b = autograd.project(x, A)            # x [nz, ny, nx] or [B, nz, ny, nx]
    loss = 0.5 * ((b - y) ** 2).sum()
    loss.backward()                      # x.grad = A^T (A x - y)

Argument marshalling only: both directions run in libkct.
"""
from __future__ import annotations

import torch


def _fwd(op, x):
    return op.project_batch(x) if x.dim() == 4 else op.project(x)


def _bwd(op, y):
    return op.backproject_batch(y) if y.dim() == 4 else op.backproject(y)


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return _fwd(op, x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return _bwd(ctx.op, g.contiguous()), None


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, op):
        ctx.op = op
        return _bwd(op, y.contiguous())

    @staticmethod
    def backward(ctx, g):
        return _fwd(ctx.op, g.contiguous()), None


def project(x: torch.Tensor, op) -> torch.Tensor:
    """A x with autograd support (backward = A^T)."""
    return _Project.apply(x, op)


def backproject(y: torch.Tensor, op) -> torch.Tensor:
    """A^T y with autograd support (backward = A)."""
    return _Backproject.apply(y, op)
