"""FP64 reference of the 3x3x3 convolution used by the learned CGLS warm start -- test
infrastructure only (tests and the smoke check use it; the product path never does).

The convolution is its definition (stride 1, zero padding 1, no dilation):
    y[n, co, z, y, x] = b[co] + sum_{ci, dz, dy, dx} w[co, ci, dz, dy, dx] x[n, ci, z+dz-1, y+dy-1, x+dx-1]
evaluated with torch's CPU conv3d in float64 (a library primitive serving as one step), and
its gradients with torch's CPU autograd in float64. Layouts here are channels-first
(torch's NCDHW, weights [cout, cin, 3, 3, 3]); the tests convert.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def conv3d(x, w, b=None):
    """x [n, cin, d, h, w], w [cout, cin, 3, 3, 3], b [cout] -> float64 [n, cout, d, h, w]."""
    x = torch.as_tensor(x, dtype=torch.float64)
    w = torch.as_tensor(w, dtype=torch.float64)
    b = None if b is None else torch.as_tensor(b, dtype=torch.float64)
    return F.conv3d(x, w, b, padding=1)


def conv3d_grads(x, w, gy):
    """Gradients of sum(gy * conv3d(x, w)) with respect to x and w (float64)."""
    x = torch.as_tensor(x, dtype=torch.float64).clone().requires_grad_(True)
    w = torch.as_tensor(w, dtype=torch.float64).clone().requires_grad_(True)
    y = F.conv3d(x, w, None, padding=1)
    (y * torch.as_tensor(gy, dtype=torch.float64)).sum().backward()
    return x.grad, w.grad


def conv3d_loops(x, w, b=None):
    """The same convolution as explicit loops over taps (tiny inputs only)."""
    x = torch.as_tensor(x, dtype=torch.float64)
    w = torch.as_tensor(w, dtype=torch.float64)
    n, ci, d, h, wd = x.shape
    co = w.shape[0]
    xp = torch.zeros((n, ci, d + 2, h + 2, wd + 2), dtype=torch.float64)
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    y = torch.zeros((n, co, d, h, wd), dtype=torch.float64)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + d, dy:dy + h, dx:dx + wd]          # x at (z+dz-1, y+dy-1, x+dx-1)
                y += torch.einsum("oc,ncdhw->nodhw", w[:, :, dz, dy, dx], patch)
    if b is not None:
        y += torch.as_tensor(b, dtype=torch.float64)[None, :, None, None, None]
    return y
