"""FP64 CPU reference of the warm-start U-Net's forward pass -- test infrastructure only.

The same architecture as the GPU network (two 3x3x3 convolutions with bias and ReLU per
level; 2x2x2 max pooling; nearest x2 upsampling, a halving convolution, concatenation with
the skip, two convolutions; a final convolution whose channel 0 corrects the input), written
with torch CPU float64 operations (conv3d as a library primitive) in channels-first layout.
Gradients come from torch's CPU autograd on this graph.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def _w(p, name):
    w = p[name + "_w"]                                   # [cout, 27, cin] -> [cout, cin, 3, 3, 3]
    co, _, ci = w.shape
    return w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3), p[name + "_b"]


def _c(p, name, x, relu=True):
    w, b = _w(p, name)
    y = F.conv3d(x, w, b, padding=1)
    return torch.relu(y) if relu else y


def forward(p: dict, inp: torch.Tensor, levels: int = 4, base: int = 16, scale: float = 1.0) -> torch.Tensor:
    """p: float64 parameters by name ([cout, 27, cin] weights, [cout] biases);
    inp: float64 [n, d, h, w] -> float64 [n, d, h, w]. The network sees inp * scale and its
    correction is divided by scale."""
    n, d, h, w = inp.shape
    x = torch.zeros((n, base, d, h, w), dtype=torch.float64)
    x[:, 0] = inp * scale
    skips = []
    for i in range(levels):
        if i > 0:
            x = F.max_pool3d(x, 2)
        x = _c(p, f"enc{i}a", x)
        x = _c(p, f"enc{i}b", x)
        skips.append(x)
    for i in range(levels - 2, -1, -1):
        x = F.interpolate(x, scale_factor=2, mode="nearest")
        x = _c(p, f"up{i}", x)
        x = torch.cat([x, skips[i]], dim=1)
        x = _c(p, f"dec{i}a", x)
        x = _c(p, f"dec{i}b", x)
    y = _c(p, "head", x, relu=False)
    return inp + y[:, 0] / scale
