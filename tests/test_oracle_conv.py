"""Pins of the oracle convolution against its definition and closed forms."""
import numpy as np
import torch

from oracle import conv


def test_library_conv_equals_explicit_loops():
    g = torch.Generator().manual_seed(3)
    x = torch.randn((2, 3, 4, 5, 6), generator=g, dtype=torch.float64)
    w = torch.randn((4, 3, 3, 3, 3), generator=g, dtype=torch.float64)
    b = torch.randn(4, generator=g, dtype=torch.float64)
    torch.testing.assert_close(conv.conv3d(x, w, b), conv.conv3d_loops(x, w, b), rtol=1e-12, atol=1e-12)


def test_delta_kernel_is_a_shift_with_zero_fill():
    x = torch.arange(4 * 4 * 4, dtype=torch.float64).reshape(1, 1, 4, 4, 4)
    w = torch.zeros((1, 1, 3, 3, 3), dtype=torch.float64)
    w[0, 0, 2, 1, 0] = 1.0                     # reads x[z + 1, y, x - 1]
    y = conv.conv3d(x, w)
    ref = torch.zeros_like(x)
    ref[0, 0, :3, :, 1:] = x[0, 0, 1:, :, :3]
    torch.testing.assert_close(y, ref, rtol=0, atol=0)


def test_ones_count_neighbours_inside_the_box():
    x = torch.ones((1, 1, 5, 5, 5), dtype=torch.float64)
    y = conv.conv3d(x, torch.ones((1, 1, 3, 3, 3), dtype=torch.float64))
    assert y[0, 0, 2, 2, 2] == 27 and y[0, 0, 0, 0, 0] == 8 and y[0, 0, 0, 2, 2] == 18


def test_gradients_match_finite_differences():
    g = torch.Generator().manual_seed(5)
    x = torch.randn((1, 2, 3, 4, 4), generator=g, dtype=torch.float64)
    w = torch.randn((3, 2, 3, 3, 3), generator=g, dtype=torch.float64)
    gy = torch.randn((1, 3, 3, 4, 4), generator=g, dtype=torch.float64)
    gx, gw = conv.conv3d_grads(x, w, gy)
    h = 1e-6
    for (t, gt) in ((x, gx), (w, gw)):
        for idx in [(0, 1, 1, 2, 3), (0, 0, 0, 0, 0)] if t is x else [(2, 1, 0, 2, 1), (0, 0, 1, 1, 1)]:
            tp, tm = t.clone(), t.clone()
            tp[idx] += h
            tm[idx] -= h
            args_p = (tp, w) if t is x else (x, tp)
            args_m = (tm, w) if t is x else (x, tm)
            fd = float(((conv.conv3d_loops(*args_p) - conv.conv3d_loops(*args_m)) * gy).sum()) / (2 * h)
            assert abs(fd - float(gt[idx])) <= 1e-7 * max(1.0, abs(fd))
