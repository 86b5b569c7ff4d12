"""The learned warm start gains CGLS iterations: a short training of the U-Net on the GPU (its
tensor-core convolutions, forward and both gradients) at a small size, then CGLS to the 1e-3
normal-equation residual from the network's start and from zero on held-out phantoms.

Problem: 64^3 voxels of 1 mm (the 64 mm phantoms of the 128^3 CGLS workload at half the
resolution), 90 views over 360 deg, SID 750 / SDD 1200 mm, 128 x 96 detector at 1.6 mm, Poisson
noise at 1e5 photons, relaxed operator. Network: the U-Net with three levels (16/32/64 channels;
a 64^3 volume has no fourth level the convolution kernels take), trained with the recipe of the
full-size run (mean squared error plus 16 x that of the finite differences, learning rate 1e-3
after 100 warm-up steps, cosine decay).
"""
import pytest
import torch

from paper_2110_09841_b300 import inputs, warmstart
from paper_2110_09841_b300.unet import UNet3D

pytestmark = pytest.mark.gpu


def geometry():
    return inputs.make_geometry((64, 64, 64), (1.0, 1.0, 1.0), (128, 96), (1.6, 1.6), 90, 750.0, 1200.0, 360.0)


def test_short_training_saves_cgls_iterations():
    g = geometry()
    prob = warmstart.Problem(g, "relaxed")
    xs, ts = warmstart.generate(prob, range(30000, 30400))
    model = UNet3D(levels=3).cuda()
    hist = warmstart.train(model, xs, ts, epochs=4, lr=1e-3, warmup=100, edge_weight=16.0)
    assert hist[-1] < hist[0]
    del xs, ts
    rows = warmstart.evaluate(model, prob, range(31000, 31006))
    s = warmstart.summarise(rows)
    print(s)
    assert s["all_converged"]
    # the trained start is closer to the phantom than the normalised backprojection it came from
    assert s["rel_err_x0"] < 0.5
    saved = s["iters_zero"] - s["iters_warm"]
    assert saved >= 3.0, s
    assert all(r["iters_warm"] < r["iters_zero"] for r in rows)
