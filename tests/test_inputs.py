"""Synthetic inputs: geometry conventions and the paper's printed problem sizes."""
import json
import math
import os

import numpy as np
import pytest

from paper_2110_09841_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_benchmarks.json")


@pytest.mark.parametrize("name", ["long2010", "pfeiffer2021"])
def test_paper_benchmark_sizes(name):
    """The benchmark workloads have the sizes printed in Sec. IV-A."""
    gold = json.load(open(GOLDEN))[name]
    g = inputs.workload_geometry(name)
    assert [g.nx, g.ny, g.nz] == gold["volume"]
    assert [g.nu, g.nv] == gold["detector"]
    assert g.nviews == gold["views"]
    assert g.nx * g.ny * g.nz / 1e6 == pytest.approx(gold["x_elements_printed_millions"], abs=0.1)
    assert g.nu * g.nv * g.nviews / 1e6 == pytest.approx(gold["b_elements_printed_millions"], abs=0.1)


def test_circular_matrices_conventions():
    """Source on the circle, isocentre at the principal point, chi_2 opposite to x_3,
    column projection independent of x_3 (Sec. III-A)."""
    P = inputs.circular_pmats(8, 750.0, 1200.0, 64, 48, 0.8, 0.8)
    for k in range(8):
        M, p4 = P[k, :, :3], P[k, :, 3]
        s = -np.linalg.solve(M, p4)
        phi = 2 * math.pi * k / 8
        np.testing.assert_allclose(s, [750 * math.cos(phi), 750 * math.sin(phi), 0.0], atol=1e-9)
        h = P[k] @ np.array([0, 0, 0, 1.0])
        np.testing.assert_allclose(h[:2] / h[2], [31.5, 23.5], atol=1e-12)
        up = P[k] @ np.array([0, 0, 1.0, 1.0])
        assert up[1] / up[2] < 23.5                      # +x_3 goes to smaller v
        assert M[0, 2] == 0.0 and M[2, 2] == 0.0          # u independent of x_3
        # magnification at the isocentre: 1 mm along u -> sdd / sid / pitch pixels
        side = P[k] @ np.array([-math.sin(phi), math.cos(phi), 0.0, 1.0])
        assert side[0] / side[2] - 31.5 == pytest.approx(1200 / 750 / 0.8, rel=1e-12)


def test_phantom_is_seeded_and_additive():
    a = inputs.workload_phantom("cvp32").numpy()
    b = inputs.workload_phantom("cvp32").numpy()
    assert np.array_equal(a, b)
    assert a.shape == (32, 32, 32) and a.dtype == np.float32
    assert a.min() == 0.0 and 0.005 <= a.max() <= 6 * 0.02
    ells = inputs.random_ellipsoids(1001, 6, 32.0, (3.0, 12.0), (0.005, 0.02))
    g = inputs.workload_geometry("cvp32")
    one = [inputs.voxelize(g, [e]).numpy() for e in ells]
    np.testing.assert_allclose(sum(one), a, atol=1e-7)


def test_poisson_log_data_statistics():
    """b = -ln(max(N, 1) / I0), N ~ Poisson(I0 exp(-clean)): mean close to the clean line
    integral, variance close to exp(clean) / I0 (delta method), seeded."""
    import torch

    clean = torch.full((200000,), 0.8)
    b = inputs.poisson_log_data(clean, 1e5, 11)
    assert torch.equal(b, inputs.poisson_log_data(clean, 1e5, 11))
    assert abs(float(b.mean()) - 0.8) < 1e-4
    var = float(b.double().var())
    assert abs(var / (math.exp(0.8) / 1e5) - 1.0) < 0.02
    # no photons counted: clamped to one count
    assert float(inputs.poisson_log_data(torch.full((4,), 60.0), 1e5, 1).max()) == pytest.approx(math.log(1e5), rel=1e-6)


def test_perfusion_frames_follow_bolus_curves():
    """Frames differ only inside the vessel ellipsoids; the static background is shared."""
    g = inputs.make_geometry((24, 24, 20), (1.0, 1.0, 1.0), (48, 40), (0.8, 0.8), 4, 750.0, 1200.0, 360.0)
    f = inputs.perfusion_frames(g, 31, frames=6)
    assert f.shape == (6,) + g.vol_shape
    d = (f - f[0]).abs().amax(dim=0)
    assert 0 < int((d > 0).sum()) < d.numel() // 2
    assert bool((f >= 0).all())


def test_cgls_workload_shapes():
    g = inputs.workload_geometry("cgls128")
    assert g.vol_shape == (128, 128, 128) and g.proj_shape == (180, 192, 256)
