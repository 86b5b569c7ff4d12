"""GPU parity: the CUDA projector (through the C ABI) against the FP64 CPU oracle.

Tolerance (float32 arithmetic with float atomics): per view, over pixels whose oracle
value is at least 1e-3 of that view's maximum, max |gpu - oracle| / |oracle| <= 1e-4, and
over all pixels max |gpu - oracle| <= 1e-4 * view maximum; the same rule over voxels for
the adjoint. Adjoint identity <A x, y> = <x, A^T y> with float64 dot products to 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09841_b300 import inputs
from paper_2110_09841_b300.kct import Projector

pytestmark = pytest.mark.gpu

VARIANTS = [("exact", 0), ("relaxed", 1)]
SCALINGS = [("cos", 0), ("exact", 1)]
TOL = 1e-4


def assert_close_per_view(g, o, tol=TOL, what="projection"):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    assert g.shape == o.shape
    worst_rel = worst_abs = 0.0
    for view in range(o.shape[0]):
        mx = np.abs(o[view]).max()
        if mx == 0.0:
            assert np.abs(g[view]).max() <= 1e-30, f"{what} view {view} should be empty"
            continue
        d = np.abs(g[view] - o[view])
        big = np.abs(o[view]) >= 1e-3 * mx
        worst_rel = max(worst_rel, float((d[big] / np.abs(o[view][big])).max()))
        worst_abs = max(worst_abs, float(d.max() / mx))
    assert worst_rel <= tol, f"{what}: max relative error {worst_rel:.3e}"
    assert worst_abs <= tol, f"{what}: max error / view max {worst_abs:.3e}"
    return worst_rel, worst_abs


def assert_close_volume(g, o, tol=TOL):
    return assert_close_per_view(np.asarray(g)[None], np.asarray(o)[None], tol, "backprojection")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def cvp32():
    g = inputs.workload_geometry("cvp32")
    x = inputs.workload_phantom("cvp32").numpy()
    y = inputs.uniform_projections(g.proj_shape, 2024).numpy()
    return g, x, y


@pytest.mark.parametrize("vname,variant", VARIANTS)
@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_project_cvp32(cvp32, vname, variant, sname, scaling):
    g, x, y = cvp32
    ref = oracle.project(g, x.astype(np.float64), variant, scaling)
    A = Projector(g, vname, sname)
    b = A.project(dev(x))
    torch.cuda.synchronize()
    assert A.device_error() == 0
    assert_close_per_view(b.cpu().numpy(), ref)


@pytest.mark.parametrize("vname,variant", VARIANTS)
@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_backproject_cvp32(cvp32, vname, variant, sname, scaling):
    g, x, y = cvp32
    ref = oracle.backproject(g, y.astype(np.float64), variant, scaling)
    A = Projector(g, vname, sname)
    xb = A.backproject(dev(y))
    torch.cuda.synchronize()
    assert A.device_error() == 0
    assert_close_volume(xb.cpu().numpy(), ref)


@pytest.mark.parametrize("vname", ["exact", "relaxed"])
@pytest.mark.parametrize("name", ["cvp32", "ragged"])
def test_adjoint_gap(vname, name):
    if name == "cvp32":
        g = inputs.workload_geometry("cvp32")
    else:
        g = inputs.make_geometry((13, 7, 11), (0.9, 1.3, 0.7), (37, 29), (0.7, 0.9), 5, 300.0, 500.0, 170.0)
    x = inputs.uniform_volume(g.vol_shape, 11, device="cuda")
    y = inputs.uniform_projections(g.proj_shape, 12, device="cuda")
    A = Projector(g, vname, "cos")
    Ax = A.project(x).double()
    Aty = A.backproject(y).double()
    lhs = float((Ax * y.double()).sum())
    rhs = float((x.double() * Aty).sum())
    gap = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    assert gap <= 1e-5, gap


@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_ragged_and_truncated(vname, variant):
    """Odd sizes, anisotropic voxels, a detector that truncates the volume, half-integer
    principal point, views at 0 and 90 degrees (boundaries through voxel faces)."""
    g = inputs.make_geometry((13, 7, 11), (0.9, 1.3, 0.7), (17, 9), (0.7, 0.9), 4, 300.0, 500.0, 360.0)
    x = np.random.default_rng(3).random(g.vol_shape)
    y = np.random.default_rng(4).random(g.proj_shape)
    A = Projector(g, vname, "cos")
    b = A.project(dev(x)).cpu().numpy()
    assert_close_per_view(b, oracle.project(g, x, variant, 0))
    xb = A.backproject(dev(y)).cpu().numpy()
    assert_close_volume(xb, oracle.backproject(g, y, variant, 0))


@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_single_voxel_and_accumulate(vname, variant):
    """One 2 mm voxel spanning ~8 x 6 pixels (more columns than one pass handles): every
    pixel value is a single pair, including thin slivers at the footprint's edges."""
    g = inputs.make_geometry((1, 1, 1), (2.0, 2.0, 2.0), (14, 12), (0.5, 0.5), 3, 400.0, 600.0, 360.0)
    x = np.ones(g.vol_shape)
    A = Projector(g, vname, "cos")
    ref = oracle.project(g, x, variant, 0)
    b = A.project(dev(x)).cpu().numpy()
    assert_close_per_view(b, ref)
    out = dev(np.full(g.proj_shape, 0.25))
    A.project(dev(x), out=out, accumulate=True)
    assert_close_per_view(out.cpu().numpy() - 0.25, ref, tol=1e-4)
    xb = dev(np.full(g.vol_shape, 2.0))
    y = np.ones(g.proj_shape)
    A.backproject(dev(y), out=xb, accumulate=True)
    refx = oracle.backproject(g, y, variant, 0) + 2.0
    assert abs(float(xb.cpu()[0, 0, 0]) - refx[0, 0, 0]) <= 1e-5 * refx[0, 0, 0]


@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_rows_along_plus_x3(vname, variant):
    """Detector row index growing with x_3 (the v axis flipped: v' = nv - 1 - v), the other
    orientation of the paper's arrangement; forward and adjoint against the oracle."""
    g = inputs.make_geometry((13, 7, 11), (0.9, 1.3, 0.7), (17, 15), (0.7, 0.9), 4, 300.0, 500.0, 360.0)
    P = g.pmats.copy()
    P[:, 1, :] = (g.nv - 1) * P[:, 2, :] - P[:, 1, :]
    g = inputs.Geometry(**{**g.__dict__, "pmats": P})
    x = np.random.default_rng(13).random(g.vol_shape)
    y = np.random.default_rng(14).random(g.proj_shape)
    for sname, scaling in SCALINGS:
        A = Projector(g, vname, sname)
        b = A.project(dev(x)).cpu().numpy()
        assert_close_per_view(b, oracle.project(g, x, variant, scaling))
        xb = A.backproject(dev(y)).cpu().numpy()
        assert_close_volume(xb, oracle.backproject(g, y, variant, scaling))
        assert A.device_error() == 0


@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_elevated_source_thin_slivers(vname, variant):
    """Source 100 mm below the volume centre, so that row boundaries meet the voxels about
    100 mm above the source plane: a boundary's height over a voxel face is then the small
    difference of two ~100 mm coordinates. The detector cuts the footprints into thin slivers
    at its edge rows; forward and adjoint against the oracle element by element."""
    P = inputs.circular_pmats(4, 300.0, 500.0, 17, 16, 0.7, 0.9, 360.0, 10.0, cv=197.0)
    P[:, :, 3] -= P[:, :, :3] @ np.array([0.0, 0.0, -100.0])
    g = inputs.Geometry(13, 7, 11, 0.9, 1.3, 0.7, 17, 16, 0.7, 0.9, P)
    x = np.random.default_rng(21).random(g.vol_shape)
    y = np.random.default_rng(22).random(g.proj_shape)
    A = Projector(g, vname, "cos")
    b = A.project(dev(x)).cpu().numpy()
    ref = oracle.project(g, x, variant, 0)
    assert all(np.abs(ref[v]).max() > 0 for v in range(g.nviews))
    assert_close_per_view(b, ref)
    xb = A.backproject(dev(y)).cpu().numpy()
    assert_close_volume(xb, oracle.backproject(g, y, variant, 0))
    assert A.device_error() == 0


@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_largest_footprints(vname, variant):
    """Voxels near the largest footprint the kernels take: 1 mm voxels at magnification 1.5
    on 0.15 x 0.065 mm pixels span 24-28 detector rows (the per-voxel bound is 31) and 12-16
    columns (two or three column-cut passes); a lane walks that many rows per column cut, the
    faces of a 64-voxel run are crossed by 150-210 row planes (several evaluation rounds of a
    warp), 66 voxels along x_3 fill both runs of a brick, and every brick overflows the shared
    tile. Forward, adjoint and the adjoint identity against the oracle, element by element."""
    g = inputs.make_geometry((3, 3, 66), (1.0, 1.0, 1.0), (64, 1600), (0.15, 0.065), 2, 300.0, 450.0, 75.0)
    x = np.random.default_rng(41).random(g.vol_shape)
    y = np.random.default_rng(42).random(g.proj_shape)
    A = Projector(g, vname, "cos")
    b = A.project(dev(x)).cpu().numpy()
    assert_close_per_view(b, oracle.project(g, x, variant, 0))
    xb = A.backproject(dev(y)).cpu().numpy()
    assert_close_volume(xb, oracle.backproject(g, y, variant, 0))
    assert A.device_error() == 0
    lhs = float((b.astype(np.float64) * y).sum())
    rhs = float((x * xb.astype(np.float64)).sum())
    assert abs(lhs - rhs) / max(abs(lhs), abs(rhs)) <= 1e-5


def test_volume_off_detector_gives_zeros():
    # a detector far off to the side: no voxel projects onto it
    P = inputs.circular_pmats(2, 300.0, 500.0, 16, 16, 0.5, 0.5, cu=-400.0)
    g = inputs.Geometry(8, 8, 8, 1.0, 1.0, 1.0, 16, 16, 0.5, 0.5, P)
    A = Projector(g, "exact", "cos")
    b = A.project(dev(np.ones(g.vol_shape)))
    assert float(b.abs().max()) == 0.0
    xb = A.backproject(dev(np.ones(g.proj_shape)))
    assert float(xb.abs().max()) == 0.0


@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_pixel_factors(sname, scaling):
    g = inputs.workload_geometry("cvp256").subset_views([0, 77, 200])
    A = Projector(g, "exact", sname)
    F = A.pixel_factors().cpu().numpy()
    rng = np.random.default_rng(5)
    for view in range(3):
        for u, v in list(zip(rng.integers(0, g.nu, 20), rng.integers(0, g.nv, 20))) + [(0, 0), (g.nu - 1, g.nv - 1)]:
            ref = oracle.pixel_factor(g.pmats[view], u, v, scaling)
            assert F[view, v, u] == pytest.approx(ref, rel=2e-6)


def sampled_pixels(g, rng, views, per_view):
    pix = []
    for view in views:
        for _ in range(per_view):
            pix.append((view, int(rng.integers(0, g.nv)), int(rng.integers(0, g.nu))))
    return np.array(pix, dtype=np.int32)


@pytest.mark.parametrize("name", ["cvp256", "cvp512"])
@pytest.mark.parametrize("vname,variant", VARIANTS)
def test_sampled_parity_full_size(name, vname, variant):
    """Full-size workload, projected in full on the GPU; the oracle computes sampled
    pixels one by one."""
    g = inputs.workload_geometry(name)
    x = inputs.workload_phantom(name, device="cuda")
    A = Projector(g, vname, "cos")
    b = A.project(x)
    torch.cuda.synchronize()
    assert A.device_error() == 0
    rng = np.random.default_rng(77)
    views = [0, g.nviews // 3, g.nviews - 1]
    # pixels where the phantom projects (nonzero), plus random ones
    bc = b.cpu().numpy()
    pix = []
    for view in views:
        nz = np.argwhere(bc[view] > 0.05 * bc[view].max())
        sel = nz[rng.choice(len(nz), 12, replace=False)]
        pix += [(view, int(r), int(c)) for r, c in sel]
    pix = np.array(pix + [tuple(p) for p in sampled_pixels(g, rng, views, 4)], dtype=np.int32)
    ref = oracle.project_pixels(g, x.cpu().numpy(), pix, variant, 0)
    got = bc[pix[:, 0], pix[:, 1], pix[:, 2]]
    vmax = np.array([bc[v].max() for v in pix[:, 0]])
    err = np.abs(got - ref)
    assert np.all(err <= TOL * vmax), float((err / vmax).max())
    big = ref >= 1e-3 * vmax
    assert np.all(err[big] <= TOL * ref[big]), float((err[big] / ref[big]).max())
