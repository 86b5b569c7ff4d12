"""GPU parity at the full workload sizes, and the kernels' fallback paths.

The CUDA projector runs over the whole volume and detector stack, in the launch
configuration the benchmark times; the FP64 oracle computes sampled voxels (adjoint) or
pixels (forward) one by one. Tolerance rule (the same as the small-size parity tests):
max |gpu - oracle| <= 1e-4 * max (the view's maximum for projections, the volume's maximum
for the adjoint), and max |gpu - oracle| / |oracle| <= 1e-4 where the oracle value is at
least 1e-3 of that maximum. Adjoint identity (Sec. III-D, Eq. fundament) with FP64 dots:
|<A x, y> - <x, A^T y>| / max(|<A x, y>|, |<x, A^T y>|) <= 1e-5.

The sampled voxels include every brick boundary along x_3 of both adjoint kernels (bricks
of 128 voxels near-exact, 64 relaxed), so every x_3 segment of the launch is compared.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_09841_b300 import inputs
from paper_2110_09841_b300.kct import Projector


VARIANTS = [("exact", 0), ("relaxed", 1)]
SCALINGS = [("cos", 0), ("exact", 1)]
FULL = ["cvp256", "cvp512", "cvp512wide"]
TOL = 1e-4
GAP = 1e-5


def check_sampled(got, ref, vmax, what):
    err = np.abs(got - ref)
    assert np.all(err <= TOL * vmax), f"{what}: max |err| / max = {float((err / vmax).max()):.3e}"
    big = ref >= 1e-3 * vmax
    assert big.sum() >= len(ref) // 2, f"{what}: too few samples carry signal ({int(big.sum())})"
    rel = float((err[big] / ref[big]).max())
    assert rel <= TOL, f"{what}: max relative error {rel:.3e}"
    return rel


_Y_CACHE = {}


def projections(g):
    """U[0,1) adjoint input of the geometry's shape on the device, plus its FP64 host copy
    (cached: the two 512^3 workloads share the shape)."""
    key = g.proj_shape
    if key not in _Y_CACHE:
        _Y_CACHE.clear()
        y = inputs.uniform_projections(g.proj_shape, 4242, device="cuda")
        _Y_CACHE[key] = (y, y.cpu().double().numpy())
    return _Y_CACHE[key]


def sampled_voxels(g, vol, rng, count=24):
    """Voxels at the x_3 brick boundaries of both adjoint kernels and at x_1 brick
    boundaries, plus random ones, among the voxels that the detector sees: above 10 % of the
    backprojection's maximum where a slice has such voxels, else above 0.1 % (the slices at
    the ends of a tall volume are seen by a few views only)."""
    nz = g.nz
    ks = sorted({k for b in (64, 128) for s in range(0, nz, b) for k in (s, s + 1, s + b - 1) if k < nz} | {nz - 1})
    mx = float(vol.max())

    def pool_of(k):
        cand = np.argwhere(vol[k] > 0.1 * mx)
        return cand if len(cand) else np.argwhere(vol[k] > 1e-3 * mx)

    out = []
    for k in ks:
        cand = pool_of(k)
        if len(cand) == 0:
            continue
        # one voxel on an x_1 brick edge (i % 8 in {0, 7}) and one random voxel per slice
        edge = cand[(cand[:, 1] % 8 == 0) | (cand[:, 1] % 8 == 7)]
        for pool in (edge, cand):
            if len(pool):
                j, i = pool[rng.integers(0, len(pool))]
                out.append((k, int(j), int(i)))
    for _ in range(count):
        k = int(rng.integers(0, nz))
        cand = np.argwhere(vol[k] > 0.1 * mx)
        if len(cand):
            j, i = cand[rng.integers(0, len(cand))]
            out.append((k, int(j), int(i)))
    return np.array(out, dtype=np.int32)


def seen_bricks(vol, b):
    """x_3 bricks of b voxels that hold a voxel above 0.1 % of the maximum."""
    seen = (vol > 1e-3 * float(vol.max())).reshape(vol.shape[0], -1).any(axis=1)
    return {k // b for k in np.flatnonzero(seen)}


@pytest.mark.gpu
@pytest.mark.parametrize("name", FULL)
@pytest.mark.parametrize("vname,variant", VARIANTS)
@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_sampled_adjoint_full_size(name, vname, variant, sname, scaling):
    g = inputs.workload_geometry(name)
    y, y64 = projections(g)
    A = Projector(g, vname, sname)
    xb = A.backproject(y)
    torch.cuda.synchronize()
    assert A.device_error() == 0
    vol = xb.cpu().numpy()
    rng = np.random.default_rng(1000 + 10 * FULL.index(name) + 2 * variant + scaling)
    vox = sampled_voxels(g, vol, rng)
    # every x_3 brick of both adjoint kernels that the detector sees holds a sample
    for b in (64, 128):
        assert seen_bricks(vol, b) <= set((vox[:, 0] // b).tolist())
    ref = oracle.backproject_voxels(g, y64, vox, variant, scaling)
    got = vol[vox[:, 0], vox[:, 1], vox[:, 2]].astype(np.float64)
    check_sampled(got, ref, float(vol.max()), f"{name} {vname}/{sname} adjoint")


@pytest.mark.gpu
@pytest.mark.parametrize("name", FULL)
@pytest.mark.parametrize("vname,variant", VARIANTS)
@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_sampled_forward_full_size(name, vname, variant, sname, scaling):
    g = inputs.workload_geometry(name)
    x = inputs.workload_phantom(name, device="cuda")
    A = Projector(g, vname, sname)
    b = A.project(x)
    torch.cuda.synchronize()
    assert A.device_error() == 0
    rng = np.random.default_rng(2000 + 10 * FULL.index(name) + 2 * variant + scaling)
    views = [0, g.nviews // 4, g.nviews // 2 + 1, g.nviews - 1]
    pix = []
    vmax = {}
    for view in views:
        bv = b[view].cpu().numpy()
        vmax[view] = float(bv.max())
        cand = np.argwhere(bv > 0.05 * vmax[view])
        for r, c in cand[rng.choice(len(cand), 10, replace=False)]:
            pix.append((view, int(r), int(c)))
    pix = np.array(pix, dtype=np.int32)
    ref = oracle.project_pixels(g, x.cpu().numpy(), pix, variant, scaling)
    got = b[pix[:, 0], pix[:, 1], pix[:, 2]].cpu().double().numpy()
    check_sampled(got, ref, np.array([vmax[v] for v in pix[:, 0]]), f"{name} {vname}/{sname} forward")


@pytest.mark.gpu
@pytest.mark.parametrize("name", FULL)
@pytest.mark.parametrize("vname", ["exact", "relaxed"])
def test_adjoint_gap_full_size(name, vname):
    g = inputs.workload_geometry(name)
    x = inputs.uniform_volume(g.vol_shape, 31, device="cuda")
    y, _ = projections(g)
    A = Projector(g, vname, "cos")
    lhs = 0.0
    Ax = A.project(x)
    for v0 in range(0, g.nviews, 64):           # FP64 dot in view slices (bounded memory)
        lhs += float((Ax[v0:v0 + 64].double() * y[v0:v0 + 64].double()).sum())
    del Ax
    Aty = A.backproject(y)
    rhs = float((x.double() * Aty.double()).sum())
    torch.cuda.synchronize()
    assert A.device_error() == 0
    gap = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    assert gap <= GAP, gap


# ---------------------------------------------------------------------------------------
# Fallback paths: brick footprints larger than the shared detector tile
# ---------------------------------------------------------------------------------------

TILE_FLOATS = {0: 12288, 1: 8192}     # shared detector tile of the near-exact / relaxed kernels
BRICK_Z = {0: (128, 128), 1: (128, 64)}   # voxels along x_3 of a forward / adjoint brick


def brick_tile_pixels(g, view, i0, j0, k0, bx, by, bz):
    """Pixels of the window (bounding box of the projected brick corners plus one pixel of
    margin, clipped to the detector) that a brick covers in one view."""
    P = g.pmats[view]
    x0 = [-(g.nx - 1) * g.ax / 2, -(g.ny - 1) * g.ay / 2, -(g.nz - 1) * g.az / 2]
    us, vs = [], []
    for i in (i0, min(i0 + bx, g.nx)):
        for j in (j0, min(j0 + by, g.ny)):
            for k in (k0, min(k0 + bz, g.nz)):
                X = np.array([x0[0] + (i - 0.5) * g.ax, x0[1] + (j - 0.5) * g.ay, x0[2] + (k - 0.5) * g.az, 1.0])
                h = P @ X
                us.append(h[0] / h[2])
                vs.append(h[1] / h[2])
    u0 = max(int(np.floor(min(us) + 0.5)) - 1, 0)
    u1 = min(int(np.floor(max(us) + 0.5)) + 1, g.nu - 1)
    v0 = max(int(np.floor(min(vs) + 0.5)) - 1, 0)
    v1 = min(int(np.floor(max(vs) + 0.5)) + 1, g.nv - 1)
    return (u1 - u0 + 1) * (v1 - v0 + 1)


def overflow_geometry():
    """8 x 8 x 40 voxels of 1 mm seen through 0.25 mm pixels at magnification 5/3: a voxel
    spans about 7 x 7 pixels and a brick's window ~ 60 x 290 pixels, larger than either
    kernel's shared tile. The detector cuts off the top and bottom rows of the footprint."""
    P = inputs.circular_pmats(4, 300.0, 500.0, 90, 250, 0.25, 0.25, 360.0, 10.0, cu=46.3, cv=121.8)
    return inputs.Geometry(8, 8, 40, 1.0, 1.0, 1.0, 90, 250, 0.25, 0.25, P)


def test_overflow_geometry_exceeds_the_tiles():
    g = overflow_geometry()
    for variant in (0, 1):
        for bz in BRICK_Z[variant]:
            for view in range(g.nviews):
                assert brick_tile_pixels(g, view, 0, 0, 0, 8, 8, bz) > TILE_FLOATS[variant]


@pytest.mark.gpu
@pytest.mark.parametrize("vname,variant", VARIANTS)
@pytest.mark.parametrize("sname,scaling", SCALINGS)
def test_tile_overflow_falls_back_to_global_memory(vname, variant, sname, scaling):
    """Every brick overflows the shared tile, so the forward adds each pair to global
    memory (times F) and the adjoint reads each y from global memory (times F): compared
    element by element with the oracle, plus the adjoint identity."""
    g = overflow_geometry()
    x = np.random.default_rng(71).random(g.vol_shape)
    y = np.random.default_rng(72).random(g.proj_shape)
    A = Projector(g, vname, sname)
    xd = torch.as_tensor(x, dtype=torch.float32).cuda()
    yd = torch.as_tensor(y, dtype=torch.float32).cuda()
    b = A.project(xd)
    xb = A.backproject(yd)
    torch.cuda.synchronize()
    assert A.device_error() == 0
    ref_b = oracle.project(g, xd.cpu().double().numpy(), variant, scaling)
    ref_x = oracle.backproject(g, yd.cpu().double().numpy(), variant, scaling)
    bn, xn = b.cpu().double().numpy(), xb.cpu().double().numpy()
    for view in range(g.nviews):
        check_sampled(bn[view].ravel(), ref_b[view].ravel(), float(np.abs(ref_b[view]).max()),
                      f"overflow forward view {view}")
    d = np.abs(xn - ref_x)
    mx = float(np.abs(ref_x).max())
    assert d.max() <= TOL * mx
    big = np.abs(ref_x) >= 1e-3 * mx
    assert (d[big] / np.abs(ref_x[big])).max() <= TOL
    lhs = float((bn * yd.cpu().double().numpy()).sum())
    rhs = float((xd.cpu().double().numpy() * xn).sum())
    assert abs(lhs - rhs) / max(abs(lhs), abs(rhs)) <= GAP
