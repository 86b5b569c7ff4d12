"""The paper's accuracy comparison (Sec. IV-B) on the oracle.

Single voxel: the projection of a 1 x 1 x 5 mm voxel at the centre of rotation onto a fine
detector (616 x 480 cells of 0.154 mm, SID 749 / SDD 1198 mm), per view, by the relative
Frobenius error of the view. The near-exact and relaxed CVP values must agree with the K = 32
ray average far better than a single ray through each pixel centre does, and the ray average
must approach them as K grows (the remaining difference is the ray average's own sampling
error).

Against the truth: the oracle's truth mode gives the pixel value each scaling approximates,
the limit of ray integration with no sampling error: for the exact scaling the solid-angle
average of the line integrals over the pixel (Eq. integub; pair weights J = int_cut r^-2 dV,
Eq. intcut), for the cos scaling their area average (Eq. integ). Each variant's error against
it is what its pair weight approximates: the near-exact weight |V_cut| / r^2 with r at the
cut's centre of mass (Eq. vox) errs by O((diam / r)^2), the relaxed A_n d / r_vox^2 (Eq.
cutvolume) by more; the cos scaling adds its pixel factor taken at the pixel centre. Measured
on the single voxel and on sampled pixels of the benchmark workloads.
"""
import numpy as np
import pytest

import oracle
from paper_2110_09841_b300 import inputs


def frob(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("variant", [oracle.EXACT, oracle.RELAXED])
def test_single_voxel_cvp_error_far_below_single_ray(variant):
    g = inputs.make_geometry((1, 1, 1), (1.0, 1.0, 5.0), (616, 480), (0.154, 0.154), 8, 749.0, 1198.0, 360.0)
    x = np.ones(g.vol_shape)
    b = oracle.project(g, x, variant)
    for view in (0, 1, 3):
        m_idx, n_idx = np.nonzero(b[view])
        m0, m1 = m_idx.min() - 1, m_idx.max() + 2
        n0, n1 = n_idx.min() - 1, n_idx.max() + 2
        ref = np.array([[oracle.ray_pixel(g, x, view, float(n), float(m), 32) for n in range(n0, n1)]
                        for m in range(m0, m1)])
        ref64 = np.array([[oracle.ray_pixel(g, x, view, float(n), float(m), 64) for n in range(n0, n1)]
                          for m in range(m0, m1)])
        one = np.array([[oracle.ray_pixel(g, x, view, float(n), float(m), 1) for n in range(n0, n1)]
                        for m in range(m0, m1)])
        e_cvp = frob(b[view, m0:m1, n0:n1], ref)
        e_ray = frob(one, ref)
        assert e_cvp < 5e-3, (view, e_cvp)
        assert e_cvp < 0.2 * e_ray, (view, e_cvp, e_ray)
        assert frob(b[view, m0:m1, n0:n1], ref64) < 0.75 * e_cvp


def rel_l2(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def test_single_voxel_errors_against_the_truth():
    g = inputs.make_geometry((1, 1, 1), (1.0, 1.0, 5.0), (616, 480), (0.154, 0.154), 8, 749.0, 1198.0, 360.0)
    x = np.ones(g.vol_shape)
    for view in (0, 1):
        b = oracle.project(g.subset_views([view]), x, oracle.EXACT, oracle.SCALE_EXACT)[0]
        m_idx, n_idx = np.nonzero(b)
        pix = np.array([[view, m, n] for m in range(m_idx.min() - 1, m_idx.max() + 2)
                        for n in range(n_idx.min() - 1, n_idx.max() + 2)])
        truth = oracle.project_pixels(g, x, pix, oracle.TRUTH, oracle.SCALE_EXACT)
        e_ex = rel_l2(oracle.project_pixels(g, x, pix, oracle.EXACT, oracle.SCALE_EXACT), truth)
        e_rel = rel_l2(oracle.project_pixels(g, x, pix, oracle.RELAXED, oracle.SCALE_EXACT), truth)
        e_k32 = rel_l2(np.array([oracle.ray_pixel(g, x, view, float(n), float(m), 32, weighting=1)
                                 for _, m, n in pix]), truth)
        assert e_ex < 1e-6, e_ex
        assert 3 * e_ex < e_rel < 2e-5, (e_ex, e_rel)
        assert e_k32 > 100 * e_ex, (e_ex, e_k32)


def signal_pixels(g, views, count, seed):
    """(view, v, u) of pixels that see the phantom: projections of random points of the ball
    (radius 0.35 of the volume edge) that holds the ellipsoid centres, `count` per view."""
    rng = np.random.default_rng(seed)
    edge = g.nx * g.ax
    out = []
    for view in views:
        n = 0
        while n < count:
            p = rng.uniform(-0.35, 0.35, 3) * edge
            if np.linalg.norm(p) >= 0.35 * edge:
                continue
            h = g.pmats[view] @ np.append(p, 1.0)
            u, v = int(round(h[0] / h[2])), int(round(h[1] / h[2]))
            if 0 <= u < g.nu and 0 <= v < g.nv:
                out.append((view, v, u))
                n += 1
    return np.array(out, dtype=np.int32)


ACCURACY_WORKLOADS = ["cvp256", "cvp512", "cvp512wide"]
_PHANTOMS = {}


def workload_phantom64(name):
    """The workload's seeded phantom in float64; the last one is kept (the tests of one
    workload follow each other, and a 512^3 phantom holds 1 GB)."""
    if name not in _PHANTOMS:
        _PHANTOMS.clear()
        _PHANTOMS[name] = inputs.workload_phantom(name).numpy().astype(np.float64)
    return _PHANTOMS[name]


@pytest.mark.parametrize("scaling", [oracle.SCALE_EXACT, oracle.SCALE_COS])
@pytest.mark.parametrize("name", ACCURACY_WORKLOADS)
def test_variants_against_the_truth_at_workload_geometries(name, scaling):
    """8 views, 25 sampled pixels each, of the seeded phantom. With the exact scaling the
    near-exact error is the centroid approximation (about 1e-7 here); the cos scaling adds
    the pixel factor taken at the pixel centre (Eq. cvp: cos theta and R constant over the
    pixel), up to a few 1e-6 on single pixels at the 20 degree cone. The relaxed error is at
    least 10x larger."""
    g = inputs.workload_geometry(name)
    views = list(range(0, g.nviews, g.nviews // 8))[:8]
    x = workload_phantom64(name)
    pix = signal_pixels(g, views, 25, 31)
    truth = oracle.project_pixels(g, x, pix, oracle.TRUTH, scaling)
    keep = truth > 0.05 * truth.max()
    assert keep.sum() > 150
    e_ex = rel_l2(oracle.project_pixels(g, x, pix, oracle.EXACT, scaling)[keep], truth[keep])
    e_rel = rel_l2(oracle.project_pixels(g, x, pix, oracle.RELAXED, scaling)[keep], truth[keep])
    sname = "exact" if scaling == oracle.SCALE_EXACT else "cos"
    print(f"{name} {sname} scaling: near-exact {e_ex:.2e}, relaxed {e_rel:.2e} (relative L2 against the truth)")
    assert e_ex < (3e-7 if scaling == oracle.SCALE_EXACT else 1e-6), e_ex
    assert e_rel > 10 * e_ex, (e_ex, e_rel)
