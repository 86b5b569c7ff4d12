"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests compare the oracle with itself: each one checks it against a
closed form, a textbook routine written here in numpy, an invariant of the method
(Kulvait & Rose, arXiv 2110.09841), or an independent brute-force construction.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2110_09841_b300 import inputs

RNG = np.random.default_rng(12345)


def small_geometry(n=(4, 4, 4), a=(1.0, 1.0, 1.0), det=(24, 20), pitch=(1.0, 1.0), nviews=6,
                   sid=60.0, sdd=90.0, arc=360.0):
    return inputs.make_geometry(n, a, det, pitch, nviews, sid, sdd, arc)


def voxel_bounds(g, i, j, k):
    a = np.array([g.ax, g.ay, g.az])
    n = np.array([g.nx, g.ny, g.nz])
    c = (-n * a + a) / 2.0 + np.array([i, j, k]) * a
    return c - a / 2, c + a / 2, c


def project_uv(P, X):
    h = P @ np.append(X, 1.0)
    return h[0] / h[2], h[1] / h[2]


def corners(lo, hi):
    return [np.array([hi[0] if n & 1 else lo[0], hi[1] if n & 2 else lo[1], hi[2] if n & 4 else lo[2]])
            for n in range(8)]


# --------------------------------------------------------------------------------------
# Convex polytope clipping: closed forms
# --------------------------------------------------------------------------------------

def test_clip_corner_tetrahedron():
    # plane x/p + y/q + z/r <= 1 cuts the corner tetrahedron of the positive octant:
    # volume p q r / 6, centroid (p, q, r) / 4
    lo, hi = np.zeros(3), np.array([3.0, 4.0, 5.0])
    p, q, r = 1.3, 2.1, 0.7
    V, c = oracle.box_clip(lo, hi, [[-1 / p, -1 / q, -1 / r, 1.0]])
    assert V == pytest.approx(p * q * r / 6, rel=1e-13)
    np.testing.assert_allclose(c, [p / 4, q / 4, r / 4], rtol=1e-12)


def test_clip_half_box_and_complement():
    lo, hi = np.array([-1.0, -2.0, 0.5]), np.array([2.0, 1.0, 1.5])
    V, c = oracle.box_clip(lo, hi, [[1.0, 0.0, 0.0, -0.5]])          # x >= 0.5
    assert V == pytest.approx(1.5 * 3.0 * 1.0, rel=1e-14)
    np.testing.assert_allclose(c, [1.25, -0.5, 1.0], atol=1e-13)
    for _ in range(50):
        n = RNG.normal(size=3)
        d = RNG.uniform(-1.0, 1.0)
        V1, c1 = oracle.box_clip(lo, hi, [[*n, d]])
        V2, c2 = oracle.box_clip(lo, hi, [[*(-n), -d]])
        assert V1 + V2 == pytest.approx(9.0, rel=1e-13)
        if V1 > 1e-9 and V2 > 1e-9:   # first moments add up to the box's
            np.testing.assert_allclose(V1 * c1 + V2 * c2, 9.0 * (lo + hi) / 2, atol=1e-11)


def test_clip_face_coincident_planes():
    lo, hi = np.zeros(3), np.ones(3)
    V, _ = oracle.box_clip(lo, hi, [[1.0, 0.0, 0.0, 0.0]])     # x >= 0 contains the -x face
    assert V == pytest.approx(1.0, rel=1e-15)
    V, _ = oracle.box_clip(lo, hi, [[-1.0, 0.0, 0.0, 0.0]])    # x <= 0 touches the box only
    assert V == 0.0
    V, _ = oracle.box_clip(lo, hi, [[0.0, 1.0, 0.0, -0.5], [0.0, -1.0, 0.0, 0.5]])   # y = 0.5 slab
    assert V == pytest.approx(0.0, abs=1e-14)


def test_clip_two_planes_monte_carlo():
    # box cut by two random planes, checked against a stratified point count
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 1.5])
    n1, n2 = np.array([1.0, 0.3, -0.4]), np.array([-0.2, 1.0, 0.5])
    planes = [[*n1, -0.3], [*n2, -0.8]]
    V, c = oracle.box_clip(lo, hi, planes)
    m = 120
    g = [(np.arange(m) + 0.5) / m * (hi[d] - lo[d]) + lo[d] for d in range(3)]
    X, Y, Z = np.meshgrid(*g, indexing="ij")
    inside = (n1[0] * X + n1[1] * Y + n1[2] * Z - 0.3 >= 0) & (n2[0] * X + n2[1] * Y + n2[2] * Z - 0.8 >= 0)
    dv = np.prod(hi - lo) / m ** 3
    assert V == pytest.approx(inside.sum() * dv, rel=3e-3)
    np.testing.assert_allclose(c, [X[inside].mean(), Y[inside].mean(), Z[inside].mean()], atol=5e-3)


# --------------------------------------------------------------------------------------
# int r^-2 dV by the divergence theorem vs tensor Gauss-Legendre (P3)
# --------------------------------------------------------------------------------------

def gauss_legendre_box(lo, hi, s, n=24, split=4):
    xg, wg = np.polynomial.legendre.leggauss(n)
    total = 0.0
    edges = [np.linspace(lo[d], hi[d], split + 1) for d in range(3)]
    for a in range(split):
        for b in range(split):
            for c in range(split):
                pts, wts = [], []
                for d, idx in zip(range(3), (a, b, c)):
                    l, h = edges[d][idx], edges[d][idx + 1]
                    pts.append((xg + 1) / 2 * (h - l) + l)
                    wts.append(wg * (h - l) / 2)
                X, Y, Z = np.meshgrid(*pts, indexing="ij")
                W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
                total += (W / ((X - s[0]) ** 2 + (Y - s[1]) ** 2 + (Z - s[2]) ** 2)).sum()
    return total


@pytest.mark.parametrize("s", [(40.0, 3.0, -2.0), (-6.0, 9.0, 4.0), (2.0, -3.5, 0.7)])
def test_inv_r2_face_formula(s):
    lo, hi = np.array([-1.0, -0.5, 0.0]), np.array([1.5, 1.0, 2.0])
    ref = gauss_legendre_box(lo, hi, np.array(s))
    J = oracle.box_inv_r2(lo, hi, np.array(s), level=5)
    assert J == pytest.approx(ref, rel=1e-12)
    # the face rule is of degree 5: halving the triangles divides the error by ~2^6
    e2 = abs(oracle.box_inv_r2(lo, hi, np.array(s), level=1) - ref)
    e3 = abs(oracle.box_inv_r2(lo, hi, np.array(s), level=2) - ref)
    if e3 > 1e-13 * ref:
        assert 30.0 < e2 / e3 < 130.0


# --------------------------------------------------------------------------------------
# Solid angle of a pixel (exact scaling factor) and cos-scaling factor
# --------------------------------------------------------------------------------------

def vos_triangle(a, b, c):
    """Van Oosterom & Strackee (1983): solid angle of the triangle a, b, c seen from 0."""
    la, lb, lc = (np.linalg.norm(v) for v in (a, b, c))
    num = abs(np.dot(a, np.cross(b, c)))
    den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
    return 2.0 * math.atan2(num, den)


def corner_dirs(P, u, v):
    M = P[:, :3]
    return [np.linalg.solve(M, [uu, vv, 1.0]) for uu, vv in
            ((u - .5, v - .5), (u + .5, v - .5), (u + .5, v + .5), (u - .5, v + .5))]


def test_solid_angle_vs_van_oosterom_strackee():
    g = small_geometry(det=(40, 30), pitch=(3.0, 2.0), sid=50.0, sdd=80.0)
    for view in range(g.nviews):
        P = g.pmats[view]
        for u, v in ((0, 0), (19, 14), (39, 29), (7, 22)):
            t = corner_dirs(P, u, v)
            ref = vos_triangle(t[0], t[1], t[2]) + vos_triangle(t[0], t[2], t[3])
            assert oracle.pixel_solid_angle(P, u, v) == pytest.approx(ref, rel=1e-11)
            assert oracle.pixel_factor(P, u, v, oracle.SCALE_EXACT) == pytest.approx(1 / ref, rel=1e-11)


def rectangle_solid_angle(x0, x1, y0, y1, d):
    """Closed form for a rectangle in the plane at distance d, coordinates relative to
    the foot of the perpendicular: sum of +-atan(x y / (d sqrt(d^2 + x^2 + y^2)))."""
    f = lambda x, y: math.atan(x * y / (d * math.sqrt(d * d + x * x + y * y)))
    return f(x1, y1) - f(x0, y1) - f(x1, y0) + f(x0, y0)


def test_solid_angles_tile_the_detector():
    nu, nv, pu, pv, sdd = 12, 9, 5.0, 4.0, 40.0
    P = inputs.circular_pmats(1, 25.0, sdd, nu, nv, pu, pv, cu=4.3, cv=6.1)[0]
    tot = sum(oracle.pixel_solid_angle(P, u, v) for u in range(nu) for v in range(nv))
    ref = rectangle_solid_angle((-0.5 - 4.3) * pu, (nu - 0.5 - 4.3) * pu,
                                (-0.5 - 6.1) * pv, (nv - 0.5 - 6.1) * pv, sdd)
    assert tot == pytest.approx(ref, rel=1e-12)


def test_cos_factor_closed_form():
    # Eq. cvp: F = f^2 / (a cos^3 theta); at the principal point cos theta = 1
    sdd, pu, pv = 1200.0, 0.8, 0.6
    P = inputs.circular_pmats(3, 750.0, sdd, 64, 48, pu, pv)
    for view in range(3):
        assert oracle.pixel_factor(P[view], 31.5, 23.5, 0) == pytest.approx(sdd * sdd / (pu * pv), rel=1e-13)
        u, v = 3.0, 40.0
        du, dv = (u - 31.5) * pu, (v - 23.5) * pv
        cth = sdd / math.sqrt(sdd * sdd + du * du + dv * dv)
        assert oracle.pixel_factor(P[view], u, v, 0) == pytest.approx(sdd * sdd / (pu * pv * cth ** 3), rel=1e-13)
        # small pixels: 1 / F_cos is the midpoint value of the solid angle, O(p^2/f^2) apart
        assert oracle.pixel_factor(P[view], u, v, 1) == pytest.approx(oracle.pixel_factor(P[view], u, v, 0), rel=1e-6)


# --------------------------------------------------------------------------------------
# Invariants of the cutting voxel projector
# --------------------------------------------------------------------------------------

def footprint(P, lo, hi, nu, nv):
    uv = np.array([project_uv(P, c) for c in corners(lo, hi)])
    u0, u1 = int(math.floor(uv[:, 0].min() + 0.5)), int(math.floor(uv[:, 0].max() + 0.5))
    v0, v1 = int(math.floor(uv[:, 1].min() + 0.5)), int(math.floor(uv[:, 1].max() + 0.5))
    inside = u0 >= 0 and v0 >= 0 and u1 < nu and v1 < nv
    return u0, u1, v0, v1, inside


@pytest.mark.parametrize("view", [0, 1, 3])
def test_partition_of_unity(view):
    """P1: the cut volumes of a voxel over all pixels add up to its volume."""
    g = small_geometry(n=(5, 5, 5), a=(1.0, 0.8, 1.3), det=(40, 40), pitch=(0.7, 0.6))
    P = g.pmats[view]
    for (i, j, k) in [(0, 0, 0), (2, 2, 2), (4, 1, 3), (1, 4, 4)]:
        lo, hi, c = voxel_bounds(g, i, j, k)
        u0, u1, v0, v1, inside = footprint(P, lo, hi, g.nu, g.nv)
        assert inside
        sV = sWr = 0.0
        s = oracle.source(P)
        for u in range(u0, u1 + 1):
            for v in range(v0, v1 + 1):
                r = oracle.box_pixel(P, lo, hi, u, v)
                sV += r["V"]
                sWr += r["Wrel"] * np.sum((c - s) ** 2)
        vol = g.ax * g.ay * g.az
        assert sV == pytest.approx(vol, rel=1e-12)
        # relaxed: sum_n A_n = base area and sum_m d_m = a3
        assert sWr == pytest.approx(vol, rel=1e-12)


def test_additivity_over_voxels():
    """P1b: sum over voxels of V_cut(vox, pix) = |pyramid(pix) ∩ whole volume box|."""
    g = small_geometry(n=(4, 3, 5), a=(1.0, 1.2, 0.9))
    P = g.pmats[2]
    lo_all = -0.5 * np.array([g.nx * g.ax, g.ny * g.ay, g.nz * g.az])
    for u, v in [(11, 9), (12, 10), (10, 7), (13, 12)]:
        total = 0.0
        for k in range(g.nz):
            for j in range(g.ny):
                for i in range(g.nx):
                    lo, hi, _ = voxel_bounds(g, i, j, k)
                    total += oracle.box_pixel(P, lo, hi, u, v)["V"]
        ref = oracle.box_pixel(P, lo_all, -lo_all, u, v)["V"]
        assert ref > 0
        assert total == pytest.approx(ref, rel=1e-12)


def test_centroid_weight_vs_exact_integral():
    """W = V / |c - s|^2 approximates J = int r^-2 dV to O((diam / r)^2) (Eq. vox)."""
    g = small_geometry()
    P = g.pmats[1]
    s = oracle.source(P)
    for (i, j, k) in [(0, 0, 0), (3, 2, 1)]:
        lo, hi, c = voxel_bounds(g, i, j, k)
        u0, u1, v0, v1, _ = footprint(P, lo, hi, g.nu, g.nv)
        r2 = np.sum((c - s) ** 2)
        for u in range(u0, u1 + 1):
            for v in range(v0, v1 + 1):
                q = oracle.box_pixel(P, lo, hi, u, v, quad_level=1)
                if q["V"] > 1e-6:
                    assert abs(q["W"] - q["J"]) <= 3.0 / r2 * q["J"]


def gauss_legendre_box_fn(lo, hi, f, n=12, split=2):
    """Tensor Gauss-Legendre integral of f(X, Y, Z) over the box [lo, hi]."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    total = 0.0
    edges = [np.linspace(lo[d], hi[d], split + 1) for d in range(3)]
    for a in range(split):
        for b in range(split):
            for c in range(split):
                pts, wts = [], []
                for d, idx in zip(range(3), (a, b, c)):
                    l, h = edges[d][idx], edges[d][idx + 1]
                    pts.append((xg + 1) / 2 * (h - l) + l)
                    wts.append(wg * (h - l) / 2)
                X, Y, Z = np.meshgrid(*pts, indexing="ij")
                W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
                total += (W * f(X, Y, Z)).sum()
    return total


@pytest.mark.parametrize("scaling", [oracle.SCALE_EXACT, oracle.SCALE_COS])
def test_truth_mode_adds_up_to_the_voxel_integral(scaling):
    """The truth mode of the sampled projection, summed over a voxel's pixels, is the voxel's
    whole integral of the pair integrand: exact scaling, int r^-2 dV (Eq. intcut; the pixel
    factor 1 / abar divided out); cos scaling, the area element per volume element
    |det M| r / |w|^3 (w the depth along the detector normal, Eq. integ). Tensor
    Gauss-Legendre computes the box integrals. The CVP weights differ from them by
    O((a / r)^2) (centroid r) or more (cos factor at the pixel centre), so a truth mode that
    fell back to them would fail."""
    g = small_geometry(n=(5, 5, 5), a=(1.0, 0.8, 1.3), det=(40, 40), pitch=(0.7, 0.6))
    for view in (0, 3):
        P = g.pmats[view]
        s = oracle.source(P)
        M = P[:, :3]
        if scaling == oracle.SCALE_EXACT:
            def f(X, Y, Z):
                return 1.0 / ((X - s[0]) ** 2 + (Y - s[1]) ** 2 + (Z - s[2]) ** 2)
        else:
            def f(X, Y, Z):
                r = np.sqrt((X - s[0]) ** 2 + (Y - s[1]) ** 2 + (Z - s[2]) ** 2)
                w = M[2, 0] * (X - s[0]) + M[2, 1] * (Y - s[1]) + M[2, 2] * (Z - s[2])
                return abs(np.linalg.det(M)) * r / np.abs(w) ** 3
        for (i, j, k) in [(0, 0, 0), (2, 2, 2), (4, 1, 3)]:
            lo, hi, _ = voxel_bounds(g, i, j, k)
            u0, u1, v0, v1, inside = footprint(P, lo, hi, g.nu, g.nv)
            assert inside
            x = np.zeros(g.vol_shape)
            x[k, j, i] = 1.0
            pix = np.array([[view, v, u] for u in range(u0, u1 + 1) for v in range(v0, v1 + 1)])
            F = np.array([oracle.pixel_factor(P, u, v, oracle.SCALE_EXACT) for _, v, u in pix])
            if scaling == oracle.SCALE_COS:
                F = np.ones(len(pix))
            t = oracle.project_pixels(g, x, pix, oracle.TRUTH, scaling) / F
            w = oracle.project_pixels(g, x, pix, oracle.EXACT, scaling) / F
            ref = gauss_legendre_box_fn(lo, hi, f)
            assert t.sum() == pytest.approx(ref, rel=1e-12)
            assert abs(w.sum() / ref - 1.0) > 1e-7


@pytest.mark.parametrize("scaling", [oracle.SCALE_EXACT, oracle.SCALE_COS])
def test_truth_mode_is_the_limit_of_ray_integration(scaling):
    """The truth mode is the limit of ray integration with exact path lengths: K x K rays,
    solid-angle weighted for the exact scaling (Eq. integub), equally weighted for the cos
    scaling (Eq. integ), converge to it, and where they have converged (all but the corner
    pixel) they are closer to it than to the near-exact CVP value."""
    g = small_geometry(n=(4, 4, 4), det=(24, 20), pitch=(0.4, 0.4), nviews=3, sid=200.0, sdd=300.0)
    x = np.random.default_rng(5).uniform(0.5, 1.5, g.vol_shape)
    for view, u, v, tol in [(0, 12, 10, 1e-9), (1, 10, 8, 1e-7), (2, 13, 11, 1e-7), (1, 19, 16, 1e-8),
                            (0, 4, 3, 2e-5)]:     # the last pixel sees a corner of the volume
        pix = np.array([[view, v, u]])
        t = oracle.project_pixels(g, x, pix, oracle.TRUTH, scaling)[0]
        w = oracle.project_pixels(g, x, pix, oracle.EXACT, scaling)[0]
        r = oracle.ray_pixel(g, x, view, u, v, 256, weighting=1 if scaling == oracle.SCALE_EXACT else 0)
        assert abs(r / t - 1.0) <= tol
        if tol < 1e-6:                        # K = 256 has converged past the CVP error
            assert abs(r - t) < abs(r - w)


def test_single_voxel_in_one_big_pixel():
    """P5: a voxel wholly inside one pixel gives W = a^3 / |c - s|^2 and J equals the
    tensor Gauss-Legendre integral of r^-2 over the box."""
    P = inputs.circular_pmats(1, 100.0, 150.0, 3, 3, 40.0, 40.0)[0]
    lo, hi = np.array([-0.5, -0.4, -0.3]), np.array([0.5, 0.4, 0.3])
    q = oracle.box_pixel(P, lo, hi, 1, 1, quad_level=2)
    s = oracle.source(P)
    c = (lo + hi) / 2
    vol = np.prod(hi - lo)
    assert q["V"] == pytest.approx(vol, rel=1e-13)
    np.testing.assert_allclose(q["c"], c, atol=1e-12)
    assert q["W"] == pytest.approx(vol / np.sum((c - s) ** 2), rel=1e-13)
    assert q["J"] == pytest.approx(gauss_legendre_box(lo, hi, s, n=12, split=2), rel=1e-12)
    assert q["Wrel"] == pytest.approx(vol / np.sum((c - s) ** 2), rel=1e-13)


def slab_chord(s, d, lo, hi):
    """Textbook slab method: length of the ray s + t d (t > 0) inside box [lo, hi]."""
    t0, t1 = 0.0, np.inf
    for a in range(3):
        if d[a] == 0:
            if not (lo[a] < s[a] < hi[a]):
                return 0.0
            continue
        ta, tb = sorted(((lo[a] - s[a]) / d[a], (hi[a] - s[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(0.0, t1 - t0) * np.linalg.norm(d)


def slab_chords(s, D, lo, hi):
    """Vectorised slab method for many directions D [n, 3] (source strictly outside the
    slabs of any zero direction component)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t_a = (lo[None, :] - s[None, :]) / D
        t_b = (hi[None, :] - s[None, :]) / D
    t0 = np.maximum(np.minimum(t_a, t_b).max(axis=1), 0.0)
    t1 = np.maximum(t_a, t_b).min(axis=1)
    return np.maximum(t1 - t0, 0.0) * np.linalg.norm(D, axis=1)


@pytest.mark.parametrize("scaling", [0, 1])
def test_uniform_box_chord_length(scaling):
    """P6: for a uniform box the pixel value is the pixel average of the chord length:
    equal-area average for cos scaling (Eq. integ), solid-angle weighted average for
    exact scaling (Eq. integub). The average is taken here by brute force over K x K
    rays with the textbook slab method."""
    # at r = 400 mm the centre-of-mass r of Eq. vox differs from int r^-2 by ~1e-6
    g = small_geometry(n=(6, 6, 6), a=(1.0, 1.0, 1.0), det=(40, 40), pitch=(0.3, 0.3), nviews=3,
                       sid=400.0, sdd=600.0)
    x = np.ones(g.vol_shape)
    b = oracle.project(g, x, scaling=scaling)
    lo, hi = -3.0 * np.ones(3), 3.0 * np.ones(3)
    K = 48
    off = (np.arange(K) + 0.5) / K - 0.5
    du, dv = [a.ravel() for a in np.meshgrid(off, off, indexing="ij")]
    checked = 0
    for view in range(g.nviews):
        P = g.pmats[view]
        s = oracle.source(P)
        Minv = np.linalg.inv(P[:, :3])
        for u in range(g.nu):
            for v in range(g.nv):
                C = slab_chords(s, (Minv @ np.array([[u, u - .5, u + .5, u + .5, u - .5],
                                                     [v, v - .5, v - .5, v + .5, v + .5],
                                                     [1, 1, 1, 1, 1]])).T, lo, hi)
                if C.min() < 2.0 or C.max() - C.min() > 0.05 * C[0]:
                    continue      # pixel not wholly on the box, or chord not smooth over it
                D = (Minv @ np.stack([u + du, v + dv, np.ones_like(du)])).T
                L = slab_chords(s, D, lo, hi)
                w = np.ones_like(L) if scaling == 0 else np.linalg.norm(D, axis=1) ** -3
                ref = float((w * L).sum() / w.sum())
                assert b[view, v, u] == pytest.approx(ref, rel=1e-5)
                checked += 1
    assert checked > 50


def test_rotation_symmetry():
    """P7: turning the centred volume by 90 degrees about x3 and the trajectory by 90
    degrees gives identical projections."""
    g = small_geometry(n=(5, 5, 4), det=(26, 22), nviews=4, arc=360.0)
    x = RNG.random(g.vol_shape)
    n = g.nx
    xr = np.empty_like(x)
    for j in range(n):
        for i in range(n):
            xr[:, i, n - 1 - j] = x[:, j, i]     # (x, y) -> (-y, x)
    for variant in (0, 1):
        b = oracle.project(g, x, variant=variant)
        br = oracle.project(g, xr, variant=variant)
        for view in range(4):
            np.testing.assert_allclose(br[(view + 1) % 4], b[view], rtol=1e-11, atol=1e-13 * b.max())


def test_relaxed_exact_at_zero_elevation():
    """P8: where the row boundary plane through the voxel is horizontal (it contains the
    source, x3 = s3) the relaxed estimate A_n * d is the exact cut volume (Sec. III-A)."""
    P = inputs.circular_pmats(8, 60.0, 90.0, 30, 20, 1.0, 1.0)    # cv = 9.5: boundary at x3 = 0
    lo, hi = np.array([-0.5, 0.3, -0.4]), np.array([0.5, 1.3, 0.4])
    for view in range(8):
        s = oracle.source(P[view])
        c = (lo + hi) / 2
        r2 = np.sum((c - s) ** 2)
        for u in range(30):
            for v in (9, 10):
                q = oracle.box_pixel(P[view], lo, hi, u, v)
                assert q["Wrel"] * r2 == pytest.approx(q["V"], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("variant,scaling", [(0, 0), (0, 1), (1, 0)])
def test_adjoint_identity(variant, scaling):
    """P2 (Sec. III-D): <A x, y> = <x, A^T y>."""
    g = small_geometry(n=(4, 5, 3), det=(20, 16), nviews=3)
    x = RNG.random(g.vol_shape)
    y = RNG.random(g.proj_shape)
    Ax = oracle.project(g, x, variant, scaling)
    Aty = oracle.backproject(g, y, variant, scaling)
    lhs, rhs = float(np.sum(Ax * y)), float(np.sum(x * Aty))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_sampled_modes_match_full():
    g = inputs.workload_geometry("cvp32")
    x = inputs.workload_phantom("cvp32").numpy().astype(np.float64)
    y = inputs.uniform_projections(g.proj_shape, 7).numpy().astype(np.float64)
    sub = g.subset_views([0, 5, 13])
    b = oracle.project(sub, x)
    pix = np.array([[v, r, c] for v in range(3) for r in (0, 11, 24, 47) for c in (0, 17, 32, 63)])
    np.testing.assert_allclose(oracle.project_pixels(sub, x, pix), b[pix[:, 0], pix[:, 1], pix[:, 2]],
                               rtol=1e-13, atol=1e-16)
    xb = oracle.backproject(sub, y[[0, 5, 13]])
    vox = np.array([[k, j, i] for k in (0, 15, 31) for j in (3, 16) for i in (0, 20, 31)])
    np.testing.assert_allclose(oracle.backproject_voxels(sub, y[[0, 5, 13]], vox),
                               xb[vox[:, 0], vox[:, 1], vox[:, 2]], rtol=1e-13)


# --------------------------------------------------------------------------------------
# Convergence to ray integration (Sec. II-C: SiddonK as K -> infinity)
# --------------------------------------------------------------------------------------

@pytest.mark.slow
def test_converges_to_ray_integration():
    """P4: the area-averaged ray integral over K x K rays converges to the cos-scaled
    value and the solid-angle weighted one to the exact-scaled value; what remains at
    large K is the centre-of-mass approximation of Eq. vox, O((a / r)^2)."""
    g = small_geometry(n=(4, 4, 4), det=(24, 20), pitch=(0.4, 0.4), nviews=3, sid=200.0, sdd=300.0)
    x = RNG.uniform(0.5, 1.5, g.vol_shape)
    b_cos = oracle.project(g, x, 0, 0)
    b_ex = oracle.project(g, x, 0, 1)
    for view, u, v in [(0, 12, 10), (1, 10, 8), (2, 13, 11), (0, 4, 3), (1, 19, 16)]:
        assert b_cos[view, v, u] > 0
        r = oracle.ray_pixel(g, x, view, u, v, 256, weighting=0)
        assert r == pytest.approx(b_cos[view, v, u], rel=5e-5)
        r = oracle.ray_pixel(g, x, view, u, v, 256, weighting=1)
        assert r == pytest.approx(b_ex[view, v, u], rel=5e-5)
    # a wrong pixel factor or a dropped cut would be visible at K = 8 already
    r8 = oracle.ray_pixel(g, x, 0, 12, 10, 8, weighting=0)
    assert r8 == pytest.approx(b_cos[0, 10, 12], rel=1e-3)
