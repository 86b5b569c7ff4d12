"""Seeded synthetic inputs for the cutting voxel projector.

This module builds inputs only: circular-trajectory projection matrices, seeded
ellipsoid phantoms, perfusion-like frame stacks and uniform projection data.
It contains none of the projector's arithmetic, so both the CUDA path and the
CPU oracle may take their inputs from here.

Geometry conventions (Kulvait & Rose, arXiv 2110.09841):
  * the volume box is centred at the origin and voxel (i, j, k) has its centre at
    x0 + (i a1, j a2, k a3) with x0 = (-l + a)/2 (Sec. II-A);
  * pixel (m, n) has its centre at detector index coordinates (m, n), the origin
    being the centre of the corner pixel (Sec. II-B and Fig. 3);
  * the detector chi_2 axis is parallel to world x_3 with the opposite direction
    (Sec. III-A), which makes column projections independent of x_3;
  * each view is a 3x4 camera matrix P mapping homogeneous world points (mm) to
    homogeneous detector index coordinates (u, v, 1) (Sec. III-C).

Array layouts used throughout the package:
  volume       float32 [nz][ny][nx]   (x_1 fastest)
  projections  float32 [nviews][nv][nu]  (u = chi_1 column index fastest, v = row)
  matrices     float64 [nviews][3][4] row-major
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np


# --------------------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Geometry:
    """A cone-beam problem: voxel grid, flat detector and per-view matrices."""

    nx: int
    ny: int
    nz: int
    ax: float
    ay: float
    az: float
    nu: int
    nv: int
    pu: float
    pv: float
    pmats: np.ndarray  # float64 [nviews, 3, 4]

    @property
    def nviews(self) -> int:
        return int(self.pmats.shape[0])

    @property
    def vol_shape(self) -> tuple[int, int, int]:
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self) -> tuple[int, int, int]:
        return (self.nviews, self.nv, self.nu)

    @property
    def voxel_views(self) -> int:
        return self.nx * self.ny * self.nz * self.nviews

    def subset_views(self, idx: Sequence[int]) -> "Geometry":
        return dataclasses.replace(self, pmats=np.ascontiguousarray(self.pmats[list(idx)]))


def circular_pmats(nviews: int, sid: float, sdd: float, nu: int, nv: int,
                   pu: float, pv: float, arc_deg: float = 360.0,
                   start_deg: float = 0.0, cu: float | None = None,
                   cv: float | None = None) -> np.ndarray:
    """Projection matrices of a circular source trajectory around the x_3 axis.

    View k sits at angle phi_k = start + k * arc / nviews (half-open arc). The
    source is at sid * (cos phi, sin phi, 0); the detector is the plane at
    distance sdd from the source, normal to the central ray. Its u axis is
    (-sin phi, cos phi, 0) and its v axis is (0, 0, -1), so chi_2 runs opposite
    to x_3. The principal point defaults to the detector centre
    ((nu-1)/2, (nv-1)/2). Returns float64 [nviews, 3, 4].
    """
    if cu is None:
        cu = (nu - 1) / 2.0
    if cv is None:
        cv = (nv - 1) / 2.0
    K = np.array([[sdd / pu, 0.0, cu], [0.0, sdd / pv, cv], [0.0, 0.0, 1.0]])
    out = np.empty((nviews, 3, 4), dtype=np.float64)
    for k in range(nviews):
        phi = math.radians(start_deg + k * arc_deg / nviews)
        c, s = math.cos(phi), math.sin(phi)
        src = np.array([sid * c, sid * s, 0.0])
        R = np.array([[-s, c, 0.0],       # u axis
                      [0.0, 0.0, -1.0],   # v axis (opposite to x_3)
                      [-c, -s, 0.0]])     # central ray direction, source -> detector
        out[k, :, :3] = K @ R
        out[k, :, 3] = -(K @ R) @ src
    return out


def make_geometry(n: Sequence[int], a: Sequence[float], det: Sequence[int],
                  pitch: Sequence[float], nviews: int, sid: float, sdd: float,
                  arc_deg: float = 360.0) -> Geometry:
    nx, ny, nz = (int(v) for v in n)
    ax, ay, az = (float(v) for v in a)
    nu, nv = int(det[0]), int(det[1])
    pu, pv = float(pitch[0]), float(pitch[1])
    P = circular_pmats(nviews, sid, sdd, nu, nv, pu, pv, arc_deg)
    return Geometry(nx, ny, nz, ax, ay, az, nu, nv, pu, pv, P)


# The benchmark workloads. Each is a synthetic stand-in with the shapes of the
# cone-beam problems the projector is evaluated on.
WORKLOADS = {
    # 32^3 @ 1 mm, 24 views / 360 deg, SID 750 / SDD 1200, 64x48 @ 0.8 mm
    "cvp32": dict(n=(32, 32, 32), a=(1.0, 1.0, 1.0), det=(64, 48), pitch=(0.8, 0.8),
                  nviews=24, sid=750.0, sdd=1200.0, arc_deg=360.0,
                  phantom=dict(count=6, semi=(3.0, 12.0), mu=(0.005, 0.02))),
    # 256^3 @ 0.5 mm, 248 views / 200 deg short scan, SID 750 / SDD 1200, 616x480 @ 0.616 mm
    "cvp256": dict(n=(256, 256, 256), a=(0.5, 0.5, 0.5), det=(616, 480), pitch=(0.616, 0.616),
                   nviews=248, sid=750.0, sdd=1200.0, arc_deg=200.0,
                   phantom=dict(count=40, semi=(3.0, 30.0), mu=(0.0, 0.03))),
    # 512^3 @ 0.25 mm, 496 views / 360 deg, SID 400 / SDD 600, 1232x960 @ 0.154 mm
    "cvp512": dict(n=(512, 512, 512), a=(0.25, 0.25, 0.25), det=(1232, 960), pitch=(0.154, 0.154),
                   nviews=496, sid=400.0, sdd=600.0, arc_deg=360.0,
                   phantom=dict(count=40, semi=(3.0, 30.0), mu=(0.0, 0.03))),
    # same grid with a 0.455 mm pitch: half cone angle about 20 degrees
    "cvp512wide": dict(n=(512, 512, 512), a=(0.25, 0.25, 0.25), det=(1232, 960), pitch=(0.455, 0.455),
                       nviews=496, sid=400.0, sdd=600.0, arc_deg=360.0,
                       phantom=dict(count=40, semi=(3.0, 30.0), mu=(0.0, 0.03))),
    # Table I geometry of the paper: 512x512x128 @ 0.5 mm, 720 views, SID 541 / SDD 949, 512x512 @ 1 mm
    "long2010": dict(n=(512, 512, 128), a=(0.5, 0.5, 0.5), det=(512, 512), pitch=(1.0, 1.0),
                     nviews=720, sid=541.0, sdd=949.0, arc_deg=360.0,
                     phantom=dict(count=40, semi=(3.0, 30.0), mu=(0.0, 0.03))),
    # Table II geometry of the paper: 256^3 @ 0.5 mm, 100 views / 198 deg, SID 750 / SDD 1000, 1280x960 @ 0.25 mm
    "pfeiffer2021": dict(n=(256, 256, 256), a=(0.5, 0.5, 0.5), det=(1280, 960), pitch=(0.25, 0.25),
                         nviews=100, sid=750.0, sdd=1000.0, arc_deg=198.0,
                         phantom=dict(count=40, semi=(3.0, 30.0), mu=(0.0, 0.03))),
    # CGLS reconstruction problem: 128^3 @ 0.5 mm, 180 views / 360 deg, SID 750 / SDD 1200,
    # 256x192 detector @ 0.8 mm; data with Poisson noise at 1e5 photons per pixel
    "cgls128": dict(n=(128, 128, 128), a=(0.5, 0.5, 0.5), det=(256, 192), pitch=(0.8, 0.8),
                    nviews=180, sid=750.0, sdd=1200.0, arc_deg=360.0,
                    phantom=dict(count=20, semi=(3.0, 16.0), mu=(0.005, 0.02))),
}

WORKLOAD_SEEDS = {"cvp32": 1001, "cvp256": 1002, "cvp512": 1003, "cvp512wide": 1003,
                  "long2010": 1011, "pfeiffer2021": 1012, "cgls128": 1013}


def workload_geometry(name: str) -> Geometry:
    w = WORKLOADS[name]
    return make_geometry(w["n"], w["a"], w["det"], w["pitch"], w["nviews"], w["sid"],
                         w["sdd"], w["arc_deg"])


# --------------------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Ellipsoid:
    centre: np.ndarray   # (3,) mm
    semi: np.ndarray     # (3,) mm
    rot: np.ndarray      # (3, 3) rotation, columns = ellipsoid axes in world
    mu: float            # mm^-1, added inside


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    # uniform random unit quaternion (Shoemake) -> rotation matrix
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_ellipsoids(seed: int, count: int, box_edge: float, semi=(3.0, 12.0),
                      mu=(0.005, 0.02)) -> list[Ellipsoid]:
    """Seeded ellipsoids: centres uniform in a ball of radius 0.35 * box_edge,
    uniform random orientation, semi-axes and attenuation uniform in the ranges."""
    rng = np.random.default_rng(seed)
    out = []
    rball = 0.35 * box_edge
    for _ in range(count):
        while True:
            c = rng.uniform(-1.0, 1.0, 3)
            if c @ c <= 1.0:
                break
        centre = c * rball
        semi_ax = rng.uniform(semi[0], semi[1], 3)
        rot = _random_rotation(rng)
        m = float(rng.uniform(mu[0], mu[1]))
        out.append(Ellipsoid(centre, semi_ax, rot, m))
    return out


def voxelize(geom: Geometry, ellipsoids: Sequence[Ellipsoid], device="cpu"):
    """Additive ellipsoid phantom sampled at voxel centres -> torch float32 [nz, ny, nx].

    Each ellipsoid is evaluated only inside its axis-aligned bounding box, slab
    by slab, so 512^3 volumes are built in seconds on a GPU.
    """
    import torch

    nx, ny, nz = geom.nx, geom.ny, geom.nz
    a = (geom.ax, geom.ay, geom.az)
    n = (nx, ny, nz)
    x0 = [(-n[d] * a[d] + a[d]) / 2.0 for d in range(3)]
    vol = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    for e in ellipsoids:
        # axis-aligned half extents of the rotated ellipsoid
        half = np.sqrt(((e.rot * e.semi[None, :]) ** 2).sum(axis=1))
        lo = [max(0, int(math.floor((e.centre[d] - half[d] - x0[d]) / a[d]))) for d in range(3)]
        hi = [min(n[d] - 1, int(math.ceil((e.centre[d] + half[d] - x0[d]) / a[d]))) for d in range(3)]
        if any(lo[d] > hi[d] for d in range(3)):
            continue
        # quadratic form: (x-c)^T Q (x-c) <= 1, Q = R diag(1/s^2) R^T
        Q = e.rot @ np.diag(1.0 / e.semi ** 2) @ e.rot.T
        Qt = torch.tensor(Q, dtype=torch.float64, device=device)
        xs = torch.arange(lo[0], hi[0] + 1, device=device, dtype=torch.float64) * a[0] + x0[0] - e.centre[0]
        ys = torch.arange(lo[1], hi[1] + 1, device=device, dtype=torch.float64) * a[1] + x0[1] - e.centre[1]
        step = max(1, int(2 ** 24 // max(1, xs.numel() * ys.numel())))
        for k0 in range(lo[2], hi[2] + 1, step):
            k1 = min(hi[2] + 1, k0 + step)
            zs = torch.arange(k0, k1, device=device, dtype=torch.float64) * a[2] + x0[2] - e.centre[2]
            Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
            q = (Qt[0, 0] * X * X + Qt[1, 1] * Y * Y + Qt[2, 2] * Z * Z
                 + 2 * Qt[0, 1] * X * Y + 2 * Qt[0, 2] * X * Z + 2 * Qt[1, 2] * Y * Z)
            vol[k0:k1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += (q <= 1.0).to(torch.float32) * e.mu
    return vol


def workload_phantom(name: str, device="cpu"):
    w = WORKLOADS[name]
    geom = workload_geometry(name)
    ph = w["phantom"]
    edge = geom.nx * geom.ax
    ells = random_ellipsoids(WORKLOAD_SEEDS[name], ph["count"], edge, ph["semi"], ph["mu"])
    return voxelize(geom, ells, device=device)


def perfusion_frames(geom: Geometry, seed: int, frames: int = 8, device="cpu"):
    """A batch of perfusion-like time frames: one static ellipsoid phantom plus five
    vessel ellipsoids whose attenuation follows seeded Gaussian bolus curves
    mu(t) = base + amp * exp(-(t - t0)^2 / (2 sigma^2)).  -> float32 [frames, nz, ny, nx]"""
    import torch

    rng = np.random.default_rng(seed)
    edge = geom.nx * geom.ax
    static = voxelize(geom, random_ellipsoids(seed, 20, edge, (2.0, 0.25 * edge), (0.0, 0.02)),
                      device=device)
    vessels = random_ellipsoids(seed + 1, 5, edge, (1.0, 0.08 * edge), (1.0, 1.0))
    masks = [voxelize(geom, [v], device=device) for v in vessels]
    amp = rng.uniform(0.005, 0.03, 5)
    t0 = rng.uniform(0.25, 0.75, 5) * frames
    sig = rng.uniform(0.1, 0.3, 5) * frames
    out = torch.empty((frames,) + geom.vol_shape, dtype=torch.float32, device=device)
    for f in range(frames):
        fr = static.clone()
        for v in range(5):
            fr += masks[v] * float(amp[v] * math.exp(-((f - t0[v]) ** 2) / (2 * sig[v] ** 2)))
        out[f] = fr
    return out


def poisson_log_data(clean, photons: float, seed: int):
    """Noisy line integrals from noise-free ones (Beer-Lambert with Poisson counts):
    b = -ln(max(N, 1) / I0), N ~ Poisson(I0 exp(-clean)), seeded; same device as `clean`."""
    import torch

    g = torch.Generator(device=clean.device)
    g.manual_seed(seed)
    lam = photons * torch.exp(-clean.double())
    counts = torch.poisson(lam, generator=g).clamp_(min=1.0)
    return (-torch.log(counts / photons)).to(torch.float32)


def uniform_projections(shape, seed: int, device="cpu"):
    """Projection-side input for the adjoint: U[0,1) float32, seeded."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.rand(shape, generator=g, dtype=torch.float32, device=device)


def uniform_volume(shape, seed: int, device="cpu"):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.rand(shape, generator=g, dtype=torch.float32, device=device)
