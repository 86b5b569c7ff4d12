"""ctypes wrapper of the FP64 CPU oracle (oracle.c) -- test infrastructure only.

Every function takes numpy arrays and a geometry description and returns float64
results. See oracle.c for the paper passages each computation follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EXACT, RELAXED = 0, 1
TRUTH = 2          # project_pixels only: the exact pixel value the scaled projection approximates
SCALE_COS, SCALE_EXACT = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-D_GNU_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            grid = [I, I, I, D, D, D, I, I]
            lib.or_num_threads.restype = I
            lib.or_set_num_threads.argtypes = [I]
            lib.or_source.argtypes = [P, P]
            lib.or_source.restype = I
            lib.or_box_pixel.argtypes = [P, P, P, D, D, I, P]
            lib.or_box_pixel.restype = I
            lib.or_box_clip.argtypes = [P, P, P, I, P]
            lib.or_box_clip.restype = I
            lib.or_box_inv_r2.argtypes = [P, P, P, I]
            lib.or_box_inv_r2.restype = D
            lib.or_pixel_factor.argtypes = [P, D, D, I]
            lib.or_pixel_factor.restype = D
            lib.or_pixel_solid_angle.argtypes = [P, D, D]
            lib.or_pixel_solid_angle.restype = D
            lib.or_project.argtypes = grid + [P, I, I, I, P, P]
            lib.or_project.restype = I
            lib.or_backproject.argtypes = grid + [P, I, I, I, P, P]
            lib.or_backproject.restype = I
            lib.or_backproject_voxels.argtypes = grid + [P, I, I, I, P, P, I, P]
            lib.or_backproject_voxels.restype = I
            lib.or_project_pixels.argtypes = grid + [P, I, I, I, P, P, I, P]
            lib.or_project_pixels.restype = I
            lib.or_ray_pixel.argtypes = [I, I, I, D, D, D, P, P, D, D, I, I]
            lib.or_ray_pixel.restype = D
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _grid(g):
    return (g.nx, g.ny, g.nz, g.ax, g.ay, g.az, g.nu, g.nv)


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(int(n))


def source(P) -> np.ndarray:
    P = _f64(P).reshape(12)
    out = np.zeros(3)
    if _load().or_source(_ptr(P), _ptr(out)) != 0:
        raise ValueError("singular projection matrix")
    return out


def box_pixel(P, lo, hi, u: float, v: float, quad_level: int = -1) -> dict:
    """Pair quantities for an arbitrary box and pixel (u, v)."""
    P = _f64(P).reshape(12)
    lo, hi = _f64(lo), _f64(hi)
    out = np.zeros(7)
    if _load().or_box_pixel(_ptr(P), _ptr(lo), _ptr(hi), float(u), float(v), int(quad_level), _ptr(out)):
        raise ValueError("singular projection matrix")
    return dict(V=out[0], c=out[1:4].copy(), W=out[4], J=out[5], Wrel=out[6])


def box_clip(lo, hi, planes) -> tuple[float, np.ndarray]:
    """Volume and centroid of box [lo, hi] intersected with half-spaces n.x + d >= 0."""
    lo, hi = _f64(lo), _f64(hi)
    planes = _f64(planes).reshape(-1, 4)
    out = np.zeros(4)
    _load().or_box_clip(_ptr(lo), _ptr(hi), _ptr(planes), planes.shape[0], _ptr(out))
    return float(out[0]), out[1:4].copy()


def box_inv_r2(lo, hi, s, level: int = 0) -> float:
    lo, hi, s = _f64(lo), _f64(hi), _f64(s)
    return float(_load().or_box_inv_r2(_ptr(lo), _ptr(hi), _ptr(s), int(level)))


def pixel_factor(P, u: float, v: float, scaling: int = SCALE_COS) -> float:
    P = _f64(P).reshape(12)
    return float(_load().or_pixel_factor(_ptr(P), float(u), float(v), int(scaling)))


def pixel_solid_angle(P, u: float, v: float) -> float:
    P = _f64(P).reshape(12)
    return float(_load().or_pixel_solid_angle(_ptr(P), float(u), float(v)))


def project(geom, x, variant: int = EXACT, scaling: int = SCALE_COS) -> np.ndarray:
    """b = A x over the whole detector stack -> float64 [nviews, nv, nu]."""
    x = _f64(x).reshape(geom.vol_shape)
    P = _f64(geom.pmats)
    b = np.zeros(geom.proj_shape)
    rc = _load().or_project(*_grid(geom), _ptr(P), geom.nviews, int(variant), int(scaling), _ptr(x), _ptr(b))
    if rc:
        raise ValueError(f"oracle project failed ({rc})")
    return b


def backproject(geom, y, variant: int = EXACT, scaling: int = SCALE_COS) -> np.ndarray:
    """x = A^T y over the whole volume -> float64 [nz, ny, nx]."""
    y = _f64(y).reshape(geom.proj_shape)
    P = _f64(geom.pmats)
    x = np.zeros(geom.vol_shape)
    rc = _load().or_backproject(*_grid(geom), _ptr(P), geom.nviews, int(variant), int(scaling), _ptr(y), _ptr(x))
    if rc:
        raise ValueError(f"oracle backproject failed ({rc})")
    return x


def project_pixels(geom, x, pix, variant: int = EXACT, scaling: int = SCALE_COS) -> np.ndarray:
    """(A x) at selected pixels; pix int array [count, 3] of (view, v, u).
    variant TRUTH gives the value the projection approximates, with no ray sampling: for the
    exact scaling the solid-angle average of the pixel's line integrals (pair weights
    J = int_cut r^-2 dV), for the cos scaling their area average over the pixel (pair weights
    |det M| int_cut |x - s| / |w|^3 dV, w the depth along the detector normal)."""
    x = _f64(x).reshape(geom.vol_shape)
    P = _f64(geom.pmats)
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(pix.shape[0])
    rc = _load().or_project_pixels(*_grid(geom), _ptr(P), geom.nviews, int(variant), int(scaling),
                                   _ptr(x), _ptr(pix), pix.shape[0], _ptr(out))
    if rc:
        raise ValueError(f"oracle project_pixels failed ({rc})")
    return out


def backproject_voxels(geom, y, vox, variant: int = EXACT, scaling: int = SCALE_COS) -> np.ndarray:
    """(A^T y) at selected voxels; vox int array [count, 3] of (k, j, i)."""
    y = _f64(y).reshape(geom.proj_shape)
    P = _f64(geom.pmats)
    vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(vox.shape[0])
    rc = _load().or_backproject_voxels(*_grid(geom), _ptr(P), geom.nviews, int(variant), int(scaling),
                                       _ptr(y), _ptr(vox), vox.shape[0], _ptr(out))
    if rc:
        raise ValueError(f"oracle backproject_voxels failed ({rc})")
    return out


def ray_pixel(geom, x, view: int, u: float, v: float, K: int, weighting: int = 0) -> float:
    """Ray-integration value of pixel (u, v): K x K rays with exact path lengths.
    weighting 0 = area average, 1 = solid-angle weighted average."""
    x = _f64(x).reshape(geom.vol_shape)
    P = _f64(geom.pmats[view]).reshape(12)
    return float(_load().or_ray_pixel(geom.nx, geom.ny, geom.nz, geom.ax, geom.ay, geom.az,
                                      _ptr(P), _ptr(x), float(u), float(v), int(K), int(weighting)))
