"""Python binding of libkct (the cutting voxel projector C ABI, include/kct.h).

Argument marshalling only: every step of the projector runs in the CUDA library.
Tensors must be contiguous float32 CUDA tensors; the work is enqueued on the current
torch CUDA stream unless another stream is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkct.so")

EXACT, RELAXED = 0, 1
SCALE_COS, SCALE_EXACT = 0, 1
_VARIANTS = {"exact": EXACT, "relaxed": RELAXED, EXACT: EXACT, RELAXED: RELAXED}
_SCALINGS = {"cos": SCALE_COS, "exact": SCALE_EXACT, SCALE_COS: SCALE_COS, SCALE_EXACT: SCALE_EXACT}

STATUS = {0: "KCT_OK", 1: "KCT_ERR_INVALID_ARG", 2: "KCT_ERR_GEOMETRY", 3: "KCT_ERR_CUDA",
          4: "KCT_ERR_OOM", 5: "KCT_ERR_DEVICE_CHECK", 6: "KCT_ERR_UNSUPPORTED"}

EXPORTED = ["kct_plan_create", "kct_plan_destroy", "kct_project", "kct_backproject",
            "kct_pixel_factors", "kct_count_pairs", "kct_last_device_error", "kct_status_string",
            "kct_last_error_message", "kct_version", "kct_project_static", "kct_project_batch",
            "kct_backproject_batch", "kct_cgls_workspace_bytes", "kct_cgls", "kct_plan_autotune",
            "kct_plan_set_view_chunk", "kct_plan_get_view_chunk", "kct_siddon_project",
            "kct_project_static_device_error"]


class KctError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class VolumeDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("az", ctypes.c_double)]


class DetectorDesc(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("pu", ctypes.c_double), ("pv", ctypes.c_double)]


class CglsReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("normal_residual", ctypes.c_double), ("data_residual", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load libkct.so (or the library named by $KCT_LIB). Raises if it is missing: there is
    no fallback path."""
    global _lib
    if _lib is None:
        p = path or os.environ.get("KCT_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libkct.so not built ({p}); run `python -m paper_2110_09841_b300.build`")
        lib = ctypes.CDLL(p)
        V, I32, I = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
        lib.kct_plan_create.argtypes = [ctypes.POINTER(V), ctypes.POINTER(VolumeDesc), ctypes.POINTER(DetectorDesc),
                                        V, I32, I, I]
        lib.kct_plan_create.restype = I
        lib.kct_plan_destroy.argtypes = [V]
        lib.kct_plan_destroy.restype = I
        lib.kct_project.argtypes = [V, V, V, I32, V]
        lib.kct_project.restype = I
        lib.kct_backproject.argtypes = [V, V, V, I32, V]
        lib.kct_backproject.restype = I
        lib.kct_project_batch.argtypes = [V, V, I32, V, I32, V]
        lib.kct_project_batch.restype = I
        lib.kct_backproject_batch.argtypes = [V, V, I32, V, I32, V]
        lib.kct_backproject_batch.restype = I
        lib.kct_pixel_factors.argtypes = [V, V, V]
        lib.kct_pixel_factors.restype = I
        lib.kct_count_pairs.argtypes = [V, ctypes.POINTER(ctypes.c_uint64), V]
        lib.kct_count_pairs.restype = I
        lib.kct_last_device_error.argtypes = [V, ctypes.POINTER(I32), V]
        lib.kct_last_device_error.restype = I
        lib.kct_status_string.argtypes = [I]
        lib.kct_status_string.restype = ctypes.c_char_p
        lib.kct_last_error_message.argtypes = []
        lib.kct_last_error_message.restype = ctypes.c_char_p
        lib.kct_version.argtypes = []
        lib.kct_version.restype = I32
        lib.kct_project_static.argtypes = [ctypes.POINTER(VolumeDesc), ctypes.POINTER(DetectorDesc), V, I32, I, I,
                                           V, V, I32, V]
        lib.kct_project_static.restype = I
        lib.kct_project_static_device_error.argtypes = [ctypes.POINTER(I32), V]
        lib.kct_project_static_device_error.restype = I
        lib.kct_siddon_project.argtypes = [V, V, V, I32, I32, V]
        lib.kct_siddon_project.restype = I
        lib.kct_plan_autotune.argtypes = [V, V, V, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_float), V]
        lib.kct_plan_autotune.restype = I
        lib.kct_plan_set_view_chunk.argtypes = [V, I32]
        lib.kct_plan_set_view_chunk.restype = I
        lib.kct_plan_get_view_chunk.argtypes = [V, ctypes.POINTER(I32)]
        lib.kct_plan_get_view_chunk.restype = I
        lib.kct_cgls_workspace_bytes.argtypes = [V]
        lib.kct_cgls_workspace_bytes.restype = ctypes.c_size_t
        lib.kct_cgls.argtypes = [V, V, V, V, I32, I32, ctypes.c_double, V, ctypes.c_size_t, V, V,
                                 ctypes.POINTER(CglsReport), V]
        lib.kct_cgls.restype = I
        _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        lib = load()
        raise KctError(status, lib.kct_last_error_message().decode() or lib.kct_status_string(status).decode())


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, shape, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape[-len(shape):]) != tuple(shape) or t.numel() != int(np.prod(shape)):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Projector:
    """CVP operator A for one geometry: project(x) = A x, backproject(y) = A^T y.

    geom: paper_2110_09841_b300.inputs.Geometry (voxel grid, detector, float64 [V,3,4] matrices).
    variant: "exact" | "relaxed";  scaling: "cos" | "exact".
    The plan lives on the CUDA device current at construction (`self.device`).
    """

    def __init__(self, geom, variant="exact", scaling="cos"):
        import torch

        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.geom = geom
        self.variant = _VARIANTS[variant]
        self.scaling = _SCALINGS[scaling]
        vol = VolumeDesc(geom.nx, geom.ny, geom.nz, geom.ax, geom.ay, geom.az)
        det = DetectorDesc(geom.nu, geom.nv, geom.pu, geom.pv)
        self._pm = np.ascontiguousarray(geom.pmats, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(self.lib.kct_plan_create(ctypes.byref(h), ctypes.byref(vol), ctypes.byref(det),
                                        self._pm.ctypes.data_as(ctypes.c_void_p), int(geom.nviews),
                                        self.variant, self.scaling))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.kct_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def project(self, x, out=None, accumulate=False, stream=None):
        import torch

        g = self.geom
        xp = _dev_ptr(x, g.vol_shape, "x")
        if out is None:
            out = torch.empty(g.proj_shape, dtype=torch.float32, device=x.device)
        _check(self.lib.kct_project(self._h, xp, _dev_ptr(out, g.proj_shape, "out"), int(bool(accumulate)),
                                    _stream_handle(stream)))
        return out

    def backproject(self, y, out=None, accumulate=False, stream=None):
        import torch

        g = self.geom
        yp = _dev_ptr(y, g.proj_shape, "y")
        if out is None:
            out = torch.empty(g.vol_shape, dtype=torch.float32, device=y.device)
        _check(self.lib.kct_backproject(self._h, yp, _dev_ptr(out, g.vol_shape, "out"), int(bool(accumulate)),
                                        _stream_handle(stream)))
        return out

    def project_batch(self, x, out=None, accumulate=False, stream=None):
        """x: [B, nz, ny, nx] -> [B, nviews, nv, nu], one launch."""
        import torch

        g = self.geom
        if x.dim() != 4:
            raise ValueError("x must be [B, nz, ny, nx]")
        B = int(x.shape[0])
        xp = _dev_ptr(x, (B,) + g.vol_shape, "x")
        if out is None:
            out = torch.empty((B,) + g.proj_shape, dtype=torch.float32, device=x.device)
        _check(self.lib.kct_project_batch(self._h, xp, B, _dev_ptr(out, (B,) + g.proj_shape, "out"),
                                          int(bool(accumulate)), _stream_handle(stream)))
        return out

    def backproject_batch(self, y, out=None, accumulate=False, stream=None):
        """y: [B, nviews, nv, nu] -> [B, nz, ny, nx], one launch."""
        import torch

        g = self.geom
        if y.dim() != 4:
            raise ValueError("y must be [B, nviews, nv, nu]")
        B = int(y.shape[0])
        yp = _dev_ptr(y, (B,) + g.proj_shape, "y")
        if out is None:
            out = torch.empty((B,) + g.vol_shape, dtype=torch.float32, device=y.device)
        _check(self.lib.kct_backproject_batch(self._h, yp, B, _dev_ptr(out, (B,) + g.vol_shape, "out"),
                                              int(bool(accumulate)), _stream_handle(stream)))
        return out

    def autotune(self, x, scratch=None, stream=None):
        """Pick the forward kernel's views per block by timing (kct_plan_autotune) on volume x.
        Returns (chunk, forward ms over the first min(nviews, 64) views)."""
        import torch

        g = self.geom
        xp = _dev_ptr(x, g.vol_shape, "x")
        if scratch is None:
            scratch = torch.empty(g.proj_shape, dtype=torch.float32, device=x.device)
        c = ctypes.c_int32(0)
        ms = ctypes.c_float(0.0)
        _check(self.lib.kct_plan_autotune(self._h, xp, _dev_ptr(scratch, g.proj_shape, "scratch"), ctypes.byref(c),
                                          ctypes.byref(ms), _stream_handle(stream)))
        return int(c.value), float(ms.value)

    @property
    def view_chunk(self) -> int:
        c = ctypes.c_int32(0)
        _check(self.lib.kct_plan_get_view_chunk(self._h, ctypes.byref(c)))
        return int(c.value)

    @view_chunk.setter
    def view_chunk(self, chunk: int):
        _check(self.lib.kct_plan_set_view_chunk(self._h, int(chunk)))

    def cgls_workspace(self):
        """Device scratch for cgls(): a uint8 CUDA tensor of kct_cgls_workspace_bytes."""
        import torch

        return torch.empty(int(self.lib.kct_cgls_workspace_bytes(self._h)), dtype=torch.uint8, device=self.device)

    def cgls(self, b, x0=None, max_iter=100, tol=1e-3, out=None, workspace=None, atb=None, stream=None):
        """CGLS for min |b - A x| (kct_cgls): from x0 (warm start) or from 0, until the
        normal-equation residual |A^T(b - A x)| / |A^T b| <= tol or max_iter steps.
        atb: optional A^T b already at hand (saves the solve one backprojection).
        Returns (x, info) with info = dict(iterations, converged, normal, data); normal and
        data are the residual histories (entry k after k steps)."""
        import torch

        g = self.geom
        bp = _dev_ptr(b, g.proj_shape, "b")
        if out is None:
            out = torch.empty(g.vol_shape, dtype=torch.float32, device=b.device)
        xp = _dev_ptr(out, g.vol_shape, "out")
        if x0 is not None:
            _dev_ptr(x0, g.vol_shape, "x0")
            if x0.data_ptr() != out.data_ptr():
                out.copy_(x0)
        if workspace is None:
            workspace = self.cgls_workspace()
        hn = np.zeros(max_iter + 1)
        hd = np.zeros(max_iter + 1)
        rep = CglsReport()
        ap = _dev_ptr(atb, g.vol_shape, "atb") if atb is not None else None
        _check(self.lib.kct_cgls(self._h, bp, xp, ap, int(x0 is not None), int(max_iter), float(tol),
                                 ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel()),
                                 hn.ctypes.data_as(ctypes.c_void_p), hd.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(rep), _stream_handle(stream)))
        k = int(rep.iterations)
        return out, dict(iterations=k, converged=bool(rep.converged), normal=hn[:k + 1].copy(),
                         data=hd[:k + 1].copy())

    def siddon(self, x, K=8, weighted=False, out=None, stream=None):
        """Ray-driven comparator: K x K rays per pixel, exact path lengths (kct_siddon_project)."""
        import torch

        g = self.geom
        xp = _dev_ptr(x, g.vol_shape, "x")
        if out is None:
            out = torch.empty(g.proj_shape, dtype=torch.float32, device=x.device)
        _check(self.lib.kct_siddon_project(self._h, xp, _dev_ptr(out, g.proj_shape, "out"), int(K), int(bool(weighted)),
                                           _stream_handle(stream)))
        return out

    def pixel_factors(self, stream=None):
        import torch

        out = torch.empty(self.geom.proj_shape, dtype=torch.float32, device=self.device)
        _check(self.lib.kct_pixel_factors(self._h, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def count_pairs(self, stream=None) -> int:
        c = ctypes.c_uint64(0)
        _check(self.lib.kct_count_pairs(self._h, ctypes.byref(c), _stream_handle(stream)))
        return int(c.value)

    def device_error(self, stream=None) -> int:
        c = ctypes.c_int32(0)
        _check(self.lib.kct_last_device_error(self._h, ctypes.byref(c), _stream_handle(stream)))
        return int(c.value)
