"""kct_project_static: the forward projection for callers that must not allocate device
memory (code inside another framework's memory pool or an allocator-free runtime). It keeps
its scratch in a fixed array compiled into the library instead of a plan's workspace.

Checked against kct_project through the C ABI, on two calls in a row (the shared array keeps
the previous call's contents, so the second call shows that what must start at zero is
cleared). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2110_09841_b300 import inputs
from paper_2110_09841_b300.kct import DetectorDesc, Projector, VolumeDesc, load

pytestmark = pytest.mark.gpu

TOL = 1e-4


def call_static(lib, g, variant, scaling, x, out, accumulate=0):
    vol = VolumeDesc(g.nx, g.ny, g.nz, g.ax, g.ay, g.az)
    det = DetectorDesc(g.nu, g.nv, g.pu, g.pv)
    pm = np.ascontiguousarray(g.pmats, dtype=np.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.kct_project_static(ctypes.byref(vol), ctypes.byref(det), pm.ctypes.data_as(ctypes.c_void_p),
                                  g.nviews, variant, scaling, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), accumulate, stream)


def static_error(lib):
    code = ctypes.c_int32(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.kct_project_static_device_error(ctypes.byref(code), stream) == 0
    return int(code.value)


def assert_close_per_view(g, o, tol=TOL):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    for view in range(o.shape[0]):
        mx = np.abs(o[view]).max()
        d = np.abs(g[view] - o[view])
        assert d.max() <= tol * mx
        big = np.abs(o[view]) >= 1e-3 * mx
        assert (d[big] / np.abs(o[view][big])).max() <= tol


@pytest.mark.parametrize("variant,vname", [(0, "exact"), (1, "relaxed")])
def test_static_matches_planned_projection(variant, vname):
    lib = load()
    g = inputs.workload_geometry("cvp32")
    x = inputs.workload_phantom("cvp32").cuda()
    ref = Projector(g, vname, "cos").project(x)
    for _ in range(2):
        out = torch.full(g.proj_shape, 7.0, dtype=torch.float32, device="cuda")
        assert call_static(lib, g, variant, 0, x, out) == 0, lib.kct_last_error_message()
        assert static_error(lib) == 0
        torch.cuda.synchronize()
        assert_close_per_view(out.cpu().numpy(), ref.cpu().numpy())
    # accumulate adds to the output
    out = torch.full(g.proj_shape, 0.5, dtype=torch.float32, device="cuda")
    assert call_static(lib, g, variant, 0, x, out, accumulate=1) == 0
    assert static_error(lib) == 0
    torch.cuda.synchronize()
    assert_close_per_view(out.cpu().numpy() - 0.5, ref.cpu().numpy())


def test_static_rejects_requests_beyond_its_array():
    lib = load()
    g = inputs.workload_geometry("cvp256")          # 616 x 480 x 248 pixels: above the limit
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    assert call_static(lib, g, 0, 0, x, out) == 6
    assert b"8388608" in lib.kct_last_error_message()


@pytest.mark.parametrize("variant", [0, 1])
def test_static_reports_a_skipped_footprint(variant):
    """A 1 mm voxel seen through 0.0002 mm wide pixels covers about 8000 detector columns,
    more than the kernel's bound (4096): the voxel is skipped, the array's error word says
    so, and the next call starts from a cleared word."""
    lib = load()
    P = inputs.circular_pmats(1, 400.0, 600.0, 9000, 16, 0.0002, 0.25)
    g = inputs.Geometry(1, 1, 1, 1.0, 1.0, 1.0, 9000, 16, 0.0002, 0.25, P)
    x = torch.ones(g.vol_shape, dtype=torch.float32, device="cuda")
    out = torch.zeros(g.proj_shape, dtype=torch.float32, device="cuda")
    assert call_static(lib, g, variant, 0, x, out) == 0, lib.kct_last_error_message()
    assert static_error(lib) == 1
    assert float(out.abs().max()) == 0.0
    g32 = inputs.workload_geometry("cvp32")
    x32 = inputs.workload_phantom("cvp32").cuda()
    out32 = torch.zeros(g32.proj_shape, dtype=torch.float32, device="cuda")
    assert call_static(lib, g32, variant, 0, x32, out32) == 0
    assert static_error(lib) == 0
