"""The C ABI library: it builds, loads, exports what include/kct.h declares, and rejects
invalid arguments and geometry before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2110_09841_b300 import build, inputs, kct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return kct.load()


def declared_functions(header="kct.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kct_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(kct.EXPORTED)
    for n in names:
        assert hasattr(lib, n), n


def test_conv_library_exports_every_declared_symbol():
    from paper_2110_09841_b300 import conv

    build.build()
    clib = conv.load()
    names = declared_functions("kct_conv.h")
    assert set(names) == {"kct_conv3d_fwd", "kct_conv3d_wgrad", "kct_conv_last_error"}
    for n in names:
        assert hasattr(clib, n), n
    # invalid descriptors are rejected before any launch
    d = conv.ConvDesc(1, 4, 8, 16, 24, 16)               # cin not a multiple of 16
    assert clib.kct_conv3d_fwd(ctypes.byref(d), None, None, None, None, 0, None, None) == 6
    d = conv.ConvDesc(1, 4, 8, 16, 16, 16)
    assert clib.kct_conv3d_fwd(ctypes.byref(d), None, None, None, None, 0, None, None) == 1
    assert clib.kct_conv3d_fwd(None, None, None, None, None, 0, None, None) == 1


def test_version_and_status_strings(lib):
    assert lib.kct_version() == 101
    for s in range(7):
        assert lib.kct_status_string(s).decode()
    assert lib.kct_status_string(99).decode() == "unknown status"


def _create(lib, geom, variant=0, scaling=0, nviews=None, vol=None, det=None):
    v = vol or kct.VolumeDesc(geom.nx, geom.ny, geom.nz, geom.ax, geom.ay, geom.az)
    d = det or kct.DetectorDesc(geom.nu, geom.nv, geom.pu, geom.pv)
    pm = np.ascontiguousarray(geom.pmats, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib.kct_plan_create(ctypes.byref(h), ctypes.byref(v), ctypes.byref(d),
                             pm.ctypes.data_as(ctypes.c_void_p),
                             geom.nviews if nviews is None else nviews, variant, scaling)
    return st, h


def test_rejects_invalid_arguments(lib):
    g = inputs.workload_geometry("cvp32")
    assert _create(lib, g, nviews=0)[0] == 1
    assert _create(lib, g, variant=7)[0] == 1
    assert _create(lib, g, scaling=-1)[0] == 1
    assert _create(lib, g, vol=kct.VolumeDesc(0, 32, 32, 1.0, 1.0, 1.0))[0] == 1
    assert _create(lib, g, vol=kct.VolumeDesc(32, 32, 32, 1.0, -1.0, 1.0))[0] == 1
    assert _create(lib, g, det=kct.DetectorDesc(64, 0, 0.8, 0.8))[0] == 1
    h = ctypes.c_void_p()
    assert lib.kct_plan_create(ctypes.byref(h), None, None, None, 1, 0, 0) == 1
    assert lib.kct_plan_create(None, None, None, None, 1, 0, 0) == 1
    # calls with a null plan fail cleanly
    assert lib.kct_project(None, None, None, 0, None) == 1
    assert lib.kct_backproject(None, None, None, 0, None) == 1
    assert lib.kct_plan_destroy(None) == 0
    assert lib.kct_project_batch(None, None, 1, None, 0, None) == 1
    assert lib.kct_backproject_batch(None, None, 1, None, 0, None) == 1
    assert lib.kct_plan_set_view_chunk(None, 4) == 1
    assert lib.kct_plan_autotune(None, None, None, None, None, None) == 1
    assert lib.kct_cgls_workspace_bytes(None) == 0
    assert lib.kct_cgls(None, None, None, None, 0, 1, 1e-3, None, 0, None, None, None, None) == 1
    assert lib.kct_siddon_project(None, None, None, 8, 0, None) == 1
    assert lib.kct_plan_get_view_chunk(None, None) == 1


def test_rejects_geometry_outside_the_arrangement(lib):
    g = inputs.workload_geometry("cvp32")
    bad = g.pmats.copy()
    bad[3, 0, 2] = 5.0                                 # u depends on x3
    st, _ = _create(lib, inputs.Geometry(**{**g.__dict__, "pmats": bad}))
    assert st == 2
    assert b"view 3" in lib.kct_last_error_message()
    bad = g.pmats.copy()
    bad[1, 1, :3] += 0.3 * bad[1, 0, :3] / np.linalg.norm(bad[1, 0, :3]) * np.linalg.norm(bad[1, 1, :3]) \
        * np.array([1.0, 1.0, 0.0])                    # skewed rows
    st, _ = _create(lib, inputs.Geometry(**{**g.__dict__, "pmats": bad}))
    assert st == 2
    # source inside the volume
    inside = inputs.circular_pmats(4, 10.0, 40.0, 64, 48, 0.8, 0.8)
    st, _ = _create(lib, inputs.Geometry(**{**g.__dict__, "pmats": inside}))
    assert st == 2
    bad = g.pmats.copy()
    bad[0, 2, 1] = np.nan
    st, _ = _create(lib, inputs.Geometry(**{**g.__dict__, "pmats": bad}))
    assert st == 2
    # the paper's arrangement with the opposite v orientation and a scaled matrix is fine
    ok = inputs.circular_pmats(4, 750.0, 1200.0, 64, 48, 0.8, 0.8) * -2.5
    ok[:, 1, :] *= -1.0
    st, h = _create(lib, inputs.Geometry(**{**g.__dict__, "pmats": ok}))
    assert st in (0, 3)      # 3 only where no GPU is present
    if st == 0:
        lib.kct_plan_destroy(h)

