"""kct_cgls (CGLS with the CVP operator on the GPU) against the oracle's FP64 CGLS.

The GPU and oracle operators agree to float32 rounding (per-pixel relative differences of
1e-6 typical, 1e-4 at most), and the first CGLS iterates are smooth functions of the
operator, so the iterates and residual histories of the two agree to a few 1e-4 relative;
1e-3 is the bound used here. The stopping decision is checked with the oracle itself: the
oracle's normal-equation residual of the GPU's final x must meet the tolerance (up to the
same operator difference).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle.cgls import cgls_cvp
from paper_2110_09841_b300 import inputs
from paper_2110_09841_b300.kct import KctError, Projector

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-3


def small():
    return inputs.make_geometry((16, 16, 16), (1.0, 1.0, 1.0), (40, 32), (0.8, 0.8), 12, 750.0, 1200.0, 360.0)


def ragged():
    return inputs.make_geometry((13, 11, 9), (1.0, 1.0, 1.0), (37, 29), (0.8, 0.8), 7, 750.0, 1200.0, 360.0)


def phantom(g, seed):
    return inputs.voxelize(g, inputs.random_ellipsoids(seed, 5, g.nx * g.ax, (2.0, 6.0), (0.005, 0.02)))


def oracle_normal_residual(g, b, x, variant):
    r = b - oracle.project(g, x, variant)
    return np.linalg.norm(oracle.backproject(g, r, variant)) / np.linalg.norm(oracle.backproject(g, b, variant))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("vname,variant", [("exact", oracle.EXACT), ("relaxed", oracle.RELAXED)])
@pytest.mark.parametrize("gname", ["small", "ragged"])
def test_iterates_match_oracle(vname, variant, gname):
    g = small() if gname == "small" else ragged()
    b = inputs.uniform_projections(g.proj_shape, 21).numpy().astype(np.float64)
    ref = cgls_cvp(g, b, 5, variant, keep_iterates=True)
    A = Projector(g, vname, "cos")
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    for k in (1, 3, 5):
        x, info = A.cgls(bd, max_iter=k, tol=0.0)
        assert info["iterations"] == k
        assert rel(x.cpu().numpy(), ref["iterates"][k]) <= ITER_TOL, k
        np.testing.assert_allclose(info["normal"], ref["normal"][:k + 1], rtol=ITER_TOL)
        np.testing.assert_allclose(info["data"], ref["data"][:k + 1], rtol=ITER_TOL)


@pytest.mark.parametrize("vname,variant", [("exact", oracle.EXACT), ("relaxed", oracle.RELAXED)])
def test_reaches_tolerance_checked_by_oracle(vname, variant):
    g = small()
    b = oracle.project(g, phantom(g, 5), variant)
    A = Projector(g, vname, "cos")
    x, info = A.cgls(torch.from_numpy(b.astype(np.float32)).cuda(), max_iter=300, tol=1e-3)
    assert info["converged"] and info["normal"][-1] <= 1e-3
    assert np.all(np.diff(info["data"]) <= 1e-6)          # |b - A x_k| never grows in CGLS
    assert oracle_normal_residual(g, b, x.cpu().numpy().astype(np.float64), variant) <= 1.05e-3
    ref = cgls_cvp(g, b, 300, variant, tol=1e-3)
    assert abs(info["iterations"] - ref["iterations"]) <= 1


def test_warm_start():
    g = small()
    b = oracle.project(g, phantom(g, 6))
    A = Projector(g, "exact", "cos")
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    x, info = A.cgls(bd, max_iter=300, tol=1e-3)
    # starting at the solution takes no step
    x2, info2 = A.cgls(bd, x0=x.clone(), max_iter=300, tol=1e-3)
    assert info2["iterations"] == 0 and info2["converged"]
    torch.testing.assert_close(x2, x, rtol=0, atol=0)
    # a warm start matches the oracle's warm-started CGLS
    x0 = (0.5 * x).cpu().numpy().astype(np.float64)
    ref = cgls_cvp(g, b, 3, oracle.EXACT, x0=x0, keep_iterates=True)
    x3, info3 = A.cgls(bd, x0=0.5 * x, max_iter=3, tol=0.0)
    assert rel(x3.cpu().numpy(), ref["iterates"][3]) <= ITER_TOL
    np.testing.assert_allclose(info3["normal"], ref["normal"], rtol=ITER_TOL)


def test_rejects_bad_workspace_and_alignment():
    g = small()
    A = Projector(g, "exact", "cos")
    b = torch.zeros(g.proj_shape, device="cuda")
    small_ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(KctError) as e:
        A.cgls(b, workspace=small_ws)
    assert e.value.status == 1
    ws = A.cgls_workspace()
    buf = torch.zeros(g.nx * g.ny * g.nz + 1, device="cuda")
    rc = A.lib.kct_cgls(A.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(buf.data_ptr() + 4), None, 0, 2,
                        1e-3, ctypes.c_void_p(ws.data_ptr()), ws.numel(), None, None, None,
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1


@pytest.mark.parametrize("warm", [False, True])
def test_precomputed_atb_gives_the_same_solve(warm):
    """Passing A^T b (which a learned warm start already computes) skips one backprojection
    and changes nothing else: the same iterates and residual histories."""
    g = small()
    A = Projector(g, "relaxed", "cos")
    truth = phantom(g, 5).cuda()
    b = A.project(truth)
    x0 = 0.5 * truth if warm else None
    x1, i1 = A.cgls(b, x0=x0, max_iter=6, tol=0.0)
    x2, i2 = A.cgls(b, x0=x0, max_iter=6, tol=0.0, atb=A.backproject(b))
    assert i1["iterations"] == i2["iterations"] == 6
    np.testing.assert_allclose(i2["normal"], i1["normal"], rtol=1e-5)
    np.testing.assert_allclose(i2["data"], i1["data"], rtol=1e-5)
    assert float((x1 - x2).abs().max()) <= 1e-5 * float(x1.abs().max())


def test_zero_data_gives_zero():
    g = small()
    A = Projector(g, "relaxed", "cos")
    x, info = A.cgls(torch.zeros(g.proj_shape, device="cuda"), max_iter=5, tol=1e-3)
    assert info["iterations"] == 0 and info["converged"]
    assert float(x.abs().max()) == 0.0
