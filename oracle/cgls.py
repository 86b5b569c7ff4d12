"""FP64 CGLS for the oracle -- test infrastructure only (tests, smoke check and the CPU
baseline of the benchmark use it; the product path never does).

The paper uses CGLS as the reconstruction that drives its projector timings (Sec. IV-A: 40
iterations on uniform random projection data) and names Krylov LSQR and CGLS as the methods of
its software (Sec. V "Software"). It does not restate the method, so this is the textbook
algorithm: conjugate gradients on the normal equations A^T A x = A^T b in the factored form
that applies A and A^T once per iteration and never forms A^T A (Hestenes and Stiefel 1952;
Bjorck, "Numerical Methods for Least Squares Problems", 1996, Sec. 7.4). With r = b - A x and
s = A^T r:

    start   r0 = b - A x0,  s0 = A^T r0,  p0 = s0,  gamma0 = |s0|^2
    step    q = A p;  alpha = gamma / |q|^2;  x += alpha p;  r -= alpha q;
            s = A^T r;  gamma' = |s|^2;  beta = gamma' / gamma;  p = s + beta p

Residuals reported after k steps (both with fixed denominators):
    normal  |A^T (b - A x_k)| / |A^T b|     (the stopping rule)
    data    |b - A x_k| / |b|
"""
from __future__ import annotations

import numpy as np

from . import oracle


def cgls(matvec, rmatvec, b, iterations: int, x0=None, tol: float | None = None, keep_iterates=False):
    """Run up to `iterations` CGLS steps for min |b - A x| with A given by `matvec` (x -> A x)
    and `rmatvec` (y -> A^T y), in float64.

    Stops early once the normal residual is <= tol (checked before each step, so a start
    that already meets it takes no step). Returns dict(x, iterations, normal, data, iterates):
    normal[k] and data[k] are the residuals after k steps, iterates[k] = x_k when
    keep_iterates is set."""
    b = np.asarray(b, dtype=np.float64)
    atb = rmatvec(b)
    atb_norm = float(np.linalg.norm(atb))
    b_norm = float(np.linalg.norm(b))
    if x0 is None:
        x = np.zeros_like(atb)
        r = b.copy()
        s = atb.copy()
    else:
        x = np.array(x0, dtype=np.float64).reshape(atb.shape)
        r = b - matvec(x)
        s = rmatvec(r)
    p = s.copy()
    gamma = float(np.vdot(s, s))
    normal = [np.sqrt(gamma) / atb_norm if atb_norm > 0 else 0.0]
    data = [float(np.linalg.norm(r)) / b_norm if b_norm > 0 else 0.0]
    iterates = [x.copy()] if keep_iterates else None
    k = 0
    while k < iterations and not (tol is not None and normal[-1] <= tol) and gamma > 0:
        q = matvec(p)
        alpha = gamma / float(np.vdot(q, q))
        x = x + alpha * p
        r = r - alpha * q
        s = rmatvec(r)
        gamma_new = float(np.vdot(s, s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        k += 1
        normal.append(np.sqrt(gamma) / atb_norm)
        data.append(float(np.linalg.norm(r)) / b_norm)
        if keep_iterates:
            iterates.append(x.copy())
    return dict(x=x, iterations=k, normal=np.array(normal), data=np.array(data), iterates=iterates)


def cgls_cvp(geom, b, iterations: int, variant: int = oracle.EXACT, scaling: int = oracle.SCALE_COS,
             x0=None, tol: float | None = None, keep_iterates=False):
    """CGLS with the oracle's CVP operator (oracle.project / oracle.backproject)."""
    return cgls(lambda v: oracle.project(geom, v, variant, scaling),
                lambda y: oracle.backproject(geom, y, variant, scaling),
                b, iterations, x0=x0, tol=tol, keep_iterates=keep_iterates)


def dense_matrix(geom, variant: int = oracle.EXACT, scaling: int = oracle.SCALE_COS) -> np.ndarray:
    """The CVP operator as a dense [pixels, voxels] float64 matrix, one oracle projection of a
    unit voxel per column (tiny geometries only)."""
    n = geom.nx * geom.ny * geom.nz
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(oracle.project(geom, e.reshape(geom.vol_shape), variant, scaling).ravel())
    return np.stack(cols, axis=1)
