"""Pins of the oracle's CGLS against textbook least squares on the dense CVP matrix.

CGLS after k steps from x0 = 0 is the minimiser of |b - A x| over the Krylov space
K_k = span{A^T b, (A^T A) A^T b, ..., (A^T A)^(k-1) A^T b}; after n = #unknowns steps (in exact
arithmetic) it is the least-squares solution. Both facts are checked here with numpy's
dense routines (an orthonormal Krylov basis by Gram-Schmidt, numpy.linalg.lstsq), which share
nothing with the CGLS recurrences.
"""
import numpy as np
import pytest

import oracle
from oracle.cgls import cgls, cgls_cvp, dense_matrix
from paper_2110_09841_b300 import inputs


@pytest.fixture(scope="module")
def dense():
    g = inputs.make_geometry((4, 4, 4), (1.0, 1.0, 1.0), (10, 10), (1.0, 1.0), 8, 60.0, 90.0, 360.0)
    A = dense_matrix(g)
    rng = np.random.default_rng(77)
    b = A @ rng.uniform(0.0, 1.0, A.shape[1]) + 0.05 * rng.standard_normal(A.shape[0])
    return g, A, b


def test_dense_matrix_has_full_column_rank(dense):
    _, A, _ = dense
    s = np.linalg.svd(A, compute_uv=False)
    assert s[-1] > 1e-6 * s[0]


def test_cgls_converges_to_lstsq(dense):
    _, A, b = dense
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    out = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 400, tol=1e-12)
    assert out["normal"][-1] <= 1e-12
    assert np.linalg.norm(out["x"] - ref) <= 1e-7 * np.linalg.norm(ref)
    # the data residual of the solution is the least-squares residual
    assert out["data"][-1] == pytest.approx(np.linalg.norm(b - A @ ref) / np.linalg.norm(b), rel=1e-8)


def test_iterates_minimise_over_krylov_spaces(dense):
    _, A, b = dense
    out = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 6, keep_iterates=True)
    N = A.T @ A
    basis = []
    v = A.T @ b
    for k in range(1, 7):
        w = v.copy()
        for _ in range(2):                       # Gram-Schmidt, twice for orthogonality
            for q in basis:
                w -= np.dot(q, w) * q
        basis.append(w / np.linalg.norm(w))
        Q = np.stack(basis, axis=1)
        c = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        xk = Q @ c
        assert np.linalg.norm(out["iterates"][k] - xk) <= 1e-9 * np.linalg.norm(xk), k
        v = N @ basis[-1]


def test_residual_histories_match_their_definitions(dense):
    _, A, b = dense
    out = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 8, keep_iterates=True)
    atb = np.linalg.norm(A.T @ b)
    for k, xk in enumerate(out["iterates"]):
        r = b - A @ xk
        assert out["normal"][k] == pytest.approx(np.linalg.norm(A.T @ r) / atb, rel=1e-9, abs=1e-14)
        assert out["data"][k] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-9)
    assert out["normal"][0] == 1.0 and out["data"][0] == 1.0


def test_warm_start_at_the_solution_takes_no_step(dense):
    _, A, b = dense
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    out = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 50, x0=ref, tol=1e-8)
    assert out["iterations"] == 0
    # a warm start half way leaves a smaller normal residual than the zero start
    half = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 50, x0=0.5 * ref, tol=1e-8)
    assert half["normal"][0] < 1.0


def test_cvp_operator_form_equals_dense_form(dense):
    """The operator form (oracle.project / oracle.backproject per step) and the dense matrix
    give the same iterates: the oracle's backprojection is the transpose of its projection."""
    g, A, b = dense
    op = cgls_cvp(g, b.reshape(g.proj_shape), 5, oracle.EXACT, oracle.SCALE_COS)
    de = cgls(lambda v: A @ v, lambda y: A.T @ y, b, 5)
    np.testing.assert_allclose(op["x"].ravel(), de["x"], rtol=1e-9, atol=1e-12 * np.abs(de["x"]).max())
    np.testing.assert_allclose(op["normal"], de["normal"], rtol=1e-9)
