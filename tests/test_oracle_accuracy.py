"""The paper's accuracy comparison (Sec. IV-B) on the oracle: the projection of a single
1 x 1 x 5 mm voxel at the centre of rotation onto a fine detector (616 x 480 cells of
0.154 mm, SID 749 / SDD 1198 mm), per view, against K x K ray integration with exact path
lengths, measured by the relative Frobenius error of the view. The near-exact and relaxed
CVP values must agree with the K = 32 ray average far better than a single ray through each
pixel centre does, and the ray average must approach them as K grows (the remaining
difference is the ray average's own sampling error)."""
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
