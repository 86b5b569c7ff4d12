"""kct_count_pairs (nonzero voxel-pixel weights counted on the GPU) against the nonzero
entries of the oracle's dense matrix on a tiny geometry.

Both sides decide "nonzero" in floating point, so pairs whose weight is at the rounding level
may go either way: the GPU drops pairs whose cut volume is below 1e-9 of the voxel volume.
The count must lie between the oracle's entries with W > 1e-8 W_full and those with
W > 1e-11 W_full, W_full = V / r^2 the weight of the whole voxel."""
import numpy as np
import pytest

import oracle
from oracle.cgls import dense_matrix
from paper_2110_09841_b300 import inputs
from paper_2110_09841_b300.kct import Projector

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("vname,variant", [("exact", oracle.EXACT), ("relaxed", oracle.RELAXED)])
def test_pair_count_matches_oracle_nonzeros(vname, variant):
    # generic sizes (odd pixel counts, pitch unrelated to the voxel size, 7 views) so that no
    # voxel edge projects exactly onto a pixel boundary, where a zero-size cut could round
    # either way (the relaxed variant keeps any positive overlap)
    g = inputs.make_geometry((4, 4, 4), (0.93, 0.93, 0.93), (11, 11), (1.07, 1.07), 7, 61.7, 93.1, 360.0)
    A = dense_matrix(g, variant).reshape(g.nviews, g.nv, g.nu, -1)
    vol = g.ax * g.ay * g.az
    strict = loose = 0
    for view in range(g.nviews):
        s = oracle.source(g.pmats[view])
        for m in range(g.nv):
            for n in range(g.nu):
                F = oracle.pixel_factor(g.pmats[view], float(n), float(m))
                for j, e in enumerate(A[view, m, n]):
                    if e <= 0.0:
                        continue
                    k, jj, i = np.unravel_index(j, g.vol_shape)
                    c = np.array([(i - (g.nx - 1) / 2) * g.ax, (jj - (g.ny - 1) / 2) * g.ay, (k - (g.nz - 1) / 2) * g.az])
                    wfull = vol / float(np.sum((c - s) ** 2))
                    r = e / F / wfull
                    strict += r > 1e-8
                    loose += r > 1e-11
    got = Projector(g, vname, "cos").count_pairs()
    assert strict <= got <= loose, (strict, got, loose)
