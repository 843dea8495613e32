"""Pins of the nearest-neighbour inpainting reference (oracle/inpaint.py): the distance to the
chosen source equals scipy's exact Euclidean distance transform, hand-built ties resolve to
the smallest column then row, a single known cell fills everything, the radius leaves far cells
unknown, and a map without known cells stays unknown."""
import numpy as np
import pytest

from oracle.inpaint import inpaint_nearest


def test_distances_match_scipy_edt():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    z = rng.normal(size=(37, 41))
    z[rng.random(z.shape) < 0.6] = np.nan
    out, src = inpaint_nearest(z)
    known = ~np.isnan(z)
    edt = nd.distance_transform_edt(~known)  # distance of each unknown cell to the nearest known
    r, c = np.mgrid[0:37, 0:41]
    d = np.hypot(src[..., 0] - r, src[..., 1] - c)
    assert np.allclose(d, edt, atol=1e-12)
    assert np.array_equal(out[known], z[known])
    assert np.array_equal(out, z[src[..., 0], src[..., 1]])


def test_ties_take_smallest_column_then_row():
    z = np.full((7, 7), np.nan)
    # four known cells at distance 2 from the centre (3, 3): up, down, left, right
    z[1, 3], z[5, 3], z[3, 1], z[3, 5] = 1.0, 2.0, 3.0, 4.0
    out, src = inpaint_nearest(z)
    assert out[3, 3] == 3.0 and tuple(src[3, 3]) == (3, 1)  # column 1 is the smallest
    # same column, rows above and below at equal distance: the smaller row
    z2 = np.full((5, 3), np.nan)
    z2[0, 1], z2[4, 1] = 7.0, 8.0
    out2, src2 = inpaint_nearest(z2)
    assert out2[2, 1] == 7.0 and tuple(src2[2, 1]) == (0, 1)


def test_single_known_cell_and_radius():
    z = np.full((9, 12), np.nan)
    z[4, 6] = 2.5
    out, _ = inpaint_nearest(z)
    assert (out == 2.5).all()
    out_r, src_r = inpaint_nearest(z, max_cells=3)
    r, c = np.mgrid[0:9, 0:12]
    near = (r - 4) ** 2 + (c - 6) ** 2 <= 9
    assert (out_r[near] == 2.5).all() and np.isnan(out_r[~near]).all()
    assert (src_r[~near] == -1).all()


def test_all_unknown_stays_unknown():
    z = np.full((4, 5), np.nan)
    out, src = inpaint_nearest(z)
    assert np.isnan(out).all() and (src == -1).all()
