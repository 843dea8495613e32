"""Pins of the SE(2) signed-distance reference (oracle/sdf.py) against independent mathematics:
scipy's exact Euclidean distance transform on random masks, the radial field of a single
obstacle, the linear field of a half-plane, empty and full obstacle sets, the clamp, and the
ring indexing of the storage."""
import numpy as np
import pytest

from oracle.sdf import risk_sdf

RES = 0.1


def test_matches_scipy_edt():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    risk = rng.uniform(0, 1, size=(3, 23, 31))
    risk[rng.random(risk.shape) < 0.15] = 1.0
    sdf = risk_sdf(risk, RES)
    for k in range(3):
        obst = risk[k] >= 1.0
        # distance_transform_edt gives, for each nonzero entry, the distance to the nearest zero
        d_obs = nd.distance_transform_edt(~obst)   # free cells: distance to the nearest obstacle
        d_free = nd.distance_transform_edt(obst)   # obstacle cells: distance to the nearest free cell
        assert np.allclose(sdf[k], RES * (d_obs - d_free), atol=1e-12)


def test_single_obstacle_is_radial():
    risk = np.zeros((1, 15, 17))
    risk[0, 6, 9] = 1.0
    sdf = risk_sdf(risk, RES)
    r, c = np.mgrid[0:15, 0:17]
    ref = RES * np.hypot(r - 6, c - 9)
    ref[6, 9] = -RES  # the obstacle cell: its four neighbours are free, one cell away
    assert np.allclose(sdf[0], ref, atol=1e-12)


def test_half_plane_is_linear_and_clamped():
    risk = np.zeros((2, 10, 12))
    risk[:, :, 7:] = 1.0  # obstacles from column 7 on
    sdf = risk_sdf(risk, RES, clamp=0.35)
    c = np.arange(12)
    ref = np.where(c < 7, RES * (7 - c), -RES * (c - 6))
    assert np.allclose(sdf, np.clip(ref, -0.35, 0.35)[None, None, :], atol=1e-12)


def test_nan_is_an_obstacle():
    risk = np.zeros((1, 9, 9))
    risk[0, 4, 4] = np.nan
    sdf = risk_sdf(risk, RES)
    r, c = np.mgrid[0:9, 0:9]
    ref = RES * np.hypot(r - 4, c - 4)
    ref[4, 4] = -RES
    assert np.allclose(sdf[0], ref, atol=1e-12)


def test_empty_and_full_sets_and_threshold():
    risk = np.full((2, 5, 6), 0.5)
    risk[1] = 1.0
    sdf = risk_sdf(risk, RES, clamp=2.0)
    assert (sdf[0] == 2.0).all() and (sdf[1] == -2.0).all()
    lower = risk_sdf(risk, RES, risk_obstacle=0.4, clamp=2.0)  # everything is an obstacle
    assert (lower == -2.0).all()


def test_ring_storage_and_cell_selection():
    rng = np.random.default_rng(1)
    logical = rng.uniform(0, 1, size=(2, 9, 11))
    logical[rng.random(logical.shape) < 0.2] = 1.0
    ring = (4, 3)
    stored = np.empty_like(logical)
    r = (np.arange(9) + ring[1]) % 9
    c = (np.arange(11) + ring[0]) % 11
    stored[:, r[:, None], c[None, :]] = logical
    a = risk_sdf(logical, RES)
    b = risk_sdf(stored, RES, ring=ring)
    assert np.allclose(b[:, r[:, None], c[None, :]], a)
    cells = np.array([[0, 0, 0], [10, 8, 1], [5, 4, 1]])
    sel = risk_sdf(stored, RES, ring=ring, cells=cells)
    assert np.allclose(sel, [a[0, 0, 0], a[1, 8, 10], a[1, 4, 5]])
