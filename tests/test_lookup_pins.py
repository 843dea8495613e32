"""Pins of the trilinear SE(2) lookup reference (oracle/se2_lookup.py) against what the
mathematics fixes: values at the grid nodes, exact reproduction of multilinear functions,
SO(2) periodicity and the wrap cell, central differences of the value, scipy's linear
RegularGridInterpolator on the unrolled periodic grid, and the outside rule."""
import numpy as np
import pytest

from oracle.se2_lookup import UNKNOWN, se2_lookup

K, NY, NX = 8, 9, 11
RES = 0.2
ORIGIN = (-3, 5)
RING = (4, 7)


def logical_to_ring(L):
    """Store a logical [K][ny][nx] grid at ring-indexed positions."""
    K_, ny, nx = L.shape
    V = np.empty_like(L)
    r = (np.arange(ny) + RING[1]) % ny
    c = (np.arange(nx) + RING[0]) % nx
    V[:, r[:, None], c[None, :]] = L
    return V


def world(c, r, k):
    return np.stack([(ORIGIN[0] + c + 0.5) * RES, (ORIGIN[1] + r + 0.5) * RES, 2 * np.pi * k / K], axis=-1)


def test_grid_nodes():
    rng = np.random.default_rng(0)
    L = rng.normal(size=(K, NY, NX))
    kk, rr, cc = np.meshgrid(np.arange(K), np.arange(NY), np.arange(NX), indexing="ij")
    P = world(cc.ravel(), rr.ravel(), kk.ravel())
    val, _, fl = se2_lookup(logical_to_ring(L), P, RES, ORIGIN, RING)
    assert np.allclose(val, L.ravel(), atol=1e-12, rtol=0)
    assert not fl.any()


def test_multilinear_functions_are_reproduced():
    # V = (1 + 0.3 c)(2 - 0.1 r)(0.5 + 0.7 k) on the grid -> the interpolant is the same product
    # of the continuous coordinates inside the grid (away from the yaw wrap cell)
    kk, rr, cc = np.meshgrid(np.arange(K), np.arange(NY), np.arange(NX), indexing="ij")
    L = (1 + 0.3 * cc) * (2 - 0.1 * rr) * (0.5 + 0.7 * kk)
    rng = np.random.default_rng(1)
    u = rng.uniform(0, NX - 1, 5000)
    v = rng.uniform(0, NY - 1, 5000)
    w = rng.uniform(0, K - 1, 5000)
    P = world(u, v, w)
    val, grad, _ = se2_lookup(logical_to_ring(L), P, RES, ORIGIN, RING)
    assert np.allclose(val, (1 + 0.3 * u) * (2 - 0.1 * v) * (0.5 + 0.7 * w), atol=1e-10)
    # its gradient in world units
    gx = 0.3 * (2 - 0.1 * v) * (0.5 + 0.7 * w) / RES
    gy = (1 + 0.3 * u) * (-0.1) * (0.5 + 0.7 * w) / RES
    gt = (1 + 0.3 * u) * (2 - 0.1 * v) * 0.7 * K / (2 * np.pi)
    assert np.allclose(grad, np.stack([gx, gy, gt], 1), atol=1e-9)


def test_so2_periodicity_and_wrap_cell():
    rng = np.random.default_rng(2)
    L = rng.normal(size=(K, NY, NX))
    V = logical_to_ring(L)
    P = world(rng.uniform(0, NX - 1, 2000), rng.uniform(0, NY - 1, 2000), rng.uniform(0, K, 2000))
    v0, g0, _ = se2_lookup(V, P, RES, ORIGIN, RING)
    for m in (-3, -1, 1, 2):
        Q = P.copy()
        Q[:, 2] += 2 * np.pi * m
        v1, g1, _ = se2_lookup(V, Q, RES, ORIGIN, RING)
        assert np.allclose(v0, v1, atol=1e-9) and np.allclose(g0, g1, atol=1e-8)
    # at a node in (x, y), a yaw inside the last bin interpolates between bins K-1 and 0
    t = 0.3
    P = world(np.array([4.0]), np.array([2.0]), np.array([K - 1 + t]))
    val, _, _ = se2_lookup(V, P, RES, ORIGIN, RING)
    assert np.isclose(val[0], (1 - t) * L[K - 1, 2, 4] + t * L[0, 2, 4], atol=1e-12)


def test_central_differences():
    rng = np.random.default_rng(3)
    L = rng.normal(size=(K, NY, NX))
    V = logical_to_ring(L)
    # keep away from cell faces so that the trilinear form is smooth around each pose
    u = rng.integers(0, NX - 1, 500) + rng.uniform(0.1, 0.9, 500)
    v = rng.integers(0, NY - 1, 500) + rng.uniform(0.1, 0.9, 500)
    w = rng.integers(0, K, 500) + rng.uniform(0.1, 0.9, 500)
    P = world(u, v, w)
    _, grad, _ = se2_lookup(V, P, RES, ORIGIN, RING)
    h = 1e-6
    for j, step in enumerate((h * RES, h * RES, h * 2 * np.pi / K)):
        Pp, Pm = P.copy(), P.copy()
        Pp[:, j] += step
        Pm[:, j] -= step
        fd = (se2_lookup(V, Pp, RES, ORIGIN, RING)[0] - se2_lookup(V, Pm, RES, ORIGIN, RING)[0]) / (2 * step)
        assert np.allclose(fd, grad[:, j], rtol=1e-6, atol=1e-5 * np.abs(grad[:, j]).max())


def test_matches_scipy_regular_grid_interpolator():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(4)
    L = rng.normal(size=(K, NY, NX))
    Lp = np.concatenate([L, L[:1]], axis=0)  # bin K repeats bin 0 (period 2 pi)
    f = interp.RegularGridInterpolator((np.arange(K + 1), np.arange(NY), np.arange(NX)), Lp, method="linear")
    u = rng.uniform(0, NX - 1, 3000)
    v = rng.uniform(0, NY - 1, 3000)
    w = rng.uniform(0, K, 3000)
    ref = f(np.stack([w, v, u], 1))
    val, _, _ = se2_lookup(logical_to_ring(L), world(u, v, w), RES, ORIGIN, RING)
    assert np.allclose(val, ref, atol=1e-12)


def test_outside_and_unknown():
    rng = np.random.default_rng(5)
    L = rng.normal(size=(K, NY, NX))
    L[3, 4, 5] = np.nan
    V = logical_to_ring(L)
    P = world(np.array([-0.01, NX - 1 + 1e-6, 2.0, 5.0, NX - 1.0]), np.array([3.0, 3.0, NY - 0.5, 4.0, NY - 1.0]),
              np.array([1.0, 1.0, 1.0, 3.0, 2.0]))
    val, grad, fl = se2_lookup(V, P, RES, ORIGIN, RING, fill=7.0)
    assert val[0] == 7.0 and val[1] == 7.0 and val[2] == 7.0
    assert (fl[:3] == UNKNOWN).all() and (grad[:3] == 0).all()
    assert np.isnan(val[3]) and fl[3] == UNKNOWN  # the NaN node itself
    assert np.isclose(val[4], L[2, NY - 1, NX - 1]) and fl[4] == 0  # the far corner is inside
