"""Pins for the FP64 oracle: each check compares it with something other than itself
(closed forms derived from Eqs. 1-3, hand-computed covariances, numpy's eigensolver,
finite differences), chosen so that a dropped term, a wrong sign or a transposed operand
in the oracle fails at least one of them."""
import math

import numpy as np
import pytest

import oracle
from synthetic import bumpy_plane, tilted_plane

C1 = dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)
C2 = dict(nx=400, ny=400, n_yaw=72, res=0.05, length=0.9, width=0.6)


def P(**kw):
    return oracle.OracleParams(**kw)


# ----------------------------------------------------------------------------- footprint


@pytest.mark.parametrize("cfg,count", [(C1, 35), (C2, 247)])
def test_footprint_axis_aligned_is_full_inclusive_rectangle(cfg, count):
    p = P(**cfg)
    a = p.length / (2 * p.res)
    b = p.width / (2 * p.res)
    fp = oracle.footprint(p, 0)
    ia, ib = int(math.floor(a + 1e-6)), int(math.floor(b + 1e-6))
    want = {(di, dj) for dj in range(-ib, ib + 1) for di in range(-ia, ia + 1)}
    assert len(fp) == count == len(want)
    assert set(map(tuple, fp.tolist())) == want
    # the bin at yaw + pi is the same set (pi-symmetry is part of the definition)
    fp_pi = oracle.footprint(p, p.n_yaw // 2)
    assert np.array_equal(fp, fp_pi)


def test_footprint_hand_listed_small():
    # 3 x 1 cells along the heading at yaw 0; 1 x 3 across at yaw pi/2 (n_yaw = 4).
    p = P(nx=5, ny=5, n_yaw=4, res=0.1, length=0.3, width=0.1)
    assert sorted(map(tuple, oracle.footprint(p, 0).tolist())) == [(-1, 0), (0, 0), (1, 0)]
    assert sorted(map(tuple, oracle.footprint(p, 1).tolist())) == [(0, -1), (0, 0), (0, 1)]


def test_footprint_rotation_direction():
    # a long thin footprint at yaw 45 deg lies along di == dj (heading (1, 1)), not di == -dj
    p = P(nx=5, ny=5, n_yaw=8, res=1.0, length=10.0, width=0.6)
    fp = oracle.footprint(p, 1)
    assert all(di == dj for di, dj in fp.tolist())
    assert len(fp) == 7  # |u| = sqrt(2) |d| <= 5  ->  d in [-3, 3]


@pytest.mark.parametrize("cfg", [C1, C2])
def test_footprint_symmetries_and_area(cfg):
    p = P(**cfg)
    K = p.n_yaw
    a = p.length / (2 * p.res)
    b = p.width / (2 * p.res)
    h = math.sqrt(0.5)
    for k in range(K // 2):
        s = set(map(tuple, oracle.footprint(p, k).tolist()))
        assert all((-di, -dj) in s for di, dj in s)  # central symmetry
        # unit cells around the points cover the box shrunk by the half-diagonal and stay
        # inside the box grown by it
        assert 4 * (a - h) * (b - h) <= len(s) <= 4 * (a + h) * (b + h)
        if K % 4 == 0 and k + K // 4 < K // 2:
            s90 = set(map(tuple, oracle.footprint(p, k + K // 4).tolist()))
            assert s90 == {(-dj, di) for di, dj in s}  # quarter turn rotates the set


def test_footprint_ellipse_rows():
    p = P(nx=5, ny=5, n_yaw=4, res=0.05, length=0.9, width=0.6, shape="ellipse")
    a, b = 9.0, 6.0
    fp = oracle.footprint(p, 0)
    # per row dj the columns form |di| <= a sqrt(1 - (dj/b)^2) (up to the 1e-6 tolerance)
    want = sum(2 * int(math.floor(a * math.sqrt(max(0.0, 1 - (dj / b) ** 2)) + 1e-7)) + 1
               for dj in range(-6, 7))
    assert len(fp) == want


# ----------------------------------------------------------------------------- eigen


def test_jacobi_matches_numpy_eigh_random_spd():
    rng = np.random.default_rng(1)
    worst_val = worst_vec = 0.0
    for _ in range(20000):
        M = rng.normal(size=(3, 3))
        A = M @ M.T * rng.uniform(1e-4, 10)
        ev, V = oracle.jacobi3(A)
        wn, Vn = np.linalg.eigh(A)
        scale = np.abs(wn).max()
        worst_val = max(worst_val, np.abs(ev - wn).max() / scale)
        # reconstruction and orthonormality
        assert np.allclose(V @ np.diag(ev) @ V.T, A, atol=1e-12 * scale)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)
        for j in range(3):
            sep = min(abs(wn[j] - wn[i]) for i in range(3) if i != j) / scale
            if sep > 1e-6:
                worst_vec = max(worst_vec, 1 - abs(V[:, j] @ Vn[:, j]))
    assert worst_val < 1e-13
    assert worst_vec < 1e-10


def test_jacobi_near_degenerate():
    rng = np.random.default_rng(2)
    for _ in range(5000):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = rng.uniform(0.01, 1.0)
        d = np.array([rng.uniform(0, 1e-6), lam, lam * (1 + rng.uniform(0, 1e-10))])
        A = Q @ np.diag(d) @ Q.T
        ev, V = oracle.jacobi3(A)
        assert np.abs(ev - np.sort(d)).max() < 1e-14
        # the isolated smallest eigenvector is still well defined
        assert 1 - abs(V[:, 0] @ Q[:, 0]) < 1e-12


# ----------------------------------------------------------------------------- grid


def plane_closed_form(alpha, beta, theta):
    """For z = alpha x + beta y + gamma: with p = alpha cos + beta sin (slope along the
    heading) and q = beta cos - alpha sin (slope across it), Eqs. 2-3 give
    y_b ~ (-s, c, q) and x_b ~ (c + q beta, s - q alpha, p), with norm
    sqrt((1 + q^2)(1 + alpha^2 + beta^2)); hence roll = atan(q) and
    pitch = asin(p / sqrt((1 + q^2)(1 + p^2 + q^2)))."""
    p = alpha * np.cos(theta) + beta * np.sin(theta)
    q = beta * np.cos(theta) - alpha * np.sin(theta)
    return np.arcsin(p / np.sqrt((1 + q * q) * (1 + p * p + q * q))), np.arctan(q)


@pytest.mark.parametrize("cfg", [C1, dict(C2, nx=60, ny=60)])
@pytest.mark.parametrize("alpha,beta", [(0.2, -0.1), (-0.05, 0.3), (0.0, 0.0)])
def test_tilted_plane_closed_form_every_yaw(cfg, alpha, beta):
    p = P(**dict(cfg, nx=40, ny=40))
    origin = (123, -45)
    gamma = 2.5
    e = tilted_plane(p.nx, p.ny, p.res, alpha, beta, gamma, origin)
    out, fl = oracle.assess_grid(p, e, origin)
    th = 2 * np.pi * np.arange(p.n_yaw) / p.n_yaw
    pitch, roll = plane_closed_form(alpha, beta, th)
    R = 12
    sl = (slice(None), slice(R, p.ny - R), slice(R, p.nx - R))
    assert np.abs(out[1][sl] - pitch[:, None, None]).max() < 1e-12
    assert np.abs(out[2][sl] - roll[:, None, None]).max() < 1e-12
    assert np.abs(out[3][sl]).max() < 1e-12
    xs = (origin[0] + np.arange(p.nx) + 0.5) * p.res
    ys = (origin[1] + np.arange(p.ny) + 0.5) * p.res
    zc = alpha * xs[None, :] + beta * ys[:, None] + gamma
    assert np.abs(out[0][sl] - zc[None, R:-R, R:-R]).max() < 1e-11
    risk = (np.abs(pitch) / 0.52 + np.abs(roll) / 0.52) / 3.0
    assert np.abs(out[4][sl] - risk[:, None, None]).max() < 1e-12
    assert (fl[sl] == 0).all()


def test_flat_ground():
    p = P(**dict(C1, nx=30, ny=30))
    e = np.full((30, 30), 0.7)
    out, fl = oracle.assess_grid(p, e)
    sl = (slice(None), slice(4, 26), slice(4, 26))
    for ch in (1, 2, 3, 4):
        assert np.abs(out[ch][sl]).max() < 1e-14
    assert np.abs(out[0][sl] - 0.7).max() < 1e-14


def test_yaw_plus_pi_flips_pitch_and_roll():
    p = P(**dict(C1, nx=40, ny=40))
    e = bumpy_plane(3, 40, 40, 0.1).astype(np.float64)
    out, fl = oracle.assess_grid(p, e)
    h = p.n_yaw // 2
    a, b = out[:, :h], out[:, h:]
    ok = np.isfinite(a[1]) & np.isfinite(b[1])
    assert ok.sum() > 0.8 * ok.size
    assert np.abs(a[1][ok] + b[1][ok]).max() < 1e-12
    assert np.abs(a[2][ok] + b[2][ok]).max() < 1e-12
    for ch in (0, 3, 4):
        assert np.abs(a[ch][ok] - b[ch][ok]).max() < 1e-12
    assert np.array_equal(fl[:h], fl[h:])


def test_offset_invariance():
    p = P(**dict(C1, nx=30, ny=30))
    e = bumpy_plane(4, 30, 30, 0.1).astype(np.float64)
    o1, f1 = oracle.assess_grid(p, e)
    o2, f2 = oracle.assess_grid(p, e + 3.7)
    ok = np.isfinite(o1[0])
    assert np.abs(o2[0][ok] - o1[0][ok] - 3.7).max() < 1e-12
    for ch in (1, 2, 3, 4):
        assert np.abs(o2[ch][ok] - o1[ch][ok]).max() < 1e-10
    assert np.array_equal(f1, f2)


TINY = dict(nx=5, ny=5, n_yaw=4, res=0.1, length=0.3, width=0.3)  # 3 x 3 footprint at yaw 0


def test_tiny_stripes_hand_covariance():
    h = 0.1
    e = np.array([[h * (c % 2) for c in range(5)] for r in range(5)], np.float64)
    p = P(**TINY)
    out, f, d = oracle.cell_detail(p, e, 2, 2, 0)
    # columns 1, 2, 3 carry h, 0, h: mean z = 2h/3; var x = var y = 2 (0.1)^2 / 3;
    # var z = 2 h^2 / 9; all cross terms vanish.
    want = np.diag([0.02 / 3, 0.02 / 3, 2 * h * h / 9])
    assert d["n"] == 9
    assert np.allclose(d["cov"], want, atol=1e-16)
    assert np.allclose(d["mean"], [0.25, 0.25, 2 * h / 3], atol=1e-15)
    # kappa = (2h^2/9) / (0.04/3 + 2h^2/9) = 1/7 > kappa_max -> obstacle, flat normal
    assert abs(out[3] - 1 / 7) < 1e-14
    assert out[4] == 1.0 and f == oracle.OBSTACLE
    assert abs(out[1]) < 1e-15 and abs(out[2]) < 1e-15
    assert abs(out[0] - 2 * h / 3) < 1e-15


def test_tiny_corner_spike_hand_covariance():
    h = 0.05
    e = np.zeros((5, 5))
    e[3, 3] = h  # offset (+1, +1) from the centre cell (2, 2)
    p = P(**TINY)
    out, f, d = oracle.cell_detail(p, e, 2, 2, 0)
    # mean z = h/9; cov xz = cov yz = (0.1 h)/9; var z = 8 h^2 / 81
    want = np.array([[0.02 / 3, 0, 0.1 * h / 9], [0, 0.02 / 3, 0.1 * h / 9],
                     [0.1 * h / 9, 0.1 * h / 9, 8 * h * h / 81]])
    assert np.allclose(d["cov"], want, atol=1e-17)
    assert abs(d["mean"][2] - h / 9) < 1e-17
    # normal tilts away from the raised corner: n_x, n_y < 0
    assert d["z_b"][0] < 0 and d["z_b"][1] < 0 and d["z_b"][2] > 0
    # same cell, yaw pi/2 (bin 1): the 3 x 3 set is unchanged, so Cov and kappa are too
    out1, f1, d1 = oracle.cell_detail(p, e, 2, 2, 1)
    assert np.allclose(d1["cov"], want, atol=1e-17)
    assert abs(out1[3] - out[3]) < 1e-16


def test_collinear_footprint_is_degenerate():
    p = P(nx=5, ny=5, n_yaw=4, res=0.1, length=0.3, width=0.1)  # 3 x 1 footprint
    e = np.array([[0.1 * ((c + r) % 2) for c in range(5)] for r in range(5)], np.float64)
    out, f, d = oracle.cell_detail(p, e, 2, 2, 0)
    assert f & oracle.DEGENERATE and out[4] == 1.0 and np.isnan(out[1])


def test_risk_anisotropy_and_branches():
    # slope tan(0.45) along +x: facing uphill (yaw 0) pitch = 0.45 < 0.52 -> weighted risk;
    # facing across (yaw pi/2) roll = -0.45, |roll| > phi_y_max = 0.35 -> obstacle.
    alpha = math.tan(0.45)
    p = P(nx=30, ny=30, n_yaw=4, res=0.1, length=0.6, width=0.4, phi_y_max=0.35)
    e = tilted_plane(30, 30, 0.1, alpha, 0.0, 0.0)
    out, fl = oracle.assess_grid(p, e)
    assert abs(out[1, 0, 15, 15] - 0.45) < 1e-12
    assert abs(out[4, 0, 15, 15] - (0.45 / 0.52) / 3) < 1e-12 and fl[0, 15, 15] == 0
    assert abs(out[2, 1, 15, 15] + 0.45) < 1e-12
    assert out[4, 1, 15, 15] == 1.0 and fl[1, 15, 15] == oracle.OBSTACLE
    # steeper than phi_x_max along the heading -> obstacle at yaw 0 and yaw pi
    e2 = tilted_plane(30, 30, 0.1, math.tan(0.6), 0.0, 0.0)
    out2, fl2 = oracle.assess_grid(p, e2)
    assert out2[4, 0, 15, 15] == 1.0 and out2[4, 2, 15, 15] == 1.0
    assert abs(out2[1, 2, 15, 15] + 0.6) < 1e-12


def test_unknown_corner_cells_and_nan():
    p = P(**dict(C1, nx=30, ny=30))
    e = bumpy_plane(5, 30, 30, 0.1).astype(np.float64)
    out, fl = oracle.assess_grid(p, e)
    # corner cell (0, 0) at yaw 0 keeps 4 x 3 = 12 of 35 points < ceil(35/2) = 18
    assert fl[0, 0, 0] == oracle.UNKNOWN | oracle.OBSTACLE
    assert out[4, 0, 0, 0] == 1.0 and np.isnan(out[0, 0, 0, 0]) and np.isnan(out[3, 0, 0, 0])
    # edge cell (0, 15) keeps 4 x 5 = 20 >= 18 points -> assessed
    assert fl[0, 15, 0] & oracle.UNKNOWN == 0
    e2 = e.copy()
    e2[10:20, 10:20] = np.nan
    out2, fl2 = oracle.assess_grid(p, e2)
    assert (fl2[:, 15, 15] & oracle.UNKNOWN).all()
    # a cell whose footprint loses a few points is still assessed, over the known ones
    c, r = 22, 15  # footprint at yaw 0 spans columns 19..25: columns 19 lost
    assert fl2[0, r, c] & oracle.UNKNOWN == 0
    d = oracle.cell_detail(p, e2, c, r, 0)[2]
    assert d["n"] == 35 - 5


# ----------------------------------------------------------------------------- poses


def test_pose_query_equals_grid_at_cell_centres_yaw0():
    p = P(**dict(C1, nx=40, ny=40))
    origin = (7, 11)
    e = bumpy_plane(6, 40, 40, 0.1).astype(np.float64)
    g, gf = oracle.assess_grid(p, e, origin)
    cs = np.arange(8, 32)
    cc, rr = np.meshgrid(cs, cs)
    poses = np.stack([(origin[0] + cc.ravel() + 0.5) * p.res, (origin[1] + rr.ravel() + 0.5) * p.res,
                      np.zeros(cc.size)], 1)
    q, qf = oracle.query_poses(p, e, poses, origin)
    want = g[:, 0, rr.ravel(), cc.ravel()].T
    assert np.abs(q - want).max() < 1e-9
    assert np.array_equal(qf, gf[0, rr.ravel(), cc.ravel()])


def test_pose_query_plane_closed_form_continuous_yaw():
    p = P(**dict(C1, nx=40, ny=40))
    alpha, beta = 0.15, 0.22
    origin = (-3, 2)
    e = tilted_plane(40, 40, 0.1, alpha, beta, 1.0, origin)
    rng = np.random.default_rng(0)
    n = 500
    poses = np.stack([(origin[0] + rng.uniform(8, 32, n)) * 0.1, (origin[1] + rng.uniform(8, 32, n)) * 0.1,
                      rng.uniform(0, 2 * np.pi, n)], 1)
    q, qf = oracle.query_poses(p, e, poses, origin)
    pitch, roll = plane_closed_form(alpha, beta, poses[:, 2])
    assert np.abs(q[:, 1] - pitch).max() < 1e-12
    assert np.abs(q[:, 2] - roll).max() < 1e-12
    assert np.abs(q[:, 0] - (alpha * poses[:, 0] + beta * poses[:, 1] + 1.0)).max() < 1e-12
    assert np.abs(q[:, 3]).max() < 1e-12


def test_pose_vjp_matches_central_differences():
    p = P(**dict(C1, nx=50, ny=50, kappa_max=1.0, phi_x_max=1.4, phi_y_max=1.4))
    origin = (0, 0)
    e = bumpy_plane(7, 50, 50, 0.1).astype(np.float64)
    rng = np.random.default_rng(3)
    n = 200
    poses = np.stack([rng.uniform(10, 40, n) * 0.1, rng.uniform(10, 40, n) * 0.1,
                      rng.uniform(0, 2 * np.pi, n)], 1)
    g = rng.normal(size=(n, 5))
    gp = oracle.query_poses_vjp(p, e, poses, g, origin)
    h = 1e-6
    fd = np.zeros_like(gp)
    for j in range(3):
        dp = np.zeros(3)
        dp[j] = h
        op, _ = oracle.query_poses(p, e, poses + dp, origin)
        om, _ = oracle.query_poses(p, e, poses - dp, origin)
        fd[:, j] = ((op - om) * g).sum(1) / (2 * h)
    err = np.abs(gp - fd) / (1e-3 + np.abs(fd))
    # a lattice point crossing a bilinear grid line within +-h spoils the difference
    assert np.median(err) < 1e-6
    assert (err < 1e-4).mean() > 0.97
