"""Pins of the elevation-update reference (oracle/elevation.py) against independent mathematics:
the height variance against first-order propagation with finite-difference Jacobians (right
perturbation of the attitude), the information-form fusion against the sequential 1-D Kalman
update, the gate rules, the window move, and ray casting against hand-built scenes and against
dense sampling of the segment."""
import numpy as np
import pytest

from oracle.elevation import B3, ElevationMap, ElevParams, ScanPose, point_heights, skew


def rot(rx, ry, rz):
    def R(axis, a):
        c, s = np.cos(a), np.sin(a)
        M = np.eye(3)
        i, j = [(1, 2), (0, 2), (0, 1)][axis]
        M[i, i], M[i, j], M[j, i], M[j, j] = c, -s, s, c
        return M
    return R(2, rz) @ R(1, ry) @ R(0, rx)


def expm_so3(w):
    th = np.linalg.norm(w)
    K = skew(w / th) if th > 0 else np.zeros((3, 3))
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def pose(rng=None, **kw):
    rng = rng or np.random.default_rng(0)
    A = rng.normal(size=(3, 3, 3))
    sig = [a @ a.T * 1e-4 + np.eye(3) * 1e-5 for a in A]
    d = dict(R_B=rot(0.05, -0.08, 0.7), p_B=np.array([3.2, -1.7, 0.45]), R_BS=rot(0.0, 0.1, 0.0),
             p_BS=np.array([0.1, 0.0, 0.25]), Sigma_S=sig[0], Sigma_R=sig[1], Sigma_B=sig[2])
    d.update(kw)
    return ScanPose(**d)


def test_variance_matches_finite_difference_propagation():
    P = pose()
    pts = np.random.default_rng(1).normal(size=(20, 3)) * 3
    _, _, s2 = point_heights(P, pts)

    def z(R_B, p_B, q):
        return B3 @ (R_B @ (P.R_BS @ q + P.p_BS) + p_B)

    h = 1e-6
    for i, q in enumerate(pts):
        JS = np.array([(z(P.R_B, P.p_B, q + h * e) - z(P.R_B, P.p_B, q - h * e)) / (2 * h) for e in np.eye(3)])
        JR = np.array([(z(P.R_B @ expm_so3(h * e), P.p_B, q) - z(P.R_B @ expm_so3(-h * e), P.p_B, q)) / (2 * h)
                       for e in np.eye(3)])
        JB = np.array([(z(P.R_B, P.p_B + h * e, q) - z(P.R_B, P.p_B - h * e, q)) / (2 * h) for e in np.eye(3)])
        ref = JS @ P.Sigma_S @ JS + JR @ P.Sigma_R @ JR + JB @ P.Sigma_B @ JB
        assert np.isclose(s2[i], ref, rtol=1e-6, atol=1e-12)


def flat_pose(x=0.52, y=0.52, z=0.5):
    return ScanPose(R_B=np.eye(3), p_B=np.array([x, y, z]), R_BS=np.eye(3), p_BS=np.zeros(3),
                    Sigma_S=np.eye(3) * 1e-4, Sigma_R=np.zeros((3, 3)), Sigma_B=np.zeros((3, 3)))


def sensor_points(P, world):
    """Sensor-frame coordinates of world points (identity attitude in these scenes)."""
    return np.asarray(world, np.float64) - P.p_B - P.p_BS


def test_information_fusion_is_the_sequential_kalman_update():
    p = ElevParams(nx=10, ny=10, res=0.1, gate=1e9, clear_margin=1e9)
    P = flat_pose()
    m = ElevationMap(p)
    m.integrate(P, sensor_points(P, [[0.55, 0.55, 0.20]]))  # one point initialises the cell
    zs = [0.21, 0.19, 0.205]
    m.integrate(P, sensor_points(P, [[0.55, 0.55, z] for z in zs]))
    h, s2 = 0.20, 1e-4
    for z in zs:  # sequential Kalman filter, measurement variance 1e-4 each
        K = s2 / (s2 + 1e-4)
        h, s2 = h + K * (z - h), (1 - K) * s2
    H, S2 = m.logical()
    assert np.isclose(H[5, 5], h, atol=1e-12) and np.isclose(S2[5, 5], s2, rtol=1e-9)


def test_gate_rules():
    p = ElevParams(nx=10, ny=10, res=0.1, gate=2.0, clear_margin=1e9)
    P = flat_pose()
    m = ElevationMap(p)
    m.integrate(P, sensor_points(P, [[0.55, 0.55, 0.0], [0.35, 0.55, 0.0]]))
    # sigma = 0.01: +0.05 is above the gate (reset), -0.05 below (dropped), +0.01 inside (fused)
    m.integrate(P, sensor_points(P, [[0.55, 0.55, 0.05], [0.35, 0.55, -0.05], [0.35, 0.55, 0.01]]))
    H, S2 = m.logical()
    assert np.isclose(H[5, 5], 0.05) and np.isclose(S2[5, 5], 1e-4)
    assert np.isclose(H[5, 3], 0.005) and np.isclose(S2[5, 3], 5e-5)


def test_window_move_clears_cells_that_left():
    p = ElevParams(nx=8, ny=6, res=0.1, clear_margin=1e9)
    P = flat_pose(0.45, 0.35)
    m = ElevationMap(p)
    world = [[(i + 0.5) * 0.1, (j + 0.5) * 0.1, 0.01 * i] for i in range(0, 8) for j in range(0, 6)]
    o0 = m.integrate(P, sensor_points(P, world))
    H0, _ = m.logical()
    assert o0 == (0, 0) and np.isfinite(H0).all()
    P2 = flat_pose(0.45 + 0.3, 0.35 - 0.1)
    o1 = m.integrate(P2, np.zeros((0, 3)))
    assert o1 == (3, -1)
    H1, _ = m.logical()
    # logical (c, r) of the new window is world (c + 3, r - 1)
    for r in range(6):
        for c in range(8):
            wi, wj = c + 3, r - 1
            if 0 <= wi < 8 and 0 <= wj < 6:
                assert H1[r, c] == H0[wj, wi]
            else:
                assert np.isnan(H1[r, c])


def test_raycast_clears_cells_above_the_ray():
    p = ElevParams(nx=40, ny=5, res=0.1, clear_margin=0.05, gate=1e9)  # window: world cells -20..19
    P = flat_pose(0.05, 0.25, 0.5)  # sensor above cell (0, 2) at 0.5 m
    m = ElevationMap(p)
    m.integrate(P, sensor_points(P, [[(i + 0.5) * 0.1, 0.25, 0.0] for i in range(20)]))
    m.h[2, 10] = 1.0   # a tall (stale) obstacle in the middle of the row
    m.h[2, 5] = 0.2    # low enough to stay under the ray
    m.integrate(P, sensor_points(P, [[1.95, 0.25, 0.0]]))  # one ray along the row
    # storage is indexed by world cell mod n: world column i sits at storage column i
    assert np.isnan(m.h[2, 10]) and np.isclose(m.h[2, 5], 0.2)
    assert np.isfinite(m.h[2, [6, 9, 11, 19]]).all()  # ground cells stay
    # the ray at cell 5 spans heights 0.5 * (1 - [0.45, 0.55] / 1.9): above 0.2 + 0.05


def test_raycast_cells_match_dense_sampling():
    rng = np.random.default_rng(3)
    p = ElevParams(nx=64, ny=64, res=0.1, clear_margin=-10.0, gate=1e9)  # clear every crossed cell
    for _ in range(20):
        P = flat_pose(*(rng.uniform(0.5, 2.5, 2)), 0.8)
        m = ElevationMap(p)
        m.integrate(P, np.zeros((0, 3)))
        m.h[:] = 0.0
        end = np.array([*rng.uniform(0.05, 2.95, 2), 0.0])
        m.integrate(P, sensor_points(P, [end]))
        cleared = set(zip(*np.nonzero(np.isnan(m.h))))
        sensor = P.p_B
        t = np.linspace(0, 1, 200001)[1:-1]
        xs, ys = sensor[0] + t * (end[0] - sensor[0]), sensor[1] + t * (end[1] - sensor[1])
        sampled = set(zip(np.floor(ys / 0.1).astype(int) % 64, np.floor(xs / 0.1).astype(int) % 64))
        sampled.discard((int(end[1] / 0.1) % 64, int(end[0] / 0.1) % 64))  # the point's own cell
        # dense sampling can only miss a cell the segment barely clips
        assert sampled <= cleared and len(cleared - sampled) <= 1


def test_filters():
    p = ElevParams(nx=10, ny=10, res=0.1, z_min=-0.6, z_max=0.2, clear_margin=1e9)
    P = flat_pose(0.52, 0.52, 0.5)
    m = ElevationMap(p)
    m.integrate(P, sensor_points(P, [[0.15, 0.15, 0.0], [0.25, 0.25, 0.9], [5.0, 0.15, 0.0], [0.35, 0.35, -0.3]]))
    H, _ = m.logical()
    assert np.isclose(H[1, 1], 0.0)          # kept (body height -0.5)
    assert np.isnan(H[2, 2])                 # body height +0.4 above z_max
    assert np.isnan(H[3, 3])                 # body height -0.8 below z_min
    assert np.isfinite(H).sum() == 1         # the far point is outside the window
