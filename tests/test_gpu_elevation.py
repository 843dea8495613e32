"""GPU parity of the elevation-map update (seb_elev_integrate) against the FP64 reference in
oracle/elevation.py on seeded synthetic LiDAR scans of a synthetic world, over several scans
with a moving window (the reference stores float32 like the map, so both take the gate and
clearing decisions on the same stored values)."""
import numpy as np
import pytest

from oracle.elevation import ElevationMap as RefMap, ElevParams, ScanPose
from synthetic import fractal_world, lidar_scan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES = 0.05
SIGMA_S = np.diag([0.02, 0.02, 0.02]) ** 2
SIGMA_R = np.diag([0.004, 0.004, 0.002]) ** 2
SIGMA_B = np.diag([0.01, 0.01, 0.01]) ** 2


@pytest.fixture(scope="module")
def seb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def run(seb, nx, ny, path, clear_margin=0.05, gate=2.5, n_az=256, n_rings=16, max_range=5.0):
    world = fractal_world(4, 500, res=RES)
    ref = RefMap(ElevParams(nx=nx, ny=ny, res=float(np.float32(RES)), z_min=-1.0, z_max=0.6, gate=gate,
                            clear_margin=clear_margin), store_f32=True)
    m = seb.ElevationMap(nx, ny, RES, 100_000, z_min=-1.0, z_max=0.6, gate=gate, clear_margin=clear_margin)
    stats = []
    for k, (x, y, yaw) in enumerate(path):
        R_B, p_B, R_BS, p_BS, pts = lidar_scan(10 + k, world, RES, x, y, yaw, n_rings=n_rings, n_az=n_az,
                                               max_range=max_range)
        pose = seb.scan_pose(R_B, p_B, R_BS, p_BS, SIGMA_S, SIGMA_R, SIGMA_B)
        m.integrate(pose, torch.from_numpy(pts).cuda())
        ref.integrate(ScanPose(f32(R_B), f32(p_B), f32(R_BS), f32(p_BS), f32(SIGMA_S), f32(SIGMA_R), f32(SIGMA_B)),
                      pts.astype(np.float64))
        h, v = m.outputs()
        h, v = h.cpu().numpy(), v.cpu().numpy()
        rh, rv = ref.logical()
        view = m.view()
        assert (view.origin_i, view.origin_j) == ref.origin
        assert np.array_equal(np.isnan(h), np.isnan(rh)), f"scan {k}: known cells differ"
        fin = ~np.isnan(rh)
        assert np.abs(h[fin] - rh[fin]).max() <= 1e-5
        assert (np.abs(v[fin] - rv[fin]) <= 1e-6 * rv[fin] + 1e-12).all()
        stats.append(int(fin.sum()))
    return stats


def test_scans_along_a_path(seb):
    path = [(10.0, 10.0, 0.2), (10.4, 10.1, 0.3), (10.9, 10.3, 0.5), (11.2, 10.9, 1.0)]
    known = run(seb, 160, 120, path)
    assert known[-1] > known[0] > 300  # the map fills up as the robot moves


def test_window_jump_and_odd_sizes(seb):
    # a jump farther than the window clears everything; odd window sides
    path = [(12.0, 12.0, 0.0), (20.0, 7.5, 2.0), (20.2, 7.4, 2.1)]
    run(seb, 97, 61, path)


def test_raycast_heavy_margin(seb):
    # a negative margin clears every crossed cell that holds a height: stresses the cell walk
    path = [(9.0, 14.0, 0.0), (9.05, 14.02, 0.1)]
    run(seb, 128, 128, path, clear_margin=-5.0)


def test_bad_calls(seb):
    m = seb.ElevationMap(32, 32, RES, 10)
    pose = seb.scan_pose(np.eye(3), [0, 0, 0.5], np.eye(3), [0, 0, 0], SIGMA_S, SIGMA_R, SIGMA_B)
    with pytest.raises(seb.abi.SebError):
        m.integrate(pose, torch.zeros((11, 3), device="cuda"))  # more than max_points
    m.integrate(pose, torch.zeros((0, 3), device="cuda"))
    h, _ = m.outputs()
    assert torch.isnan(h).all()
