"""GPU parity of the trilinear SE(2) lookup (seb_se2_lookup / seb_se2_lookup_vjp) against the
FP64 reference in oracle/se2_lookup.py on the same seeded grids and poses, and the lookup of a
map channel against the exact continuous query."""
import math

import numpy as np
import pytest

from oracle.se2_lookup import se2_lookup as ref_lookup
from synthetic import lookup_poses, random_se2_grid, tilted_plane

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, NY, NX = 72, 50, 61
RES = 0.05
RES_F = float(np.float32(RES))  # seb_grid.res is float32: the oracle reads the same value
ORIGIN = (-20, 35)
RING = (7, 13)
VAL_TOL = 1e-5   # FP32 blend of N(0, 1) values: a few ulps of the largest corner
GRAD_TOL = 2e-4  # derivatives in grid units (~1e-6) scaled by 1/res = 20 or K/(2 pi) = 11.5,
GRAD_RTOL = 1e-5  # plus FP32 rounding relative to the derivative itself


@pytest.fixture(scope="module")
def seb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


def special_poses():
    """Nodes, the far corner, faces, the yaw wrap, a huge yaw and non-finite entries."""
    def w(c, r, k):
        return [(ORIGIN[0] + c + 0.5) * RES, (ORIGIN[1] + r + 0.5) * RES, 2 * math.pi * k / K]
    P = [w(0, 0, 0), w(NX - 1, NY - 1, K - 1), w(NX - 1, 3, 5.5), w(2.5, NY - 1, 7.25), w(10.25, 20.75, K - 0.5),
         w(10.25, 20.75, -0.5), w(3, 4, 2e5), w(3, 4, 1.9e4), w(4.5, 6.5, -1e4 * K / (2 * math.pi) + 0.25), w(5, 5, 3)]
    P[-1][0] = float("nan")
    P.append(w(5, 5, 3))
    P[-1][2] = float("inf")
    return np.array(P, np.float32)


def compare(seb, grid_np, poses_np, fill, nan_frac=0.0):
    dev = torch.from_numpy(grid_np).cuda()
    g = seb.SE2Grid.from_tensor(dev, RES, ORIGIN, RING)
    p = torch.from_numpy(poses_np).cuda()
    val, grad, fl = seb.se2_lookup(g, p, fill=fill, with_grad=True)
    rv, rg, rf = ref_lookup(grid_np.astype(np.float64), poses_np.astype(np.float64), RES_F, ORIGIN, RING, fill)
    val, grad, fl = val.cpu().numpy(), grad.cpu().numpy(), fl.cpu().numpy()
    assert np.array_equal(fl, rf)
    fin = np.isfinite(rv)
    assert np.array_equal(np.isfinite(val), fin)
    assert np.abs(val[fin] - rv[fin]).max() <= VAL_TOL
    # gradients: a pose within 1e-4 of a cell face may take either side's derivative
    P = poses_np.astype(np.float64)
    u = P[:, 0] / RES_F - ORIGIN[0] - 0.5
    v = P[:, 1] / RES_F - ORIGIN[1] - 0.5
    wy = P[:, 2] * K / (2 * math.pi)

    def off_face(q):
        with np.errstate(invalid="ignore"):
            f = q - np.floor(q)
            return (f > 1e-4) & (f < 1 - 1e-4)

    ok = fin & off_face(u) & off_face(v) & off_face(wy)
    assert (np.abs(grad[ok] - rg[ok]) <= GRAD_TOL + GRAD_RTOL * np.abs(rg[ok])).all()
    assert (grad[rf == 1][~np.isnan(grad[rf == 1]).any(1)] == 0).all() or nan_frac > 0
    return g, p, rg


def test_random_grid_parity(seb):
    grid = random_se2_grid(11, K, NY, NX)
    poses = np.concatenate([lookup_poses(12, 200_000, NX, NY, RES, ORIGIN), special_poses()])
    compare(seb, grid, poses, fill=3.5)


def test_nan_corners_and_default_fill(seb):
    grid = random_se2_grid(13, K, NY, NX, nan_frac=0.02)
    poses = lookup_poses(14, 50_000, NX, NY, RES, ORIGIN)
    compare(seb, grid, poses, fill=float("nan"), nan_frac=0.02)


def test_vjp_and_autograd(seb):
    grid = random_se2_grid(15, K, NY, NX)
    poses = lookup_poses(16, 20_000, NX, NY, RES, ORIGIN)
    g, p, rg = compare(seb, grid, poses, fill=0.0)
    gv = torch.from_numpy(np.random.default_rng(17).normal(size=len(poses)).astype(np.float32)).cuda()
    gp = torch.empty_like(p)
    seb.abi.seb_se2_lookup_vjp(g.g, p.data_ptr(), len(poses), gv.data_ptr(), gp.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    _, grad, _ = seb.se2_lookup(g, p, with_grad=True)
    assert torch.allclose(gp, gv[:, None] * grad, rtol=1e-6, atol=1e-6)
    q = p.clone().requires_grad_(True)
    val = seb.SE2Lookup.apply(q, g, 0.0)
    (val * gv).sum().backward()
    assert torch.allclose(q.grad, gp, rtol=1e-6, atol=1e-6)


def test_degenerate_calls(seb):
    grid = torch.zeros((4, 1, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(seb.abi.SebError):
        seb.se2_lookup(seb.SE2Grid.from_tensor(grid, RES), torch.zeros((3, 3), device="cuda"))
    ok = seb.SE2Grid.from_tensor(torch.zeros((4, 2, 5), device="cuda"), RES)
    val, _, fl = seb.se2_lookup(ok, torch.zeros((0, 3), device="cuda"))
    assert val.numel() == 0 and fl.numel() == 0
    m = seb.SebMap(seb.SebParams(nx=20, ny=20, n_yaw=8, res=0.1, length=0.6, width=0.4))
    with pytest.raises(seb.abi.SebError):
        seb.SE2Grid.from_map(m, 4)


def test_max_yaw_bins(seb):
    """The interface limits: 4096 yaw bins with yaws up to |1e4| rad (the yaw reduction stays
    exact there), against the FP64 reference; 4097 bins are rejected."""
    K2, ny, nx = 4096, 6, 7
    grid = random_se2_grid(31, K2, ny, nx)
    rng = np.random.default_rng(32)
    n = 50_000
    P = np.stack([(ORIGIN[0] + rng.uniform(0, nx - 1, n) + 0.5) * RES,
                  (ORIGIN[1] + rng.uniform(0, ny - 1, n) + 0.5) * RES,
                  rng.uniform(-1e4, 1e4, n)], 1).astype(np.float32)
    ring = (3, 2)
    g = seb.SE2Grid.from_tensor(torch.from_numpy(grid).cuda(), RES, ORIGIN, ring)
    val, grad, fl = seb.se2_lookup(g, torch.from_numpy(P).cuda(), fill=0.0, with_grad=True)
    rv, rg, rf = ref_lookup(grid.astype(np.float64), P.astype(np.float64), RES_F, ORIGIN, ring, 0.0)
    val, grad, fl = val.cpu().numpy(), grad.cpu().numpy(), fl.cpu().numpy()
    assert np.array_equal(fl, rf) and (rf == 0).mean() > 0.99
    assert np.abs(val - rv).max() <= VAL_TOL
    Pd = P.astype(np.float64)
    q = [Pd[:, 0] / RES_F - ORIGIN[0] - 0.5, Pd[:, 1] / RES_F - ORIGIN[1] - 0.5, Pd[:, 2] * K2 / (2 * math.pi)]
    ok = np.ones(n, bool)
    for c in q:
        f = c - np.floor(c)
        ok &= (f > 1e-4) & (f < 1 - 1e-4)
    # a derivative in grid units carries ~1e-6 (a few ulps of the O(1) values); in world units it
    # scales by 1 / res for x, y and by K / (2 pi) = 652 for the yaw
    scale = np.array([1 / RES_F, 1 / RES_F, K2 / (2 * math.pi)])
    assert (np.abs(grad[ok] - rg[ok]) <= 1e-5 * scale + GRAD_RTOL * np.abs(rg[ok])).all()
    with pytest.raises(seb.abi.SebError):
        bad = seb.SE2Grid.from_tensor(torch.zeros((4097, 2, 2), device="cuda"), RES)
        seb.se2_lookup(bad, torch.zeros((3, 3), device="cuda"))


def test_map_channel_vs_exact_query(seb):
    """On a tilted plane the bilinear z is exact and pitch/roll differ from the exact continuous
    query by the yaw discretisation only: |error| <= (2 pi / K)^2 / 8 * max |d^2/dyaw^2|,
    which for a plane of slope s (pitch ~ -atan(s cos(yaw - a))) stays below 1.5 s."""
    from paper_2503_02412_gb300.query import query_poses
    from synthetic import random_poses

    Kq, n = 36, 100
    p = seb.SebParams(nx=n, ny=n, n_yaw=Kq, res=0.1, length=0.6, width=0.4)
    slope = math.tan(math.radians(12))
    e = torch.from_numpy(tilted_plane(n, n, 0.1, slope * 0.8, slope * 0.6, 1.0, origin=(5, -7)).astype(np.float32)).cuda()
    m = seb.SebMap(p)
    m.update(e, (5, -7))
    poses = torch.from_numpy(random_poses(3, 20_000, n, n, 0.1, 6, origin=(5, -7))).cuda()
    exact, _ = query_poses(p, e, poses, origin=(5, -7))
    bound = (2 * math.pi / Kq) ** 2 / 8 * 1.5 * slope + 1e-4
    for ch, tol in ((0, 1e-4), (1, bound), (2, bound)):
        val, _, fl = seb.se2_lookup(seb.SE2Grid.from_map(m, ch), poses)
        assert (fl == 0).all()
        err = (val - exact[:, ch]).abs().max().item()
        assert err <= tol, (ch, err, tol)
