"""GPU parity of the continuous-pose query (forward) and of its hand-written adjoint
(backward) against the FP64 oracle and finite differences, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from synthetic import bumpy_plane, random_poses, tilted_plane

from .parity import compare

pytestmark = pytest.mark.gpu

C1 = dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)


@pytest.fixture(scope="module")
def seb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300 import query  # noqa: F401

    return seb


def fwd(seb, cfg, elev, poses, origin=(0, 0)):
    from paper_2503_02412_gb300.query import query_poses

    p = seb.SebParams(**cfg)
    te = torch.from_numpy(np.ascontiguousarray(elev, np.float32)).cuda()
    tp = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    out, fl = query_poses(p, te, tp, origin)
    return out.cpu().numpy(), fl.cpu().numpy()


@pytest.mark.parametrize("n", [1, 33, 4096])
def test_forward_matches_oracle(seb, n):
    e = bumpy_plane(1)
    poses = random_poses(5, n, 100, 100, 0.1, 5, origin=(-20, 30))
    g, gf = fwd(seb, C1, e, poses, (-20, 30))
    r, rf = oracle.query_poses(oracle.OracleParams(**C1), e.astype(np.float64), poses.astype(np.float64), (-20, 30))
    compare(g, gf, r, rf, label="query fwd")


def _ambiguous_poses(seb, cfg, poses, origin=(0, 0), eps=1e-4):
    """Poses with a lattice point whose grid coordinate lies within eps cells of a grid line:
    there floor() of the FP32 coordinate may differ from the FP64 one, and with it the
    point's bilinear cell (and whether that cell touches an unknown cell or the window edge)."""
    lat = np.array(seb.abi.seb_footprint_table(seb.SebParams(**cfg).c(), 0), np.float64)
    P = poses.astype(np.float32).astype(np.float64)
    res = float(np.float32(cfg["res"]))
    c, s = np.cos(P[:, 2:3]), np.sin(P[:, 2:3])
    u = P[:, 0:1] / res - origin[0] - 0.5 + c * lat[:, 0] - s * lat[:, 1]
    v = P[:, 1:2] / res - origin[1] - 0.5 + s * lat[:, 0] + c * lat[:, 1]
    near = lambda t: np.abs(t - np.round(t)) < eps  # noqa: E731
    return (near(u) | near(v)).any(axis=1)


def test_forward_near_edges_and_unknown(seb):
    e = bumpy_plane(2)
    e[40:55, 40:60] = np.nan
    poses = random_poses(6, 4000, 100, 100, 0.1, -3)  # some poses partly outside the window
    g, gf = fwd(seb, C1, e, poses)
    r, rf = oracle.query_poses(oracle.OracleParams(**C1), e.astype(np.float64), poses.astype(np.float64))
    # the UNKNOWN bit may differ only where a lattice point sits on a grid line (FP32 vs FP64
    # floor of its grid coordinate); every such pose must be one of those
    same = (gf & 1) == (rf & 1)
    amb = _ambiguous_poses(seb, C1, poses)
    assert not (~same & ~amb).any(), np.flatnonzero(~same & ~amb)[:8]
    print(f"UNKNOWN bit differs on {int((~same).sum())} of {int(amb.sum())} poses with a point on a grid line")
    compare(g[same], gf[same], r[same], rf[same], label="query edges")
    assert (gf & 1).sum() > 100


def test_grid_equality_at_cell_centres_yaw0(seb):
    e = bumpy_plane(3)
    p = seb.SebParams(**C1)
    m = seb.SebMap(p)
    m.update(torch.from_numpy(e).cuda(), (0, 0))
    out, fl = m.outputs()
    cs = np.arange(6, 94)
    cc, rr = np.meshgrid(cs, cs)
    poses = np.stack([(cc.ravel() + 0.5) * 0.1, (rr.ravel() + 0.5) * 0.1, np.zeros(cc.size)], 1)
    g, gf = fwd(seb, C1, e, poses)
    want = out.cpu().numpy()[:, 0, rr.ravel(), cc.ravel()].T
    ok = np.isfinite(want[:, 0])
    assert np.abs(g[ok] - want[ok]).max() < 2e-5


def test_plane_closed_form_continuous_yaw(seb):
    a, b = 0.12, -0.2
    e = tilted_plane(100, 100, 0.1, a, b, 0.3).astype(np.float32)
    poses = random_poses(7, 2000, 100, 100, 0.1, 6)
    g, gf = fwd(seb, C1, e, poses)
    th = poses[:, 2].astype(np.float64)
    p = a * np.cos(th) + b * np.sin(th)
    q = b * np.cos(th) - a * np.sin(th)
    assert np.abs(g[:, 1] - np.arcsin(p / np.sqrt((1 + q * q) * (1 + p * p + q * q)))).max() < 2e-5
    assert np.abs(g[:, 2] - np.arctan(q)).max() < 2e-5
    assert np.abs(g[:, 3]).max() < 1e-6


def _bwd(seb, cfg, elev, poses, gout, use_saved=True, origin=(0, 0)):
    from paper_2503_02412_gb300.query import QueryPoses

    p = seb.SebParams(**cfg)
    te = torch.from_numpy(np.ascontiguousarray(elev, np.float32)).cuda()
    tp = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda().requires_grad_(True)
    out, fl = QueryPoses.apply(tp, te, p, origin)
    (out * torch.from_numpy(gout).float().cuda()).sum().backward()
    return tp.grad.cpu().numpy(), out.detach().cpu().numpy(), fl.cpu().numpy()


def test_backward_matches_oracle_adjoint(seb):
    cfg = dict(C1, kappa_max=1.0, phi_x_max=1.4, phi_y_max=1.4)  # keep risk on its smooth branch
    e = bumpy_plane(4)
    poses = random_poses(8, 4096, 100, 100, 0.1, 5)
    rng = np.random.default_rng(0)
    gout = rng.normal(size=(4096, 5))
    g, out, fl = _bwd(seb, cfg, e, poses, gout)
    r = oracle.query_poses_vjp(oracle.OracleParams(**cfg), e.astype(np.float64), poses.astype(np.float64), gout)
    ok = (fl & 5) == 0
    assert ok.mean() > 0.99
    # Element-wise: relative error <= 1e-3 wherever |g| is at least 1e-2 of the component's
    # largest |g| over the batch; below that floor, absolute error <= 1e-3 of the floor (a
    # relative bound there would ask FP32 for digits that cancellation in the adjoint removes).
    scale = np.abs(r[ok]).max(axis=0)
    floor = 1e-2 * scale
    big = ok[:, None] & (np.abs(r) >= floor)
    small = ok[:, None] & ~big
    rel = np.abs(g - r) / np.maximum(np.abs(r), 1e-300)
    assert big.mean() > 0.8
    assert rel[big].max() <= 1e-3, rel[big].max()
    assert (np.abs(g - r)[small] <= (1e-3 * floor * np.ones_like(r))[small]).all()


def test_backward_default_thresholds_branches(seb):
    e = bumpy_plane(5)
    poses = random_poses(9, 4096, 100, 100, 0.1, 5)
    gout = np.random.default_rng(1).normal(size=(4096, 5))
    g, out, fl = _bwd(seb, C1, e, poses, gout)
    r = oracle.query_poses_vjp(oracle.OracleParams(**C1), e.astype(np.float64), poses.astype(np.float64), gout)
    ro, rf = oracle.query_poses(oracle.OracleParams(**C1), e.astype(np.float64), poses.astype(np.float64))
    from .parity import near_threshold

    ok = ((fl & 5) == 0) & (fl == rf) & ~near_threshold(ro, margin=1e-4)
    scale = np.abs(r[ok]).max(axis=0)
    assert (np.abs(g - r)[ok] / scale).max() < 1e-3


def test_backward_saved_equals_recompute(seb):
    from paper_2503_02412_gb300 import abi

    e = bumpy_plane(6)
    n = 1000
    poses = torch.from_numpy(random_poses(10, n, 100, 100, 0.1, 5)).cuda()
    te = torch.from_numpy(e).cuda()
    p = seb.SebParams(**C1).c()
    st = torch.cuda.current_stream().cuda_stream
    out = torch.empty(n, 5, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    sv = torch.empty(n, 16, device="cuda")
    abi.seb_query_poses(p, te.data_ptr(), 0, 0, poses.data_ptr(), n, out.data_ptr(), fl.data_ptr(), sv.data_ptr(), st)
    go = torch.randn(n, 5, device="cuda")
    a = torch.empty(n, 3, device="cuda")
    b = torch.empty(n, 3, device="cuda")
    abi.seb_query_poses_backward(p, te.data_ptr(), 0, 0, poses.data_ptr(), sv.data_ptr(), go.data_ptr(), a.data_ptr(), n, st)
    abi.seb_query_poses_backward(p, te.data_ptr(), 0, 0, poses.data_ptr(), 0, go.data_ptr(), b.data_ptr(), n, st)
    assert torch.allclose(a, b, rtol=1e-5, atol=1e-6)


def test_backward_matches_fp32_central_differences(seb):
    """Central differences of the GPU forward (h = 1e-3 m / rad per the FD recipe), on poses whose
    footprint points stay clear of bilinear grid lines over +-h and whose risk branch cannot
    switch within h."""
    cfg = dict(C1, kappa_max=1.0, phi_x_max=1.4, phi_y_max=1.4)
    e = bumpy_plane(7).astype(np.float32)
    n = 20000
    poses = random_poses(11, n, 100, 100, 0.1, 6).astype(np.float32)
    lat = np.array(seb.abi.seb_footprint_table(seb.SebParams(**cfg).c(), 0), np.float64) * 0.1
    h = 1e-3
    reach = h * (1 + np.hypot(lat[:, 0], lat[:, 1]).max()) / 0.1  # cells a point can move
    th = poses[:, 2:3].astype(np.float64)
    X = poses[:, 0:1] + np.cos(th) * lat[:, 0] - np.sin(th) * lat[:, 1]
    Y = poses[:, 1:2] + np.sin(th) * lat[:, 0] + np.cos(th) * lat[:, 1]
    fx = np.abs(((X / 0.1 - 0.5) + 0.5) % 1.0 - 0.5)
    fy = np.abs(((Y / 0.1 - 0.5) + 0.5) % 1.0 - 0.5)
    clear = (np.minimum(fx, fy) > 2 * reach).all(axis=1)
    assert clear.sum() > 50
    poses = poses[clear]
    gout = np.random.default_rng(2).normal(size=(len(poses), 5))
    g, out, fl = _bwd(seb, cfg, e, poses, gout)
    fd = np.zeros_like(g, dtype=np.float64)
    for j in range(3):
        pp, pm = poses.copy(), poses.copy()
        pp[:, j] += np.float32(h)
        pm[:, j] -= np.float32(h)
        op, _ = fwd(seb, cfg, e, pp)
        om, _ = fwd(seb, cfg, e, pm)
        step = (pp[:, j].astype(np.float64) - pm[:, j].astype(np.float64))
        fd[:, j] = ((op.astype(np.float64) - om) * gout).sum(1) / step
    ok = (fl & 5) == 0
    scale = np.abs(fd[ok]).max(axis=0)
    err = np.abs(g - fd)[ok] / scale
    assert np.percentile(err, 99) < 1e-2
    assert np.median(err) < 1e-3


def test_large_batch_and_empty(seb):
    from paper_2503_02412_gb300.query import query_poses

    e = torch.from_numpy(bumpy_plane(8)).cuda()
    p = seb.SebParams(**C1)
    out, fl = query_poses(p, e, torch.empty(0, 3, device="cuda"))
    assert out.shape == (0, 5)
    n = 1 << 20
    poses = torch.from_numpy(random_poses(12, n, 100, 100, 0.1, 5)).cuda()
    out, fl = query_poses(p, e, poses)
    idx = np.random.default_rng(3).integers(0, n, 3000)
    r, rf = oracle.query_poses(oracle.OracleParams(**C1), e.cpu().numpy().astype(np.float64),
                               poses.cpu().numpy()[idx].astype(np.float64))
    compare(out.cpu().numpy()[idx], fl.cpu().numpy()[idx], r, rf, label="1M sample")


@pytest.mark.parametrize("side", [100, 160])
def test_one_pose_per_thread_kernels(seb, side):
    """Batches of 65,536 poses or more take the one-pose-per-thread kernels (a 100 x 100 FP32
    window, 40 KB, is copied into each CTA's shared memory; a 160 x 160 one, 100 KB, is read from
    global memory): their backward against the FP64 oracle adjoint on a sample, the saved state
    against recomputation, and both directions against the grouped kernels that the first 4,096
    poses take when run alone (the moment sums are added in a different order, so agreement is to
    FP32 rounding)."""
    from paper_2503_02412_gb300 import abi

    cfg = dict(C1, nx=side, ny=side, kappa_max=1.0, phi_x_max=1.4, phi_y_max=1.4)
    e = bumpy_plane(13, side, side)
    n = 70_000
    poses = random_poses(14, n, side, side, 0.1, 5)
    gout = np.random.default_rng(15).normal(size=(n, 5))
    g, out, fl = _bwd(seb, cfg, e, poses, gout)
    gs, outs, fls = _bwd(seb, cfg, e, poses[:4096], gout[:4096])
    ok = ((fl[:4096] & 5) == 0) & (fl[:4096] == fls)
    assert ok.mean() > 0.9
    assert np.abs(out[:4096][ok] - outs[ok]).max() < 2e-5
    scale = np.abs(gs[ok]).max(axis=0)
    assert (np.abs(g[:4096] - gs)[ok] / scale).max() < 1e-3
    idx = np.random.default_rng(16).integers(0, n, 2000)
    r = oracle.query_poses_vjp(oracle.OracleParams(**cfg), e.astype(np.float64), poses[idx].astype(np.float64),
                               gout[idx])
    sel = (fl[idx] & 5) == 0
    sc = np.abs(r[sel]).max(axis=0)
    assert (np.abs(g[idx] - r)[sel] / sc).max() < 1e-3
    # saved state versus recomputation in the backward
    p = seb.SebParams(**cfg).c()
    te = torch.from_numpy(e).cuda()
    tp = torch.from_numpy(poses).cuda()
    st = torch.cuda.current_stream().cuda_stream
    o = torch.empty(n, 5, device="cuda")
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    sv = torch.empty(n, 16, device="cuda")
    abi.seb_query_poses(p, te.data_ptr(), 0, 0, tp.data_ptr(), n, o.data_ptr(), f.data_ptr(), sv.data_ptr(), st)
    go = torch.from_numpy(gout.astype(np.float32)).cuda()
    a = torch.empty(n, 3, device="cuda")
    b = torch.empty(n, 3, device="cuda")
    abi.seb_query_poses_backward(p, te.data_ptr(), 0, 0, tp.data_ptr(), sv.data_ptr(), go.data_ptr(), a.data_ptr(), n, st)
    abi.seb_query_poses_backward(p, te.data_ptr(), 0, 0, tp.data_ptr(), 0, go.data_ptr(), b.data_ptr(), n, st)
    assert torch.allclose(a, b, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("dtype,side,n", [(torch.bfloat16, 100, 4096), (torch.bfloat16, 180, 70_000),
                                          (torch.float16, 100, 70_000), (torch.float16, 180, 4096)])
def test_reduced_precision_windows(seb, dtype, side, n):
    """BF16 / FP16 windows: the query widens each corner height to FP32, so it matches the FP64
    oracle run on the stored (rounded) heights.  4,096 poses take the grouped kernels, 70,000 the
    one-pose-per-thread kernels (a 100 x 100 or 180 x 180 window of 2-byte heights, 20 or 65 KB,
    is copied into shared memory)."""
    from paper_2503_02412_gb300.query import query_poses

    cfg = dict(C1, nx=side, ny=side)
    p = seb.SebParams(**cfg, elev_dtype=dtype)
    te = torch.from_numpy(bumpy_plane(21, side, side)).cuda().to(dtype)
    stored = te.float().cpu().numpy().astype(np.float64)
    poses = random_poses(22, n, side, side, 0.1, 5)
    out, fl = query_poses(p, te, torch.from_numpy(poses).cuda())
    idx = np.random.default_rng(23).integers(0, n, min(n, 3000))
    r, rf = oracle.query_poses(oracle.OracleParams(**cfg), stored, poses[idx].astype(np.float64))
    s = compare(out.cpu().numpy()[idx], fl.cpu().numpy()[idx], r, rf, label=f"{dtype} query")
    assert s["assessed"] > 0.5 * len(idx)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_reduced_precision_backward(seb, dtype):
    """The adjoint on a BF16 / FP16 window (70,000 poses: the one-pose-per-thread kernels with the
    window in shared memory) against the FP64 oracle adjoint on the stored heights."""
    from paper_2503_02412_gb300.query import QueryPoses

    cfg = dict(C1, kappa_max=1.0, phi_x_max=1.4, phi_y_max=1.4)
    p = seb.SebParams(**cfg, elev_dtype=dtype)
    te = torch.from_numpy(bumpy_plane(24)).cuda().to(dtype)
    stored = te.float().cpu().numpy().astype(np.float64)
    n = 70_000
    poses = random_poses(25, n, 100, 100, 0.1, 5)
    gout = np.random.default_rng(26).normal(size=(n, 5))
    tp = torch.from_numpy(poses).cuda().requires_grad_(True)
    out, fl = QueryPoses.apply(tp, te, p, (0, 0))
    (out * torch.from_numpy(gout).float().cuda()).sum().backward()
    g, fl = tp.grad.cpu().numpy(), fl.cpu().numpy()
    idx = np.random.default_rng(27).integers(0, n, 2000)
    r = oracle.query_poses_vjp(oracle.OracleParams(**cfg), stored, poses[idx].astype(np.float64), gout[idx])
    sel = (fl[idx] & 5) == 0
    assert sel.mean() > 0.8
    sc = np.abs(r[sel]).max(axis=0)
    assert (np.abs(g[idx] - r)[sel] / sc).max() < 1e-3
