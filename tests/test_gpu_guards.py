"""Guard bands and failure paths of the C ABI on the GPU.

Guard bands: every workspace and output buffer handed to an entry point sits between two
4 KiB bands filled with a NaN byte pattern; after the calls (rebuild, rolling shifts, copy-out,
pose query forward / backward, the allocation-free query, lookup, SDF, inpainting, elevation
update, surrogate inference) every band must still hold the pattern, so no kernel wrote past
either end of a buffer it was given.

Failure paths, all made on the host and none of them faulting or hanging the GPU: a bounded
wait that runs out (a spin kernel of a fixed number of cycles is queued ahead of the check, so
seb_map_check with a 1 ms limit returns SEB_ERR_TIMEOUT and a later check succeeds), and the
device error word raised by a host write into the control block (SEB_ERR_DEVICE_FAULT, cleared
by that check)."""
import numpy as np
import pytest
import torch

from synthetic import bumpy_plane, fractal_steps_nan, fractal_world, lidar_scan, random_poses

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = np.frombuffer(np.array([0x7FC0DEAD], np.uint32).tobytes() * (GUARD // 4), np.uint8)
C1 = dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)


@pytest.fixture(scope="module")
def seb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


class Guarded:
    """nbytes of device memory (256-byte aligned) between two NaN-patterned guard bands."""

    def __init__(self, nbytes, fill=None):
        self.n = int(nbytes)
        self.buf = torch.empty(GUARD + ((self.n + 255) // 256) * 256 + GUARD, dtype=torch.uint8, device="cuda")
        pat = torch.from_numpy(PATTERN.copy()).cuda()
        self.buf[:GUARD] = pat
        self.buf[-GUARD:] = pat
        tail = self.buf.numel() - 2 * GUARD - self.n
        if tail > 0:  # padding up to the back band carries the pattern too
            self.buf[GUARD + self.n:-GUARD] = pat[:tail]
        if fill is not None:
            self.body.copy_(fill.reshape(-1).view(torch.uint8))
        assert self.ptr % 256 == 0

    @property
    def ptr(self):
        return self.buf.data_ptr() + GUARD

    @property
    def body(self):
        return self.buf[GUARD:GUARD + self.n]

    def view(self, dtype, shape):
        return self.body.view(dtype).view(shape)

    def intact(self):
        b = self.buf.cpu().numpy()
        tail = b.size - 2 * GUARD - self.n
        return (np.array_equal(b[:GUARD], PATTERN) and np.array_equal(b[-GUARD:], PATTERN)
                and np.array_equal(b[GUARD + self.n:b.size - GUARD], PATTERN[:tail]))


def test_map_calls_stay_inside_their_buffers(seb):
    abi = seb.abi
    cfg = dict(nx=100, ny=92, n_yaw=36, res=0.05, length=0.9, width=0.6)
    p = seb.SebParams(**cfg).c()
    nb = abi.seb_workspace_bytes(p)
    ws = Guarded(nb)
    world = torch.from_numpy(fractal_world(3, 400)).cuda()
    win = lambda o: Guarded(100 * 92 * 4, world[o[1]:o[1] + 92, o[0]:o[0] + 100].contiguous())  # noqa: E731
    st = torch.cuda.current_stream().cuda_stream
    h = abi.seb_map_create(p, ws.ptr, nb, st)
    wins = []
    try:
        o = (150, 150)
        wins.append(win(o))
        abi.seb_map_update(h, wins[-1].ptr, *o)
        for d in ((10, 0), (-7, 3), (0, -11), (13, 9), (-150, 40)):  # the last one rebuilds
            o = (min(max(o[0] + d[0], 0), 300), min(max(o[1] + d[1], 0), 300))
            wins.append(win(o))
            abi.seb_map_shift(h, wins[-1].ptr, *o)
        batch = []
        for d in ((4, 4), (-9, 2)):
            o = (o[0] + d[0], o[1] + d[1])
            batch.append((win(o), o))
        abi.seb_map_shift_batch(h, [b[0].ptr for b in batch], [b[1] for b in batch])
        wins += [b[0] for b in batch]
        out = Guarded(5 * 36 * 92 * 100 * 4)
        fl = Guarded(36 * 92 * 100)
        abi.seb_map_copy_out(h, out.ptr, fl.ptr)
        abi.seb_map_check(h, 10000)
        torch.cuda.synchronize()
        assert ws.intact() and out.intact() and fl.intact()
        assert all(w.intact() for w in wins)
        assert torch.isfinite(out.view(torch.float32, (5, 36, 92, 100))[4]).all()
        # the SE(2) lookup and the SDF of the risk channel
        g = abi.seb_map_grid(h, 4)
        n = 3000
        poses = Guarded(n * 12, torch.from_numpy(random_poses(2, n, 100, 92, 0.05, 0, origin=o)).cuda())
        val, grad, lf = Guarded(n * 4), Guarded(n * 12), Guarded(n)
        abi.seb_se2_lookup(g, poses.ptr, n, float("nan"), val.ptr, grad.ptr, lf.ptr, st)
        gv = Guarded(n * 4, torch.ones(n, device="cuda"))
        gp = Guarded(n * 12)
        abi.seb_se2_lookup_vjp(g, poses.ptr, n, gv.ptr, gp.ptr, st)
        wb = abi.seb_sdf_workspace_bytes(100, 92, 36)
        work, sdf = Guarded(wb), Guarded(36 * 92 * 100 * 4)
        abi.seb_risk_sdf(g, 1.0, 2.0, work.ptr, wb, sdf.ptr, st)
        torch.cuda.synchronize()
        for b in (ws, poses, val, grad, lf, gv, gp, work, sdf):
            assert b.intact()
    finally:
        abi.seb_map_destroy(h)


def test_query_and_inpaint_stay_inside_their_buffers(seb):
    abi = seb.abi
    p = seb.SebParams(**C1).c()
    st = torch.cuda.current_stream().cuda_stream
    e = bumpy_plane(4)
    e[30:40, 50:70] = np.nan
    elev = Guarded(e.nbytes, torch.from_numpy(e).cuda())
    for n in (777, 70_000):  # grouped and one-pose-per-thread kernels
        poses = Guarded(n * 12, torch.from_numpy(random_poses(3, n, 100, 100, 0.1, -2)).cuda())
        out, fl, sv = Guarded(n * 20), Guarded(n), Guarded(n * 4 * abi.SEB_QUERY_SAVED)
        abi.seb_query_poses(p, elev.ptr, 0, 0, poses.ptr, n, out.ptr, fl.ptr, sv.ptr, st)
        go = Guarded(n * 20, torch.randn(n, 5, device="cuda"))
        gp = Guarded(n * 12)
        abi.seb_query_poses_backward(p, elev.ptr, 0, 0, poses.ptr, sv.ptr, go.ptr, gp.ptr, n, st)
        bufs = [elev, poses, out, fl, sv, go, gp]
        if n <= abi.SEB_NOALLOC_MAX_POSES:
            o2, f2, g2 = Guarded(n * 20), Guarded(n), Guarded(n * 12)
            abi.seb_query_poses_grad_noalloc(p, elev.ptr, 0, 0, poses.ptr, n, go.ptr, o2.ptr, f2.ptr, g2.ptr, st)
            bufs += [o2, f2, g2]
        torch.cuda.synchronize()
        assert all(b.intact() for b in bufs)
    wb = abi.seb_inpaint_workspace_bytes(100, 100)
    work, res, src = Guarded(wb), Guarded(100 * 100 * 4), Guarded(100 * 100 * 8)
    abi.seb_inpaint_nearest(elev.ptr, 100, 100, 0, work.ptr, wb, res.ptr, src.ptr, st)
    torch.cuda.synchronize()
    assert work.intact() and res.intact() and src.intact() and elev.intact()
    assert torch.isfinite(res.view(torch.float32, (100, 100))).all()


def test_elevation_update_stays_inside_its_buffers(seb):
    abi = seb.abi
    ep = abi.seb_elev_params_default()
    ep.nx, ep.ny, ep.res = 96, 80, 0.05
    ep.z_min, ep.z_max = -1.0, 0.6
    max_pts = 40_000
    nb = abi.seb_elev_workspace_bytes(ep, max_pts)
    ws = Guarded(nb)
    st = torch.cuda.current_stream().cuda_stream
    h = abi.seb_elev_create(ep, max_pts, ws.ptr, nb, st)
    try:
        world = fractal_world(4, 300, res=0.05)
        sig = np.diag([0.02, 0.02, 0.02]) ** 2
        for k, (x, y, yaw) in enumerate(((6.0, 6.0, 0.3), (6.4, 6.1, 0.5))):
            R_B, p_B, R_BS, p_BS, pts = lidar_scan(10 + k, world, 0.05, x, y, yaw, n_rings=8, n_az=256, max_range=4.0)
            pts = pts[:max_pts]
            tp = Guarded(pts.nbytes, torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda())
            pose = seb.scan_pose(R_B, p_B, R_BS, p_BS, sig, sig * 0.01, sig * 0.25)
            abi.seb_elev_integrate(h, pose, tp.ptr, len(pts))
            hgt, var = Guarded(96 * 80 * 4), Guarded(96 * 80 * 4)
            abi.seb_elev_copy_out(h, hgt.ptr, var.ptr)
            torch.cuda.synchronize()
            assert ws.intact() and tp.intact() and hgt.intact() and var.intact()
    finally:
        abi.seb_elev_destroy(h)


def test_surrogate_inference_stays_inside_its_buffers(seb):
    abi = seb.abi
    p = seb.SebParams(nx=96, ny=96, n_yaw=72, res=0.05, length=0.9, width=0.6).c()
    nb = abi.seb_sur_workspace_bytes(p, 4)
    ws = Guarded(nb)
    st = torch.cuda.current_stream().cuda_stream
    h = abi.seb_sur_create(p, 4, ws.ptr, nb, st)
    try:
        abi.seb_sur_init(h, 3)
        e = fractal_steps_nan(3, 96, 96)
        elev = Guarded(e.nbytes, torch.from_numpy(e).cuda())
        out, fl, mask = Guarded(5 * 72 * 96 * 96 * 4), Guarded(72 * 96 * 96), Guarded(96 * 96)
        abi.seb_sur_infer(h, elev.ptr, 0.04, 3, 1, out.ptr, fl.ptr, mask.ptr)
        torch.cuda.synchronize()
        assert all(b.intact() for b in (ws, elev, out, fl, mask))
    finally:
        abi.seb_sur_destroy(h)


def test_bounded_wait_times_out_then_recovers(seb):
    """A spin kernel of ~2e8 cycles (about 0.1 s) sits on the map's stream ahead of the check:
    a 1 ms limit runs out (SEB_ERR_TIMEOUT, nothing is read), a 20 s limit then succeeds."""
    m = seb.SebMap(seb.SebParams(**dict(C1, nx=48, ny=48)))
    m.update(torch.from_numpy(bumpy_plane(1, 48, 48)).cuda())
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)
    with pytest.raises(seb.abi.SebError) as ei:
        m.check(timeout_ms=1)
    assert ei.value.status == seb.abi.SEB_ERR_TIMEOUT
    assert m.check(timeout_ms=20000) is not None


def test_device_error_word_is_reported_and_cleared(seb):
    """The host raises the control block's error word (the word a kernel sets on a launch-shape
    mismatch); seb_map_check reports SEB_ERR_DEVICE_FAULT with the word, clears it, and the next
    check is clean."""
    m = seb.SebMap(seb.SebParams(**dict(C1, nx=48, ny=48)))
    m.update(torch.from_numpy(bumpy_plane(1, 48, 48)).cuda())
    m.check()
    m.workspace[0:4].view(torch.int32).fill_(0x40)
    with pytest.raises(seb.abi.SebError) as ei:
        m.check()
    assert ei.value.status == seb.abi.SEB_ERR_DEVICE_FAULT and "0x40" in str(ei.value)
    m.check()
    m.update(torch.from_numpy(bumpy_plane(2, 48, 48)).cuda())
    m.check()
