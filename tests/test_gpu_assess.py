"""GPU parity of the SE(2) grid assessment (Algorithm 1 for every cell and yaw bin) against
the FP64 oracle, through the C ABI.  Sizes: the small map and the full 400 x 400 x 72 map
(both complete, element by element), plus ragged, degenerate and rolling cases."""
import numpy as np
import pytest
import torch

import oracle
from synthetic import bumpy_plane, fractal_steps_nan, fractal_world, shift_sequence, tilted_plane

from .parity import compare, grid_to_rows

pytestmark = pytest.mark.gpu

C1 = dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4)
C2 = dict(nx=400, ny=400, n_yaw=72, res=0.05, length=0.9, width=0.6)


@pytest.fixture(scope="module")
def seb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    assert torch.cuda.is_available()
    return seb


def run_map(seb, cfg, elev, origin=(0, 0), **kw):
    m = seb.SebMap(seb.SebParams(**cfg, **kw))
    dt = kw.get("elev_dtype", torch.float32)
    m.update(torch.from_numpy(np.ascontiguousarray(elev)).to("cuda", dtype=dt), origin)
    out, fl = m.outputs()
    counters = m.check()
    return m, out.cpu().numpy(), fl.cpu().numpy(), counters


def oracle_grid(cfg, elev, origin=(0, 0), **kw):
    return oracle.assess_grid(oracle.OracleParams(**cfg, **kw), np.asarray(elev, np.float64), origin, with_gap=True)


def check(out, fl, ref, label):
    o, f = grid_to_rows(out, fl)
    r, rf, g = grid_to_rows(*ref)
    return compare(o, f, r, rf, label=label, gap=g)


def test_small_map_every_cell(seb):
    e = bumpy_plane(0)
    _, out, fl, _ = run_map(seb, C1, e, (17, -4))
    s = check(out, fl, oracle_grid(C1, e, (17, -4)), "c1")
    assert s["assessed"] > 0.95 * s["n"]


def test_full_map_every_cell(seb):
    e = fractal_steps_nan(0)
    _, out, fl, (n64, ndeg) = run_map(seb, C2, e)
    s = check(out, fl, oracle_grid(C2, e), "c2")
    assert s["assessed"] > 0.8 * s["n"]
    assert ((fl & 1) != 0).mean() > 0.01  # the NaN blobs produce unknown cells


@pytest.mark.parametrize("cfg", [C1, dict(C2, nx=96, ny=96)])
@pytest.mark.parametrize("ab", [(0.2, -0.1), (-0.25, 0.05)])
def test_tilted_plane_closed_form(seb, cfg, ab):
    a, b = ab
    nx, ny = cfg["nx"], cfg["ny"]
    e = tilted_plane(nx, ny, cfg["res"], a, b, 0.4, (3, 9)).astype(np.float32)
    _, out, fl, _ = run_map(seb, cfg, e, (3, 9))
    K = cfg["n_yaw"]
    th = 2 * np.pi * np.arange(K) / K
    p = a * np.cos(th) + b * np.sin(th)
    q = b * np.cos(th) - a * np.sin(th)
    pitch = np.arcsin(p / np.sqrt((1 + q * q) * (1 + p * p + q * q)))
    roll = np.arctan(q)
    R = 12
    sl = (slice(None), slice(R, ny - R), slice(R, nx - R))
    assert np.abs(out[1][sl] - pitch[:, None, None]).max() < 2e-5
    assert np.abs(out[2][sl] - roll[:, None, None]).max() < 2e-5
    assert np.abs(out[3][sl]).max() < 1e-6
    xs = (3 + np.arange(nx) + 0.5) * cfg["res"]
    ys = (9 + np.arange(ny) + 0.5) * cfg["res"]
    zc = a * xs[None, :] + b * ys[:, None] + 0.4
    assert np.abs(out[0][sl] - zc[None, R:-R, R:-R]).max() < 1e-5


def near_degenerate_map(nx=384, ny=64, res=0.05, deltas=(1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7), base=0.3):
    """Checkerboard stripes z = base +- A whose footprint covariance at yaw 0 (19 x 13 cells of the
    0.9 x 0.6 m footprint at 0.05 m) is diag(lambda_xx, lambda_yy, A^2 (1 - 1/247^2)), with A
    chosen so that the z variance sits a relative delta below lambda_yy: the two smallest
    eigenvalues are then lambda_yy (1 - delta) and lambda_yy, a relative eigen-gap of about
    0.24 delta (at yaws 0, pi/2, pi, 3 pi/2, where the footprint's row and column sets are the
    same).  The cross terms vanish by symmetry, so the normal is vertical, and any FP32 rounding of
    the moments tilts it by up to ||dC|| / gap."""
    lam_yy = res * res * np.mean(np.arange(-6, 7) ** 2.0)
    z = np.zeros((ny, nx))
    w = nx // len(deltas)
    jj, ii = np.mgrid[0:ny, 0:nx]
    cb = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    for s, d in enumerate(deltas):
        a = np.sqrt(lam_yy * (1 - d) / (1 - 1 / 247.0 ** 2))
        z[:, s * w:(s + 1) * w] = base + a * cb[:, s * w:(s + 1) * w]
    return z.astype(np.float32)


def test_near_degenerate_footprints_against_the_gap_bound(seb):
    """Footprints with relative eigen-gaps from 2e-3 down to 2e-8 (the FP64 eigen-solve takes
    them): every value is checked, pitch / roll / z / risk against the gap-scaled bound of
    tests/parity.py and roughness against the plain tolerance; none is skipped."""
    cfg = dict(C2, nx=384, ny=64)
    e = near_degenerate_map()
    _, out, fl, (n64, ndeg) = run_map(seb, cfg, e)
    ref = oracle_grid(cfg, e)
    # the construction holds at the four axis-aligned yaws; at the others the z variance
    # exceeds the footprint's smaller in-plane variance and the normal lies almost horizontal
    # (a near-vertical plane: DEGENERATE or steep, not the case this test is about)
    ks = [0, 18, 36, 54]
    s = check(out[:, ks], fl[ks], tuple(a[ks] if a.ndim == 3 else a[:, ks] for a in ref), "near-degenerate")
    g = ref[2][ks]
    assert s["ill"] > 1000 and np.nanmin(g[np.isfinite(g)]) < 1e-7
    assert n64 > 0  # these cells took the FP64 eigen-solve
    print(s)


def test_flat_ground(seb):
    e = np.full((64, 64), 1.25, np.float32)
    _, out, fl, _ = run_map(seb, dict(C1, nx=64, ny=64), e)
    sl = (slice(None), slice(4, 60), slice(4, 60))
    assert (out[1][sl] == 0).all() and (out[2][sl] == 0).all() and (out[3][sl] == 0).all()
    assert (out[4][sl] == 0).all() and (out[0][sl] == 1.25).all()


def test_yaw_plus_pi_is_exact_negation(seb):
    e = fractal_steps_nan(5, 160, 160)
    _, out, fl, _ = run_map(seb, dict(C2, nx=160, ny=160), e)
    h = 36
    a, b = out[:, :h], out[:, h:]
    both = np.isfinite(a[1])
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[3].view(np.uint32), b[3].view(np.uint32))
    assert np.array_equal(a[4].view(np.uint32), b[4].view(np.uint32))
    assert np.array_equal(a[1][both], -b[1][both]) and np.array_equal(a[2][both], -b[2][both])
    assert np.array_equal(fl[:h], fl[h:])


def test_offset_invariance(seb):
    e = bumpy_plane(2, 80, 80)
    _, o1, f1, _ = run_map(seb, dict(C1, nx=80, ny=80), e)
    _, o2, f2, _ = run_map(seb, dict(C1, nx=80, ny=80), e + np.float32(2.0))
    ok = np.isfinite(o1[0])
    assert np.abs(o2[0][ok] - o1[0][ok] - 2.0).max() < 1e-5
    for ch in (1, 2, 3, 4):
        assert np.abs(o2[ch][ok] - o1[ch][ok]).max() < 1e-5


@pytest.mark.parametrize("shape", [(1, 1), (37, 53), (5, 300), (300, 7), (33, 33)])
def test_ragged_and_tiny_maps(seb, shape):
    ny, nx = shape
    e = fractal_steps_nan(11, nx, ny, nan_frac=0.03) if min(shape) > 4 else np.zeros(shape, np.float32)
    cfg = dict(C2, nx=nx, ny=ny)
    _, out, fl, _ = run_map(seb, cfg, e)
    check(out, fl, oracle_grid(cfg, e), f"ragged {shape}")


def test_all_unknown_map(seb):
    e = np.full((40, 50), np.nan, np.float32)
    _, out, fl, _ = run_map(seb, dict(C1, nx=50, ny=40), e)
    assert (fl == 3).all() and (out[4] == 1).all() and np.isnan(out[:4]).all()


@pytest.mark.parametrize("extra", [dict(n_yaw=2), dict(shape="ellipse"), dict(n_min=5), dict(n_yaw=8, length=1.5)])
def test_parameter_variants(seb, extra):
    cfg = dict(C1, nx=72, ny=56)
    cfg.update(extra)
    e = fractal_steps_nan(7, 72, 56, res=0.1)
    _, out, fl, _ = run_map(seb, cfg, e)
    check(out, fl, oracle_grid(cfg, e), str(extra))


def test_large_footprint_per_cell_kernel(seb):
    """A 4.0 x 3.0 m footprint at 0.05 m (reach 50 cells, ~4,800 points per cell): the sliding
    kernel's staged tile for the 16-column layout would need more than 227 KB of shared memory,
    so the launch runs the per-cell kernel in plain FP32."""
    cfg = dict(nx=120, ny=96, n_yaw=4, res=0.05, length=4.0, width=3.0)
    e = fractal_steps_nan(21, 120, 96, nan_frac=0.02)
    _, out, fl, _ = run_map(seb, cfg, e, n_min=100)
    s = check(out, fl, oracle_grid(cfg, e, n_min=100), "large footprint")
    assert s["assessed"] > 0.5 * s["n"]


FLUSH = dict(nx=96, ny=72, n_yaw=4, res=0.05, length=1.3, width=0.9)


def test_packed_moment_flush(seb):
    """A 1.3 x 0.9 m footprint at 0.05 m (reach 16 cells, ~470 points per cell): the moments of a
    whole footprint's missing points overflow the 16-bit fields that the sliding kernel packs
    the two rows of a block into, so the packed sums are moved into 32-bit sums every few row
    runs.  Every cell equals the oracle, and a rolling shift equals a rebuild bit for bit."""
    e = fractal_steps_nan(5, 96, 72, res=0.05, nan_frac=0.05)
    _, out, fl, _ = run_map(seb, FLUSH, e)
    s = check(out, fl, oracle_grid(FLUSH, e), "flushed moments")
    assert s["assessed"] > 0.5 * s["n"]
    world = torch.from_numpy(fractal_world(6, 300)).cuda()
    win = lambda o: world[o[1]:o[1] + 72, o[0]:o[0] + 96].contiguous()  # noqa: E731
    p = seb.SebParams(**FLUSH)
    m = seb.SebMap(p)
    m.update(win((100, 100)), (100, 100))
    for o in [(104, 97), (93, 99), (93, 120)]:
        m.shift(win(o), o)
    full = seb.SebMap(p)
    full.update(win((93, 120)), (93, 120))
    a, af = m.outputs()
    b, bf = full.outputs()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32)) and torch.equal(af, bf)


def test_rolling_window_bit_identical_to_rebuild(seb):
    """Sec. V-A: the window follows the robot; after 50 moves of 10 cells in random
    directions the ring-buffered map equals a fresh rebuild of the final window, bit for bit,
    and a sample of its cells equals the oracle."""
    world = fractal_world(1, 1100)
    tw = torch.from_numpy(world).cuda()
    p = seb.SebParams(**C2)
    o = [350, 350]
    win = lambda o: tw[o[1]:o[1] + 400, o[0]:o[0] + 400].contiguous()  # noqa: E731
    m = seb.SebMap(p)
    m.update(win(o), tuple(o))
    cells = 0
    for dx, dy in shift_sequence(2, 50):
        o = [min(max(o[0] + dx, 0), 700), min(max(o[1] + dy, 0), 700)]
        m.shift(win(o), tuple(o))
        cells += m.view().last_cells
    assert 0 < cells < 50 * 400 * 400 * 72
    v = m.view()
    assert (v.origin_i, v.origin_j) == tuple(o)
    ro, rf = m.outputs()
    full = seb.SebMap(p)
    full.update(win(o), tuple(o))
    fo, ff = full.outputs()
    assert torch.equal(ro.view(torch.int32), fo.view(torch.int32))
    assert torch.equal(rf, ff)
    m.check()
    # oracle on a sample of the final window
    e = world[o[1]:o[1] + 400, o[0]:o[0] + 400]
    rng = np.random.default_rng(0)
    cells = np.stack([rng.integers(0, 400, 50000), rng.integers(0, 400, 50000), rng.integers(0, 72, 50000)], 1)
    ref, rfl, gap = oracle.assess_cells(oracle.OracleParams(**C2), e.astype(np.float64), cells.astype(np.int32), tuple(o))
    g = ro.cpu().numpy()[:, cells[:, 2], cells[:, 1], cells[:, 0]].T
    gf = rf.cpu().numpy()[cells[:, 2], cells[:, 1], cells[:, 0]]
    compare(g, gf, ref, rfl, label="rolling sample", gap=gap)


def test_shift_batch_equals_single_shifts(seb):
    """seb_map_shift_batch (later launches stage and compute while the previous one finishes)
    gives the same bits as one seb_map_shift per move: 40 random moves with a zero move, a move
    beyond the window (a full rebuild inside the batch) and moves after it, then a second batch
    on the same map, after which the map equals a fresh rebuild of the final window."""
    world = fractal_world(4, 1700)
    tw = torch.from_numpy(world).cuda()
    p = seb.SebParams(**C2)
    win = lambda o: tw[o[1]:o[1] + 400, o[0]:o[0] + 400].contiguous()  # noqa: E731
    o = [650, 650]
    origins = []
    for k, (dx, dy) in enumerate(shift_sequence(7, 40)):
        if k == 11:
            dx, dy = 0, 0
        if k == 23:
            dx, dy = 450, -20  # beyond the window: a full rebuild
        o = [min(max(o[0] + dx, 0), 1300), min(max(o[1] + dy, 0), 1300)]
        origins.append(tuple(o))
    wins = [win(q) for q in origins]
    start = (650, 650)
    single = seb.SebMap(p)
    single.update(win(start), start)
    for w, q in zip(wins, origins):
        single.shift(w, q)
    batch = seb.SebMap(p)
    batch.update(win(start), start)
    batch.shift_batch(wins[:25], origins[:25])
    assert batch.view().last_cells > 0
    batch.shift_batch(wins[25:], origins[25:])
    so, sf = single.outputs()
    bo, bf = batch.outputs()
    assert torch.equal(so.view(torch.int32), bo.view(torch.int32)) and torch.equal(sf, bf)
    full = seb.SebMap(p)
    full.update(win(origins[-1]), origins[-1])
    fo, ff = full.outputs()
    assert torch.equal(bo.view(torch.int32), fo.view(torch.int32)) and torch.equal(bf, ff)
    batch.check()
    single.check()
    with pytest.raises(ValueError):
        batch.shift_batch(wins[:2], origins[:1])


@pytest.mark.parametrize("cfg,seed", [(dict(nx=200, ny=120, n_yaw=36, res=0.05, length=0.9, width=0.6), 11),
                                      (dict(nx=96, ny=160, n_yaw=8, res=0.1, length=1.5, width=0.6, shape="ellipse"), 12)])
def test_shift_batch_stress(seb, cfg, seed):
    """Batches with runs of zero moves (one batch opens with two), moves past the window (full
    rebuilds inside the batch), one-cell moves and a one-element batch, on a non-square map and
    an ellipse footprint: the same bits as separate seb_map_shift calls.  Each batch's windows
    are written just before it, the first moving one last, so that the batch's first launch
    follows the kernel that wrote its input."""
    rng = np.random.default_rng(seed)
    world = fractal_world(seed, 900, cfg["res"])
    tw = torch.from_numpy(world).cuda()
    p = seb.SebParams(**cfg)
    nx, ny = cfg["nx"], cfg["ny"]
    win = lambda o: tw[o[1]:o[1] + ny, o[0]:o[0] + nx].contiguous()  # noqa: E731
    o = [300, 300]
    origins = []
    for k in range(60):
        r = rng.random()
        if r < 0.2:
            d = (0, 0)
        elif r < 0.3:
            d = (int(rng.choice([-1, 1]) * nx), int(rng.integers(-3, 4)))
        elif r < 0.5:
            d = (int(rng.integers(-1, 2)), int(rng.integers(-1, 2)))
        else:
            d = (int(rng.integers(-25, 26)), int(rng.integers(-25, 26)))
        if k in (18, 19):
            d = (0, 0)
        elif k == 20:
            d = (5, -3)
        o = [min(max(o[0] + d[0], 0), 900 - nx), min(max(o[1] + d[1], 0), 900 - ny)]
        origins.append(tuple(o))
    wins = [win(q) for q in origins]
    single, batch = seb.SebMap(p), seb.SebMap(p)
    for mm in (single, batch):
        mm.update(win((300, 300)), (300, 300))
    for w, q in zip(wins, origins):
        single.shift(w, q)
    cuts = [0, 1, 17, 18, 40, 60]
    prev = [(300, 300)] + origins[:-1]
    for a, b in zip(cuts[:-1], cuts[1:]):
        bw = [win(q) for q in origins[a:b]]
        first = next((i for i in range(a, b) if origins[i] != prev[i]), None)
        if first is not None:
            bw[first - a] = win(origins[first])
        batch.shift_batch(bw, origins[a:b])
    so, sf = single.outputs()
    bo, bf = batch.outputs()
    assert torch.equal(so.view(torch.int32), bo.view(torch.int32)) and torch.equal(sf, bf)
    single.check()
    batch.check()


@pytest.mark.parametrize("move", [(0, 0), (1, 0), (0, -1), (-7, 13), (399, 0), (400, 5), (-1000, 2000)])
def test_shift_edge_moves(seb, move):
    world = fractal_world(3, 1400)
    tw = torch.from_numpy(world).cuda()
    p = seb.SebParams(**C2)
    o0 = [500, 500]
    win = lambda o: tw[o[1]:o[1] + 400, o[0]:o[0] + 400].contiguous()  # noqa: E731
    m = seb.SebMap(p)
    m.update(win(o0), tuple(o0))
    o1 = [o0[0] + move[0], o0[1] + move[1]]
    o1 = [min(max(o1[0], 0), 1000), min(max(o1[1], 0), 1000)]
    m.shift(win(o1), tuple(o1))
    full = seb.SebMap(p)
    full.update(win(o1), tuple(o1))
    a, af = m.outputs()
    b, bf = full.outputs()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32)) and torch.equal(af, bf)


def test_host_pointer_rejected(seb):
    m = seb.SebMap(seb.SebParams(**C1))
    host = torch.zeros(100, 100)
    with pytest.raises(seb.abi.SebError) as ei:
        seb.abi.seb_map_update(m.handle, host.data_ptr(), 0, 0)
    assert ei.value.status == seb.abi.SEB_ERR_INVALID_ARG
