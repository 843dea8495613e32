"""Reduced-precision forms on the 1024 x 1024 x 72 map (0.05 m, small-map terrain generator):
elevation stored as FP32, BF16 or FP16 and widened to FP32 in the kernel, moments either plain
or Neumaier-compensated FP32 about the per-cell reference, FP64 eigen-solve for small
eigen-gaps.  Parity: against the FP64 oracle run on the same (quantised) elevation, sampled
at the full size; the storage error itself is reported against the unquantised elevation."""
import numpy as np
import pytest
import torch

import oracle
from synthetic import bumpy_plane

from .parity import compare

pytestmark = pytest.mark.gpu

C3 = dict(nx=1024, ny=1024, n_yaw=72, res=0.05, length=0.9, width=0.6)


@pytest.fixture(scope="module")
def seb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


@pytest.fixture(scope="module")
def terrain():
    e = bumpy_plane(21, 1024, 1024, 0.05, dtype=np.float64)
    rng = np.random.default_rng(4)
    n = 60000
    cells = np.stack([rng.integers(0, 1024, n), rng.integers(0, 1024, n), rng.integers(0, 72, n)], 1).astype(np.int32)
    return e, cells


def gpu_sample(seb, e_dev, cells, **kw):
    m = seb.SebMap(seb.SebParams(**C3, elev_dtype=e_dev.dtype, **kw))
    m.update(e_dev, (0, 0))
    g = m.out_phys[:, cells[:, 2], cells[:, 1], cells[:, 0]].T.cpu().numpy()
    f = m.flags_phys[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().numpy()
    counters = m.check()
    return g, f, counters


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("precision", ["plain", "compensated"])
def test_quantised_input_parity(seb, terrain, dt, precision):
    e, cells = terrain
    ed = torch.from_numpy(e).to("cuda", dtype=dt)
    g, f, _ = gpu_sample(seb, ed, cells, precision=precision)
    eq = ed.float().cpu().numpy().astype(np.float64)  # exactly the values the kernel widens
    r, rf, gap = oracle.assess_cells(oracle.OracleParams(**C3), eq, cells)
    compare(g, f, r, rf, label=f"{dt} {precision}", gap=gap)


def test_storage_error_report(seb, terrain, record_property):
    """Error of each storage type against the FP64 oracle on the unquantised terrain.
    FP32 meets the FP32 tolerances; FP16 (quantum <= 2^-7 m below 16 m) and BF16 (quantum
    2^-4 m at 8-16 m) carry the quantisation noise of the stored heights."""
    e, cells = terrain
    r, rf, _ = oracle.assess_cells(oracle.OracleParams(**C3), e, cells)
    ok = (rf & 5) == 0
    res = {}
    for dt in (torch.float32, torch.float16, torch.bfloat16):
        g, f, _ = gpu_sample(seb, torch.from_numpy(e).to("cuda", dtype=dt), cells)
        both = ok & ((f & 5) == 0)
        for ch, name in enumerate(("z", "pitch", "roll", "rough", "risk")):
            d = np.abs(g[both, ch] - r[both, ch])
            res[(str(dt), name)] = (float(d.max()), float(np.percentile(d, 99)))
            record_property(f"{dt}_{name}_max", float(d.max()))
            record_property(f"{dt}_{name}_p99", float(np.percentile(d, 99)))
    print(res)
    f32 = {k[1]: v for k, v in res.items() if k[0] == "torch.float32"}
    f16 = {k[1]: v for k, v in res.items() if k[0] == "torch.float16"}
    b16 = {k[1]: v for k, v in res.items() if k[0] == "torch.bfloat16"}
    assert f32["pitch"][0] < 1e-4 and f32["roll"][0] < 1e-4 and f32["z"][0] < 1e-4
    for name in ("z", "pitch", "roll"):
        assert f16[name][1] <= b16[name][1]
    assert f16["pitch"][1] < 5e-3 and f16["roll"][1] < 5e-3
    assert b16["pitch"][1] < 5e-2 and b16["roll"][1] < 5e-2


def test_fp64_eigen_path(seb, terrain):
    """gap_fp64 = 1 sends every assessed cell through the FP64 eigen-solve: same results,
    FP64 flag set, counter equal to the number of assessed (cell, yaw-pair) solves."""
    e, cells = terrain
    sub = e[:256, :256].copy()
    cfg = dict(C3, nx=256, ny=256)
    m = seb.SebMap(seb.SebParams(**cfg, gap_fp64=1.0))
    m.update(torch.from_numpy(sub).float().cuda(), (0, 0))
    out, fl = m.outputs()
    n64, ndeg = m.check()
    fl = fl.cpu().numpy()
    assessed = (fl & 1) == 0
    assert ((fl[assessed] & 8) != 0).all()
    assert n64 == assessed.sum() // 2  # one solve per yaw pair
    ref, rfl, gap = oracle.assess_grid(oracle.OracleParams(**cfg), sub.astype(np.float32).astype(np.float64),
                                       with_gap=True)
    compare(out.cpu().numpy().reshape(5, -1).T, fl.reshape(-1), ref.reshape(5, -1).T, rfl.reshape(-1),
            label="fp64", gap=gap.reshape(-1))


def _reconstruct_tiled(seb, buf, nx, ny, origin=(0, 0)):
    """Heights a SEB_BF16_TILED window stands for: base of the cell's world tile + offset (FP32)."""
    d, b = seb.tiled_parts(buf, nx, ny)
    d = d.float().cpu().numpy()
    b = b.cpu().numpy()
    px, py = origin[0] % 16, origin[1] % 16
    r = (np.arange(ny) + py) // 16
    c = (np.arange(nx) + px) // 16
    return (b[r][:, c] + d).astype(np.float32)


def test_bf16_tiled_encoding(seb):
    """The encoder: per 16 x 16 world tile, base = midpoint of the smallest and largest known
    height, offsets = BF16 round-to-nearest of height - base, NaN kept; at a window origin that
    is not a multiple of 16 the tiles follow the world grid."""
    for origin in ((0, 0), (5, -13)):
        e = bumpy_plane(3, 100, 72, 0.05)
        e[10:14, 20:31] = np.nan
        e[32:48, 48:64] = np.nan  # one whole world tile unknown at origin (0, 0)
        buf = seb.encode_bf16_tiled(torch.from_numpy(e).cuda(), origin)
        d, b = seb.tiled_parts(buf, 100, 72)
        px, py = origin[0] % 16, origin[1] % 16
        bw = np.zeros(b.shape, np.float32)
        for ty in range(b.shape[0]):
            for tx in range(b.shape[1]):
                t = e[max(ty * 16 - py, 0):max(ty * 16 - py + 16, 0), max(tx * 16 - px, 0):max(tx * 16 - px + 16, 0)]
                k = t[np.isfinite(t)]
                bw[ty, tx] = np.float32(0.5) * k.min() + np.float32(0.5) * k.max() if k.size else 0.0
        assert np.array_equal(b.cpu().numpy()[:bw.shape[0], :bw.shape[1]], bw)
        r = (np.arange(72) + py) // 16
        c = (np.arange(100) + px) // 16
        want = (torch.from_numpy(e) - torch.from_numpy(bw[r][:, c])).to(torch.bfloat16)
        got = d.cpu()
        nan = torch.isnan(want)
        assert torch.equal(torch.isnan(got), nan)  # NaN stays NaN (its payload is not fixed)
        assert torch.equal(got[~nan].view(torch.int16), want[~nan].view(torch.int16))


def test_bf16_tiled_parity_and_error(seb, terrain, record_property):
    """SEB_BF16_TILED on the 1024 x 1024 map: parity against the oracle on the heights the
    encoding stands for, and the storage error against the unquantised terrain, next to plain
    BF16 (whose quantum at 8-16 m is 2^-4 m)."""
    e, cells = terrain
    buf = seb.encode_bf16_tiled(torch.from_numpy(e.astype(np.float32)).cuda())
    g, f, _ = gpu_sample_tiled(seb, buf, cells)
    eq = _reconstruct_tiled(seb, buf, 1024, 1024).astype(np.float64)
    r, rf, gap = oracle.assess_cells(oracle.OracleParams(**C3), eq, cells)
    compare(g, f, r, rf, label="bf16 tiled", gap=gap)
    r0, rf0, _ = oracle.assess_cells(oracle.OracleParams(**C3), e, cells)
    gb, fb, _ = gpu_sample(seb, torch.from_numpy(e).to("cuda", dtype=torch.bfloat16), cells)
    ok = ((rf0 & 5) == 0) & ((f & 5) == 0) & ((fb & 5) == 0)
    for ch, name in enumerate(("z", "pitch", "roll", "rough", "risk")):
        dt = np.abs(g[ok, ch] - r0[ok, ch])
        db = np.abs(gb[ok, ch] - r0[ok, ch])
        record_property(f"bf16_tiled_{name}_max", float(dt.max()))
        record_property(f"bf16_tiled_{name}_p99", float(np.percentile(dt, 99)))
        print(f"{name}: tiled max {dt.max():.3g} p99 {np.percentile(dt, 99):.3g}; "
              f"bf16 max {db.max():.3g} p99 {np.percentile(db, 99):.3g}")
        if name in ("z", "pitch", "roll"):
            assert np.percentile(dt, 99) < 0.25 * np.percentile(db, 99)
    assert np.abs(g[ok, 1] - r0[ok, 1]).max() < 5e-3


def gpu_sample_tiled(seb, buf, cells, **kw):
    m = seb.SebMap(seb.SebParams(**C3, elev_dtype="bf16_tiled", **kw))
    m.update(buf, (0, 0))
    g = m.out_phys[:, cells[:, 2], cells[:, 1], cells[:, 0]].T.cpu().numpy()
    f = m.flags_phys[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().numpy()
    return g, f, m.check()


@pytest.mark.parametrize("form", ["compensated", "bf16_tiled"])
def test_rolling_bit_identical_in_reduced_precision_forms(seb, form):
    """The compensated sums and the tiled BF16 storage keep the rolling map bit-identical to a
    rebuild: every cell's arithmetic depends on its neighbourhood only."""
    from synthetic import fractal_world, shift_sequence

    n, W = 160, 420
    world = torch.from_numpy(fractal_world(8, W)).cuda()
    kw = dict(nx=n, ny=n, n_yaw=72, res=0.05, length=0.9, width=0.6)
    if form == "compensated":
        p = seb.SebParams(**kw, precision="compensated")
        win = lambda o: world[o[1]:o[1] + n, o[0]:o[0] + n].contiguous()  # noqa: E731
    else:
        p = seb.SebParams(**kw, elev_dtype="bf16_tiled")
        enc = seb.encode_bf16_tiled(world)
        win = lambda o: seb.tiled_window(enc, W, W, o[0], o[1], n, n)  # noqa: E731
    o = [130, 130]
    m = seb.SebMap(p)
    m.update(win(o), tuple(o))
    for dx, dy in shift_sequence(9, 14, 7):
        o = [min(max(o[0] + dx, 0), W - n), min(max(o[1] + dy, 0), W - n)]
        m.shift(win(o), tuple(o))
    ro, rf = m.outputs()
    full = seb.SebMap(p)
    full.update(win(o), tuple(o))
    fo, ff = full.outputs()
    assert torch.equal(ro.view(torch.int32), fo.view(torch.int32)) and torch.equal(rf, ff)
    m.check()
