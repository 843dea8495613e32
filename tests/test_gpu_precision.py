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
