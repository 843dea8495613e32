"""GPU parity of nearest-neighbour inpainting (seb_inpaint_nearest) against the brute-force
reference in oracle/inpaint.py: an index-and-copy operation, so values and sources must be
bit-identical."""
import numpy as np
import pytest

import oracle
from oracle.inpaint import inpaint_nearest as ref_inpaint
from synthetic import bumpy_plane, fractal_steps_nan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


def check(seb, z, max_cells=0):
    out, src = seb.inpaint_nearest(torch.from_numpy(z).cuda(), max_cells, with_source=True)
    ro, rs = ref_inpaint(z, max_cells)
    out, src = out.cpu().numpy(), src.cpu().numpy()
    assert np.array_equal(src, rs)
    assert np.array_equal(np.isnan(out), np.isnan(ro))
    fin = ~np.isnan(ro)
    assert np.array_equal(out[fin].view(np.int32), ro[fin].astype(np.float32).view(np.int32))


@pytest.mark.parametrize("shape,frac", [((43, 57), 0.3), ((64, 64), 0.9), ((1, 50), 0.5), ((37, 1), 0.5),
                                        ((130, 70), 0.995)])
def test_random_maps(seb, shape, frac):
    rng = np.random.default_rng(hash(shape) % 1000)
    z = rng.normal(size=shape).astype(np.float32)
    z[rng.random(shape) < frac] = np.nan
    check(seb, z)
    check(seb, z, max_cells=3)


def test_ties_and_degenerate_maps(seb):
    z = np.full((7, 7), np.nan, np.float32)
    z[1, 3], z[5, 3], z[3, 1], z[3, 5] = 1.0, 2.0, 3.0, 4.0
    check(seb, z)
    g = np.full((12, 12), np.nan, np.float32)
    g[::4, ::4] = np.arange(9, dtype=np.float32).reshape(3, 3)  # a lattice full of ties
    check(seb, g)
    check(seb, np.full((5, 6), np.nan, np.float32))
    check(seb, np.ones((5, 6), np.float32))


def test_fractal_map_crop(seb):
    z = np.ascontiguousarray(fractal_steps_nan(3)[:200, 100:300])
    check(seb, z)
    check(seb, z, max_cells=5)


def test_inpainted_map_assessment(seb):
    """Inpaint then assess: the GPU chain against the oracle chain (the oracle inpaints and
    assesses its own copy; both inpaintings are bit-identical by the tests above)."""
    from tests.parity import compare, grid_to_rows

    rng = np.random.default_rng(5)
    z = bumpy_plane(2, 60, 60, 0.1)
    yy, xx = np.mgrid[0:60, 0:60]
    for _ in range(6):
        cy, cx, r = rng.uniform(0, 60), rng.uniform(0, 60), rng.uniform(1, 4)
        z[(yy - cy) ** 2 + (xx - cx) ** 2 <= r * r] = np.nan
    p = seb.SebParams(nx=60, ny=60, n_yaw=16, res=0.1, length=0.6, width=0.4)
    filled = seb.inpaint_nearest(torch.from_numpy(z).cuda())
    m = seb.SebMap(p)
    m.update(filled)
    out, fl = m.outputs()
    ref_z, _ = ref_inpaint(z)
    op = oracle.OracleParams(nx=60, ny=60, n_yaw=16, res=0.1, length=0.6, width=0.4)
    ro, rf, gap = oracle.assess_grid(op, ref_z.astype(np.float32).astype(np.float64), with_gap=True)
    o, f = grid_to_rows(out.cpu().numpy(), fl.cpu().numpy())
    r, rfl, g = grid_to_rows(ro, rf, gap)
    compare(o, f, r, rfl, label="inpainted", gap=g)
    # after inpainting only the window border can leave a footprint short of known cells
    raw = oracle.assess_grid(op, z.astype(np.float64))[1]
    assert (rf & 1).sum() < (raw & 1).sum()
