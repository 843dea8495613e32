"""GPU parity of the SE(2) signed distance field (seb_risk_sdf) against the brute-force FP64
reference in oracle/sdf.py on the same seeded risk grids."""
import math

import numpy as np
import pytest

from oracle.sdf import risk_sdf as ref_sdf
from synthetic import lookup_poses, obstacle_risk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES = 0.05
RES_F = float(np.float32(RES))
TOL = 2e-6  # FP32 sqrt of an exact integer squared distance, times res


@pytest.fixture(scope="module")
def seb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb

    return seb


def gpu_sdf(seb, risk_np, ring=(0, 0), origin=(0, 0), **kw):
    K, ny, nx = risk_np.shape
    t = torch.from_numpy(risk_np).cuda()
    g = seb.SE2Grid.from_tensor(t, RES, origin, ring)
    return seb.risk_sdf(g, **kw)


@pytest.mark.parametrize("shape,ring", [((6, 47, 71), (9, 31)), ((3, 1, 40), (0, 0)), ((3, 33, 1), (0, 5)),
                                        ((2, 64, 64), (63, 63)), ((150, 12, 130), (77, 5))])
def test_full_grid_parity(seb, shape, ring):
    """Every cell against the FP64 reference.  The last grid has enough 32-column stripes x bins
    (750) for the large-grid column pass (8 row segments per stripe), with a ragged last stripe
    (130 = 4 x 32 + 2 columns)."""
    K, ny, nx = shape
    risk = obstacle_risk(7, K, ny, nx, n_blobs=4, blob_cells=(1, 6))
    ring = (ring[0] % nx, ring[1] % ny)
    s = gpu_sdf(seb, risk, ring=ring)
    ref = ref_sdf(risk.astype(np.float64), RES_F, ring=ring)
    got = s._owner.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.array_equal(np.sign(got[~fin]), np.sign(ref[~fin]))
    assert np.abs(got[fin] - ref[fin]).max() <= TOL * max(1.0, np.abs(ref[fin]).max())


def test_clamp_threshold_nan_and_empty_slices(seb):
    risk = obstacle_risk(8, 5, 40, 52, n_blobs=3, nan_frac=0.01)
    risk[3] = 0.2   # no obstacle in this bin
    risk[4] = 1.0   # only obstacles
    for thr, clamp in ((1.0, 0.4), (0.5, math.inf), (0.95, 1.0)):
        got = gpu_sdf(seb, risk, ring=(3, 4), risk_obstacle=thr, clamp=clamp)._owner.cpu().numpy()
        ref = ref_sdf(risk.astype(np.float64), RES_F, risk_obstacle=thr, clamp=clamp, ring=(3, 4))
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin) and np.array_equal(np.sign(got[~fin]), np.sign(ref[~fin]))
        assert np.abs(got[fin] - ref[fin]).max() <= TOL * max(1.0, np.abs(ref[fin]).max())
    # bin 3 holds no obstacle and bin 4 nothing else: the clamp on either side
    assert (got[3] == 1.0).all() and (got[4] == -1.0).all()


def test_map_sized_grid_sampled(seb):
    K, ny, nx = 72, 400, 400
    risk = obstacle_risk(9, K, ny, nx, n_blobs=40, blob_cells=(2, 14))
    got = gpu_sdf(seb, risk, ring=(123, 321), clamp=2.0)._owner
    rng = np.random.default_rng(10)
    ks = rng.choice(K, 6, replace=False)
    cells = np.stack([rng.integers(0, nx, 1500 * 6), rng.integers(0, ny, 1500 * 6), np.repeat(ks, 1500)], 1)
    ref = ref_sdf(risk.astype(np.float64), RES_F, clamp=2.0, ring=(123, 321), cells=cells)
    pr = (cells[:, 1] + 321) % ny
    pc = (cells[:, 0] + 123) % nx
    g = got.cpu().numpy()[cells[:, 2], pr, pc]
    assert np.abs(g - ref).max() <= TOL * 2.0


def test_long_rows_clamped_search(seb):
    """Rows whose sentinel padding would exceed the row pass's shared-memory budget (6000
    columns, a 160 m clamp: W = 3201 cells) take the clamped two-offset search; sampled cells
    against the FP64 reference, with sparse obstacles so that the searches run long."""
    K, ny, nx = 2, 3, 6000
    risk = obstacle_risk(41, K, ny, nx, n_blobs=3, blob_cells=(1, 2))
    got = gpu_sdf(seb, risk, ring=(1234, 1), clamp=160.0)._owner.cpu().numpy()
    rng = np.random.default_rng(42)
    m = 1500
    cells = np.stack([rng.integers(0, nx, m), rng.integers(0, ny, m), rng.integers(0, K, m)], 1)
    ref = ref_sdf(risk.astype(np.float64), RES_F, clamp=160.0, ring=(1234, 1), cells=cells)
    g = got[cells[:, 2], (cells[:, 1] + 1) % ny, (cells[:, 0] + 1234) % nx]
    assert np.abs(ref).max() > 20.0  # long searches, not the clamp
    assert np.abs(g - ref).max() <= TOL * 160.0


def test_sdf_grid_lookup(seb):
    """The SDF comes back as a grid the trilinear lookup reads directly."""
    risk = obstacle_risk(11, 8, 30, 40)
    s = gpu_sdf(seb, risk, ring=(7, 2), origin=(-4, 9), clamp=1.0)
    poses = torch.from_numpy(lookup_poses(12, 1000, 40, 30, RES, (-4, 9), pad_cells=0.0)).cuda()
    val, grad, fl = seb.se2_lookup(s, poses, with_grad=True)
    assert (fl == 0).all() and torch.isfinite(val).all() and (val.abs() <= 1.0).all()


@pytest.mark.parametrize("clamp", [8.875, 8.925, math.inf])
def test_packed_and_padded_row_passes(seb, clamp):
    """The row pass packs two candidates per register while the search bound W = ceil(clamp /
    res) + 1 is at most 179 (W = 179 here) and keeps 32-bit candidates above (W = 180, and W =
    the row length without a clamp); sparse obstacles on 420-column rows make the searches run
    to the bound.  Sampled cells against the FP64 reference."""
    K, ny, nx = 2, 24, 420
    risk = obstacle_risk(43, K, ny, nx, n_blobs=2, blob_cells=(1, 3))
    got = gpu_sdf(seb, risk, ring=(17, 5), clamp=clamp)._owner.cpu().numpy()
    rng = np.random.default_rng(44)
    m = 2500
    cells = np.stack([rng.integers(0, nx, m), rng.integers(0, ny, m), rng.integers(0, K, m)], 1)
    ref = ref_sdf(risk.astype(np.float64), RES_F, clamp=clamp, ring=(17, 5), cells=cells)
    g = got[cells[:, 2], (cells[:, 1] + 5) % ny, (cells[:, 0] + 17) % nx]
    fin = np.isfinite(ref)
    assert np.abs(ref[fin]).max() > 5.0  # long searches
    assert np.array_equal(np.isfinite(g), fin)
    assert np.abs(g[fin] - ref[fin]).max() <= TOL * max(1.0, np.abs(ref[fin]).max())
