"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry point the
header declares, validates its arguments, and builds footprint tables equal to the
oracle's independent enumeration (Algorithm 1, FindEllipticalPoints)."""
import os
import re

import pytest

import oracle
from paper_2503_02412_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "seb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = "\n".join(l for l in text.splitlines() if not l.strip().startswith("#"))
    return sorted(set(re.findall(r"\b(seb_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    declared = header_functions()
    assert len(declared) >= 15
    assert sorted(abi.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_params_default_and_workspace(lib):
    p = abi.seb_params_default()
    assert (p.nx, p.ny, p.n_yaw) == (100, 100, 36)
    assert abs(p.phi_x_max - 0.52) < 1e-7 and abs(p.phi_y_max - 0.52) < 1e-7
    n = abi.seb_workspace_bytes(p)
    out = 5 * 36 * 100 * 100 * 4
    fl = 36 * 100 * 100
    al = lambda x: (x + 255) // 256 * 256  # noqa: E731
    assert n == 256 + al(out) + al(fl)
    p.n_yaw = 35
    assert abi.seb_workspace_bytes(p) == 0
    p.n_yaw = 36
    p.res = 0.0
    assert abi.seb_workspace_bytes(p) == 0


def test_status_strings(lib):
    assert abi.seb_status_string(0) == "ok"
    assert "workspace" in abi.seb_status_string(abi.SEB_ERR_WORKSPACE)


def test_create_rejects_bad_workspace_without_gpu(lib):
    import ctypes

    p = abi.seb_params_default()
    h = ctypes.c_void_p()
    assert lib.seb_map_create(ctypes.byref(p), None, 1 << 30, None, ctypes.byref(h)) == abi.SEB_ERR_WORKSPACE
    assert lib.seb_map_create(ctypes.byref(p), 0x1001, 1 << 30, None, ctypes.byref(h)) == abi.SEB_ERR_WORKSPACE
    assert lib.seb_map_create(ctypes.byref(p), 0x100000, 16, None, ctypes.byref(h)) == abi.SEB_ERR_WORKSPACE
    assert "small" in abi.seb_last_error()
    p.n_yaw = 3
    assert lib.seb_map_create(ctypes.byref(p), 0x100000, 1 << 30, None, ctypes.byref(h)) == abi.SEB_ERR_BAD_SHAPE
    assert lib.seb_map_destroy(None) == abi.SEB_ERR_INVALID_ARG


def test_query_rejects_null_without_gpu(lib):
    import ctypes

    p = abi.seb_params_default()
    rc = lib.seb_query_poses(ctypes.byref(p), None, 0, 0, None, 10, None, None, None, None)
    assert rc == abi.SEB_ERR_INVALID_ARG
    rc = lib.seb_query_poses_backward(ctypes.byref(p), 0x1000, 0, 0, None, None, None, None, -1, None)
    assert rc == abi.SEB_ERR_INVALID_ARG


@pytest.mark.parametrize("change", [dict(length=30.0), dict(length=9.0, width=9.0, res=0.05), dict(n_yaw=3),
                                    dict(length=4.0, width=3.0, res=0.05)])
def test_noalloc_validates_like_the_allocating_query(lib, change):
    """The allocation-free query builds its lattice through the same tables as seb_query_poses,
    so both return the same status for parameter sets the tables reject (reach beyond the
    packing, moments or staged tile too large, odd yaw count, a lattice above 256 points); the
    checks run before any CUDA call."""
    import ctypes

    p = abi.seb_params_default()
    for k, v in change.items():
        setattr(p, k, v)
    a = lib.seb_query_poses(ctypes.byref(p), 0x1000, 0, 0, 0x2000, 1, 0x3000, 0x4000, None, None)
    b = lib.seb_query_poses_grad_noalloc(ctypes.byref(p), 0x1000, 0, 0, 0x2000, 1, 0x5000, 0x3000, 0x4000, 0x6000,
                                         None)
    assert a == b and a in (abi.SEB_ERR_BAD_SHAPE, abi.SEB_ERR_INVALID_ARG), (a, b)


CONFIGS = [
    dict(nx=100, ny=100, n_yaw=36, res=0.1, length=0.6, width=0.4),
    dict(nx=400, ny=400, n_yaw=72, res=0.05, length=0.9, width=0.6),
    dict(nx=64, ny=64, n_yaw=16, res=0.05, length=0.9, width=0.6, shape="ellipse"),
    dict(nx=64, ny=64, n_yaw=2, res=0.1, length=0.3, width=0.3),
    dict(nx=64, ny=64, n_yaw=10, res=0.07, length=1.3, width=0.25),
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_tables_equal_oracle_membership(lib, cfg):
    from paper_2503_02412_gb300 import SebParams

    sp = SebParams(**cfg).c()
    op = oracle.OracleParams(**cfg)
    for k in range(cfg["n_yaw"]):
        got = abi.seb_footprint_table(sp, k)
        want = [tuple(x) for x in oracle.footprint(op, k).tolist()]
        assert got == want, (k, len(got), len(want))  # same set, same row-run order


def test_footprint_table_bad_args(lib):
    import ctypes

    p = abi.seb_params_default()
    assert lib.seb_footprint_table(ctypes.byref(p), 36, None, None, 0) == abi.SEB_ERR_INVALID_ARG
    assert lib.seb_footprint_table(None, 0, None, None, 0) == abi.SEB_ERR_INVALID_ARG
    p.length = 30.0  # reach beyond the 127-cell packing
    assert lib.seb_footprint_table(ctypes.byref(p), 0, None, None, 0) == abi.SEB_ERR_BAD_SHAPE


def test_sdf_inpaint_and_batch_argument_checks_without_gpu(lib):
    """Argument checks that return before any CUDA call: NULL and out-of-range arguments, an
    undersized workspace, an output aliasing its input, a negative clamp, a negative batch."""
    import ctypes

    nx, ny, K = 400, 400, 72
    assert lib.seb_sdf_workspace_bytes(nx, ny, K) == nx * ny * K * 4
    assert lib.seb_sdf_workspace_bytes(0, ny, K) == 0 and lib.seb_sdf_workspace_bytes(nx, 16385, K) == 0
    assert lib.seb_inpaint_workspace_bytes(nx, ny) == nx * ny * 4 and lib.seb_inpaint_workspace_bytes(nx, 0) == 0
    fake = 0x100000  # never dereferenced: every call below fails its checks first
    g = abi.seb_grid(data=fake, nx=nx, ny=ny, n_yaw=K, ring_x=0, ring_y=0, origin_i=0, origin_j=0, res=0.05)
    need = nx * ny * K * 4
    sdf = lib.seb_risk_sdf
    assert sdf(None, 1.0, 2.0, fake, need, 0x200000, None) == abi.SEB_ERR_INVALID_ARG
    assert sdf(ctypes.byref(g), 1.0, 2.0, fake, need, None, None) == abi.SEB_ERR_INVALID_ARG
    assert sdf(ctypes.byref(g), 1.0, -1.0, 0x300000, need, 0x200000, None) == abi.SEB_ERR_INVALID_ARG
    assert sdf(ctypes.byref(g), 1.0, 2.0, 0x300000, need - 4, 0x200000, None) == abi.SEB_ERR_WORKSPACE
    assert sdf(ctypes.byref(g), 1.0, 2.0, 0x300001, need, 0x200000, None) == abi.SEB_ERR_WORKSPACE
    assert sdf(ctypes.byref(g), 1.0, 2.0, 0x300000, need, fake, None) == abi.SEB_ERR_INVALID_ARG  # aliasing
    for bad in (dict(nx=0), dict(ring_x=nx), dict(ring_y=-1), dict(res=0.0), dict(n_yaw=0)):
        gb = abi.seb_grid(data=fake, nx=nx, ny=ny, n_yaw=K, ring_x=0, ring_y=0, origin_i=0, origin_j=0, res=0.05)
        for k, v in bad.items():
            setattr(gb, k, v)
        assert sdf(ctypes.byref(gb), 1.0, 2.0, 0x300000, need, 0x200000, None) == abi.SEB_ERR_BAD_SHAPE, bad
    inp = lib.seb_inpaint_nearest
    wneed = nx * ny * 4
    assert inp(None, nx, ny, 0, 0x300000, wneed, 0x200000, None, None) == abi.SEB_ERR_INVALID_ARG
    assert inp(fake, 0, ny, 0, 0x300000, wneed, 0x200000, None, None) == abi.SEB_ERR_BAD_SHAPE
    assert inp(fake, nx, ny, 0, 0x300000, wneed, fake, None, None) == abi.SEB_ERR_INVALID_ARG
    assert inp(fake, nx, ny, 0, 0x300000, wneed - 1, 0x200000, None, None) == abi.SEB_ERR_WORKSPACE
    assert lib.seb_map_shift_batch(None, None, None, 0) == abi.SEB_ERR_INVALID_ARG


def test_handle_and_shape_checks_without_gpu(lib):
    """NULL handles, bad grid shapes, negative counts and bad elevation-map parameters are
    rejected with their status codes before any CUDA call."""
    import ctypes

    INV, SHAPE, WS = abi.SEB_ERR_INVALID_ARG, abi.SEB_ERR_BAD_SHAPE, abi.SEB_ERR_WORKSPACE
    fake = 0x100000  # never dereferenced
    # rolling map entry points with no map
    assert lib.seb_map_set_stream(None, None) == INV
    assert lib.seb_map_update(None, fake, 0, 0) == INV
    assert lib.seb_map_shift(None, fake, 0, 0) == INV
    assert lib.seb_map_view(None, ctypes.byref(abi.seb_view())) == INV
    assert lib.seb_map_copy_out(None, fake, fake) == INV
    assert lib.seb_map_check(None, 10, None, None) == INV
    assert lib.seb_map_grid(None, 0, ctypes.byref(abi.seb_grid())) == INV
    # trilinear lookup: grid checks, then counts and pointers
    good = dict(data=fake, nx=40, ny=30, n_yaw=36, ring_x=0, ring_y=0, origin_i=0, origin_j=0, res=0.1)
    assert lib.seb_se2_lookup(None, fake, 1, 0.0, fake, None, None, None) == INV
    for bad in (dict(data=None), dict(nx=1), dict(ny=1), dict(n_yaw=0), dict(n_yaw=4097), dict(res=0.0),
                dict(res=float("inf")), dict(ring_x=40), dict(ring_y=-1)):
        g = abi.seb_grid(**dict(good, **bad))
        want = INV if "data" in bad else SHAPE
        assert lib.seb_se2_lookup(ctypes.byref(g), fake, 1, 0.0, fake, None, None, None) == want, bad
        assert lib.seb_se2_lookup_vjp(ctypes.byref(g), fake, 1, fake, fake, None) == want, bad
    g = abi.seb_grid(**good)
    assert lib.seb_se2_lookup(ctypes.byref(g), fake, -1, 0.0, fake, None, None, None) == INV
    assert lib.seb_se2_lookup(ctypes.byref(g), None, 5, 0.0, fake, None, None, None) == INV
    assert lib.seb_se2_lookup_vjp(ctypes.byref(g), fake, 5, fake, None, None) == INV
    # allocation-free pose query
    p = abi.seb_params_default()
    assert lib.seb_query_poses_grad_noalloc(ctypes.byref(p), None, 0, 0, fake, 1, fake, fake, fake, fake, None) == INV
    assert lib.seb_query_poses_grad_noalloc(ctypes.byref(p), fake, 0, 0, fake, -1, fake, fake, fake, fake, None) == INV
    # elevation map: parameters, workspace size, handles
    ep = abi.seb_elev_params()
    lib.seb_elev_params_default(ctypes.byref(ep))
    assert (ep.nx, ep.ny) == (400, 400) and abs(ep.res - 0.05) < 1e-7 and ep.z_min < ep.z_max and ep.gate > 0
    n = lib.seb_elev_workspace_bytes(ctypes.byref(ep), 1000)
    assert n > 0 and lib.seb_elev_workspace_bytes(ctypes.byref(ep), 2000) > n
    assert lib.seb_elev_workspace_bytes(ctypes.byref(ep), -1) == 0
    h = ctypes.c_void_p()
    assert lib.seb_elev_create(ctypes.byref(ep), 1000, fake, n, None, None) == INV
    assert lib.seb_elev_create(ctypes.byref(ep), 1000, None, n, None, ctypes.byref(h)) == WS
    assert lib.seb_elev_create(ctypes.byref(ep), 1000, fake + 16, n, None, ctypes.byref(h)) == WS  # not 256-aligned
    assert lib.seb_elev_create(ctypes.byref(ep), 1000, fake, n - 1, None, ctypes.byref(h)) == WS
    for field, value in (("nx", 0), ("ny", 16385), ("res", 0.0), ("res", float("nan")), ("gate", 0.0), ("z_min", 2.0)):
        bad = abi.seb_elev_params()
        lib.seb_elev_params_default(ctypes.byref(bad))
        setattr(bad, field, value)
        assert lib.seb_elev_workspace_bytes(ctypes.byref(bad), 10) == 0, field
        assert lib.seb_elev_create(ctypes.byref(bad), 10, fake, 1 << 30, None, ctypes.byref(h)) == INV, field
    assert lib.seb_elev_set_stream(None, None) == INV
    assert lib.seb_elev_integrate(None, ctypes.byref(abi.seb_scan_pose()), fake, 1) == INV
    assert lib.seb_elev_view_get(None, ctypes.byref(abi.seb_elev_view())) == INV
    assert lib.seb_elev_copy_out(None, fake, fake) == INV
    assert lib.seb_elev_destroy(None) == abi.SEB_OK


def test_surrogate_argument_checks_without_gpu(lib):
    """The surrogate's entry points reject NULL handles, bad batches and engines, maps smaller
    than the network's 33 x 33 window, non-FP32 elevation and bad workspaces before any CUDA
    call."""
    import ctypes

    INV, WS = abi.SEB_ERR_INVALID_ARG, abi.SEB_ERR_WORKSPACE
    fake = 0x100000  # never dereferenced
    p = abi.seb_params_default()
    p.nx = p.ny = 200
    p.n_yaw = 72
    p.res = 0.05
    n = lib.seb_sur_workspace_bytes(ctypes.byref(p), 8)
    assert n > 0 and lib.seb_sur_workspace_bytes(ctypes.byref(p), 16) > n
    assert lib.seb_sur_workspace_bytes(ctypes.byref(p), 0) == 0 and lib.seb_sur_workspace_bytes(None, 8) == 0
    h = ctypes.c_void_p()
    assert lib.seb_sur_create(None, 8, fake, n, None, ctypes.byref(h)) == INV
    assert lib.seb_sur_create(ctypes.byref(p), 0, fake, n, None, ctypes.byref(h)) == INV
    assert lib.seb_sur_create(ctypes.byref(p), 8, fake, n, None, None) == INV
    assert lib.seb_sur_create(ctypes.byref(p), 8, None, n, None, ctypes.byref(h)) == WS
    assert lib.seb_sur_create(ctypes.byref(p), 8, fake + 64, n, None, ctypes.byref(h)) == WS  # not 256-aligned
    assert lib.seb_sur_create(ctypes.byref(p), 8, fake, n - 1, None, ctypes.byref(h)) == WS
    small = abi.seb_params_default()
    small.nx = small.ny = 32
    assert lib.seb_sur_create(ctypes.byref(small), 8, fake, 1 << 34, None, ctypes.byref(h)) == INV
    half = abi.seb_params_default()
    half.nx = half.ny = 200
    half.elev_dtype = abi.SEB_BF16
    assert lib.seb_sur_create(ctypes.byref(half), 8, fake, 1 << 34, None, ctypes.byref(h)) == INV
    assert lib.seb_sur_destroy(None) == INV
    assert lib.seb_sur_set_stream(None, None) == INV
    assert lib.seb_sur_set_engine(None, abi.SEB_SUR_SIMT) == INV
    assert lib.seb_sur_view_get(None, ctypes.byref(abi.seb_sur_view())) == INV
    assert lib.seb_sur_init(None, 1) == INV
    assert lib.seb_sur_gather(None, fake, fake, 200, 200, fake, 1, 0) == INV
    assert lib.seb_sur_forward(None, 1) == INV
    assert lib.seb_sur_train_step(None, 1, 1e-3, 1, None) == INV
    assert lib.seb_sur_infer(None, fake, 0.04, 3, 1, fake, fake, None) == INV
    buf = ctypes.create_string_buffer(64)
    assert lib.seb_sur_state_bytes(None) == 0 and lib.seb_sur_step(None) == -1
    assert lib.seb_sur_save(None, buf, 64) == INV and lib.seb_sur_load(None, buf, 64) == INV


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libseb.so the binding raises at first use; nothing falls back to a CPU path."""
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "libseb.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        abi.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        abi.seb_params_default()
