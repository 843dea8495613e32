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
