"""ctypes binding of libseb's C ABI (include/seb.h), one Python function per C entry point,
same names.  Argument marshalling only: every step of the assessment runs in libseb's CUDA
kernels.  Pointers are plain integers (device addresses); streams are raw cudaStream_t
handles.  A missing libseb.so raises at first use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# SEB_LIBRARY selects another build of the same library (the bounds-checked libseb_debug.so).
LIB_PATH = os.environ.get("SEB_LIBRARY") or os.path.join(_PKG, "libseb.so")

SEB_OK = 0
SEB_ERR_INVALID_ARG = -1
SEB_ERR_BAD_SHAPE = -2
SEB_ERR_CUDA = -3
SEB_ERR_TIMEOUT = -4
SEB_ERR_DEVICE_FAULT = -5
SEB_ERR_WORKSPACE = -6

SEB_RECT, SEB_ELLIPSE = 0, 1
SEB_F32, SEB_BF16, SEB_F16, SEB_BF16_TILED = 0, 1, 2, 3
SEB_PLAIN_F32, SEB_COMPENSATED = 0, 1
SEB_FLAG_UNKNOWN, SEB_FLAG_OBSTACLE, SEB_FLAG_DEGENERATE, SEB_FLAG_FP64 = 1, 2, 4, 8
SEB_FLAG_SURROGATE = 16
SEB_SUR_SIMT, SEB_SUR_TCGEN05 = 0, 1
SEB_N_CH = 5
SEB_QUERY_SAVED = 16
SEB_NOALLOC_MAX_POSES = 65536

# Every extern "C" symbol declared in include/seb.h.
EXPORTS = (
    "seb_params_default",
    "seb_status_string",
    "seb_last_error",
    "seb_footprint_table",
    "seb_workspace_bytes",
    "seb_window_bytes",
    "seb_tiled_base_offset",
    "seb_encode_bf16_tiled",
    "seb_map_create",
    "seb_map_destroy",
    "seb_map_set_stream",
    "seb_map_update",
    "seb_map_shift",
    "seb_map_shift_batch",
    "seb_map_view",
    "seb_map_copy_out",
    "seb_map_check",
    "seb_query_poses",
    "seb_query_poses_backward",
    "seb_query_poses_grad_noalloc",
    "seb_map_grid",
    "seb_se2_lookup",
    "seb_se2_lookup_vjp",
    "seb_sdf_workspace_bytes",
    "seb_risk_sdf",
    "seb_inpaint_workspace_bytes",
    "seb_inpaint_nearest",
    "seb_elev_params_default",
    "seb_elev_workspace_bytes",
    "seb_elev_create",
    "seb_elev_destroy",
    "seb_elev_set_stream",
    "seb_elev_integrate",
    "seb_elev_view_get",
    "seb_elev_copy_out",
    "seb_sur_workspace_bytes",
    "seb_sur_create",
    "seb_sur_destroy",
    "seb_sur_set_stream",
    "seb_sur_view_get",
    "seb_sur_set_engine",
    "seb_sur_init",
    "seb_sur_gather",
    "seb_sur_train_step",
    "seb_sur_forward",
    "seb_sur_infer",
    "seb_sur_state_bytes",
    "seb_sur_save",
    "seb_sur_load",
    "seb_sur_step",
    "seb_terrain_bumpy",
)


class SebError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libseb status {status}: {msg}")
        self.status = status


class seb_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("n_yaw", ctypes.c_int32),
        ("res", ctypes.c_float),
        ("shape", ctypes.c_int32),
        ("length", ctypes.c_float),
        ("width", ctypes.c_float),
        ("kappa_max", ctypes.c_float),
        ("phi_x_max", ctypes.c_float),
        ("phi_y_max", ctypes.c_float),
        ("w", ctypes.c_float * 3),
        ("n_min", ctypes.c_int32),
        ("elev_dtype", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("gap_fp64", ctypes.c_float),
    ]


class seb_grid(ctypes.Structure):
    """One ring-indexed [n_yaw][ny][nx] float32 channel on the device (seb.h)."""
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("n_yaw", ctypes.c_int32),
        ("ring_x", ctypes.c_int32),
        ("ring_y", ctypes.c_int32),
        ("origin_i", ctypes.c_int64),
        ("origin_j", ctypes.c_int64),
        ("res", ctypes.c_float),
    ]


class seb_elev_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("res", ctypes.c_float),
                ("z_min", ctypes.c_float), ("z_max", ctypes.c_float), ("gate", ctypes.c_float),
                ("clear_margin", ctypes.c_float)]


class seb_scan_pose(ctypes.Structure):
    _fields_ = [("R_B", ctypes.c_float * 9), ("p_B", ctypes.c_float * 3), ("R_BS", ctypes.c_float * 9),
                ("p_BS", ctypes.c_float * 3), ("Sigma_S", ctypes.c_float * 9), ("Sigma_R", ctypes.c_float * 9),
                ("Sigma_B", ctypes.c_float * 9)]


class seb_elev_view(ctypes.Structure):
    _fields_ = [("height", ctypes.c_void_p), ("variance", ctypes.c_void_p), ("ring_x", ctypes.c_int32),
                ("ring_y", ctypes.c_int32), ("origin_i", ctypes.c_int64), ("origin_j", ctypes.c_int64)]


class seb_view(ctypes.Structure):
    _fields_ = [
        ("out", ctypes.c_void_p),
        ("flags", ctypes.c_void_p),
        ("ring_x", ctypes.c_int32),
        ("ring_y", ctypes.c_int32),
        ("origin_i", ctypes.c_int64),
        ("origin_j", ctypes.c_int64),
        ("out_offset", ctypes.c_size_t),
        ("flags_offset", ctypes.c_size_t),
        ("last_cells", ctypes.c_int64),
    ]


class seb_sur_view(ctypes.Structure):
    _fields_ = [
        ("n_params", ctypes.c_int64),
        ("n_out", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("master", ctypes.c_size_t),
        ("adam_m", ctypes.c_size_t),
        ("adam_v", ctypes.c_size_t),
        ("grad", ctypes.c_size_t),
        ("weights_bf16", ctypes.c_size_t),
        ("features", ctypes.c_size_t),
        ("labels", ctypes.c_size_t),
        ("act", ctypes.c_size_t * 4),
        ("dact", ctypes.c_size_t * 4),
        ("pred", ctypes.c_size_t),
        ("dpred", ctypes.c_size_t),
        ("map_features", ctypes.c_size_t),
        ("map_act", ctypes.c_size_t * 4),
        ("mask", ctypes.c_size_t),
        ("tiles", ctypes.c_size_t),
        ("partials", ctypes.c_size_t),
        ("loss_partials", ctypes.c_size_t),
        ("totals", ctypes.c_size_t),
        ("off_w", ctypes.c_int64 * 4),
        ("off_b", ctypes.c_int64 * 4),
        ("off_wh", ctypes.c_int64),
        ("off_bh", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def load():
    """Loads libseb.so (built in-tree by paper_2503_02412_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2503_02412_gb300.build` "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(seb_params)
        vp = ctypes.c_void_p
        i32, i64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "seb_params_default": (None, [P]),
            "seb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "seb_last_error": (ctypes.c_char_p, [vp]),
            "seb_footprint_table": (ctypes.c_int, [P, i32, i32p, i32p, i32]),
            "seb_workspace_bytes": (sz, [P]),
            "seb_window_bytes": (sz, [P]),
            "seb_tiled_base_offset": (sz, [i32, i32]),
            "seb_encode_bf16_tiled": (ctypes.c_int, [vp, i32, i32, i64, i64, vp, vp]),
            "seb_map_create": (ctypes.c_int, [P, vp, sz, vp, ctypes.POINTER(vp)]),
            "seb_map_destroy": (ctypes.c_int, [vp]),
            "seb_map_set_stream": (ctypes.c_int, [vp, vp]),
            "seb_map_update": (ctypes.c_int, [vp, vp, i64, i64]),
            "seb_map_shift": (ctypes.c_int, [vp, vp, i64, i64]),
            "seb_map_shift_batch": (ctypes.c_int, [vp, ctypes.POINTER(vp), i64p, i32]),
            "seb_map_view": (ctypes.c_int, [vp, ctypes.POINTER(seb_view)]),
            "seb_map_copy_out": (ctypes.c_int, [vp, vp, vp]),
            "seb_map_check": (ctypes.c_int, [vp, i32, i64p, i64p]),
            "seb_query_poses": (ctypes.c_int, [P, vp, i64, i64, vp, i64, vp, vp, vp, vp]),
            "seb_query_poses_backward": (ctypes.c_int, [P, vp, i64, i64, vp, vp, vp, vp, i64, vp]),
            "seb_query_poses_grad_noalloc": (ctypes.c_int, [P, vp, i64, i64, vp, i64, vp, vp, vp, vp, vp]),
            "seb_map_grid": (ctypes.c_int, [vp, i32, ctypes.POINTER(seb_grid)]),
            "seb_se2_lookup": (ctypes.c_int, [ctypes.POINTER(seb_grid), vp, i64, ctypes.c_float, vp, vp, vp, vp]),
            "seb_se2_lookup_vjp": (ctypes.c_int, [ctypes.POINTER(seb_grid), vp, i64, vp, vp, vp]),
            "seb_sdf_workspace_bytes": (sz, [i32, i32, i32]),
            "seb_risk_sdf": (ctypes.c_int, [ctypes.POINTER(seb_grid), ctypes.c_float, ctypes.c_float, vp, sz, vp, vp]),
            "seb_inpaint_workspace_bytes": (sz, [i32, i32]),
            "seb_inpaint_nearest": (ctypes.c_int, [vp, i32, i32, i32, vp, sz, vp, vp, vp]),
            "seb_elev_params_default": (None, [ctypes.POINTER(seb_elev_params)]),
            "seb_elev_workspace_bytes": (sz, [ctypes.POINTER(seb_elev_params), i64]),
            "seb_elev_create": (ctypes.c_int, [ctypes.POINTER(seb_elev_params), i64, vp, sz, vp, ctypes.POINTER(vp)]),
            "seb_elev_destroy": (ctypes.c_int, [vp]),
            "seb_elev_set_stream": (ctypes.c_int, [vp, vp]),
            "seb_elev_integrate": (ctypes.c_int, [vp, ctypes.POINTER(seb_scan_pose), vp, i64]),
            "seb_elev_view_get": (ctypes.c_int, [vp, ctypes.POINTER(seb_elev_view)]),
            "seb_elev_copy_out": (ctypes.c_int, [vp, vp, vp]),
            "seb_sur_workspace_bytes": (sz, [P, i32]),
            "seb_sur_create": (ctypes.c_int, [P, i32, vp, sz, vp, ctypes.POINTER(vp)]),
            "seb_sur_destroy": (ctypes.c_int, [vp]),
            "seb_sur_set_stream": (ctypes.c_int, [vp, vp]),
            "seb_sur_view_get": (ctypes.c_int, [vp, ctypes.POINTER(seb_sur_view)]),
            "seb_sur_set_engine": (ctypes.c_int, [vp, i32]),
            "seb_sur_init": (ctypes.c_int, [vp, ctypes.c_uint64]),
            "seb_sur_gather": (ctypes.c_int, [vp, vp, vp, i32, i32, vp, i32, i32]),
            "seb_sur_train_step": (ctypes.c_int, [vp, i32, ctypes.c_float, i32, vp]),
            "seb_sur_forward": (ctypes.c_int, [vp, i32]),
            "seb_sur_infer": (ctypes.c_int, [vp, vp, ctypes.c_float, i32, i32, vp, vp, vp]),
            "seb_terrain_bumpy": (ctypes.c_int, [vp, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]),
            "seb_sur_state_bytes": (sz, [vp]),
            "seb_sur_save": (ctypes.c_int, [vp, vp, sz]),
            "seb_sur_load": (ctypes.c_int, [vp, vp, sz]),
            "seb_sur_step": (i64, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc, handle=None):
    if rc != SEB_OK:
        lib = load()
        msg = lib.seb_last_error(handle)
        raise SebError(rc, (msg or b"").decode() or lib.seb_status_string(rc).decode())
    return rc


# ---------------------------------------------------------------- one wrapper per entry point


def seb_params_default() -> seb_params:
    p = seb_params()
    load().seb_params_default(ctypes.byref(p))
    return p


def seb_status_string(status: int) -> str:
    return load().seb_status_string(status).decode()


def seb_last_error(handle=None) -> str:
    return (load().seb_last_error(handle) or b"").decode()


def seb_footprint_table(p: seb_params, k: int):
    """Offsets of yaw bin k as a list of (di, dj) in row-run order (host only)."""
    lib = load()
    n = lib.seb_footprint_table(ctypes.byref(p), k, None, None, 0)
    _check(n if n < 0 else 0)
    di = (ctypes.c_int32 * max(n, 1))()
    dj = (ctypes.c_int32 * max(n, 1))()
    lib.seb_footprint_table(ctypes.byref(p), k, di, dj, n)
    return [(di[i], dj[i]) for i in range(n)]


def seb_workspace_bytes(p: seb_params) -> int:
    return int(load().seb_workspace_bytes(ctypes.byref(p)))


def seb_window_bytes(p: seb_params) -> int:
    return int(load().seb_window_bytes(ctypes.byref(p)))


def seb_tiled_base_offset(nx: int, ny: int) -> int:
    return int(load().seb_tiled_base_offset(nx, ny))


def seb_encode_bf16_tiled(elev_ptr, nx, ny, origin_i, origin_j, out_ptr, stream=0) -> None:
    _check(load().seb_encode_bf16_tiled(elev_ptr, nx, ny, origin_i, origin_j, out_ptr, stream))


def seb_map_create(p: seb_params, workspace_ptr: int, nbytes: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().seb_map_create(ctypes.byref(p), workspace_ptr, nbytes, stream, ctypes.byref(h)))
    return h.value


def seb_map_destroy(handle: int) -> None:
    _check(load().seb_map_destroy(handle))


def seb_map_set_stream(handle: int, stream: int) -> None:
    _check(load().seb_map_set_stream(handle, stream), handle)


def seb_map_update(handle: int, elev_ptr: int, origin_i: int, origin_j: int) -> None:
    _check(load().seb_map_update(handle, elev_ptr, origin_i, origin_j), handle)


def seb_map_shift(handle: int, elev_ptr: int, origin_i: int, origin_j: int) -> None:
    _check(load().seb_map_shift(handle, elev_ptr, origin_i, origin_j), handle)


def seb_map_shift_batch(handle: int, elev_ptrs, origins) -> None:
    """elev_ptrs: n device pointers (ints); origins: n (origin_i, origin_j) pairs."""
    n = len(elev_ptrs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[ctypes.c_void_p(int(x)) for x in elev_ptrs])
    org = (ctypes.c_int64 * max(2 * n, 1))(*[int(v) for o in origins for v in (o[0], o[1])])
    _check(load().seb_map_shift_batch(handle, ptrs, org, n), handle)


def seb_map_view(handle: int) -> seb_view:
    v = seb_view()
    _check(load().seb_map_view(handle, ctypes.byref(v)), handle)
    return v


def seb_map_copy_out(handle: int, out_ptr: int, flags_ptr: int) -> None:
    _check(load().seb_map_copy_out(handle, out_ptr, flags_ptr), handle)


def seb_map_check(handle: int, timeout_ms: int = 10000):
    """Returns (n_fp64, n_degenerate); raises SebError on a device error or timeout."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().seb_map_check(handle, timeout_ms, ctypes.byref(a), ctypes.byref(b)), handle)
    return a.value, b.value


def seb_query_poses(p: seb_params, elev_ptr, origin_i, origin_j, poses_ptr, n, out_ptr, flags_ptr,
                    saved_ptr, stream=0) -> None:
    _check(load().seb_query_poses(ctypes.byref(p), elev_ptr, origin_i, origin_j, poses_ptr, n, out_ptr,
                                  flags_ptr, saved_ptr, stream))


def seb_query_poses_backward(p: seb_params, elev_ptr, origin_i, origin_j, poses_ptr, saved_ptr,
                             grad_out_ptr, grad_pose_ptr, n, stream=0) -> None:
    _check(load().seb_query_poses_backward(ctypes.byref(p), elev_ptr, origin_i, origin_j, poses_ptr,
                                           saved_ptr, grad_out_ptr, grad_pose_ptr, n, stream))


def seb_map_grid(handle, channel) -> seb_grid:
    g = seb_grid()
    _check(load().seb_map_grid(handle, channel, ctypes.byref(g)))
    return g


def seb_se2_lookup(grid: seb_grid, poses_ptr, n, fill, val_ptr, grad_ptr=None, flags_ptr=None, stream=0) -> None:
    _check(load().seb_se2_lookup(ctypes.byref(grid), poses_ptr, n, fill, val_ptr, grad_ptr, flags_ptr, stream))


def seb_se2_lookup_vjp(grid: seb_grid, poses_ptr, n, grad_val_ptr, grad_pose_ptr, stream=0) -> None:
    _check(load().seb_se2_lookup_vjp(ctypes.byref(grid), poses_ptr, n, grad_val_ptr, grad_pose_ptr, stream))


def seb_sdf_workspace_bytes(nx, ny, n_yaw) -> int:
    return load().seb_sdf_workspace_bytes(nx, ny, n_yaw)


def seb_risk_sdf(risk: seb_grid, risk_obstacle, clamp, work_ptr, work_bytes, sdf_ptr, stream=0) -> None:
    _check(load().seb_risk_sdf(ctypes.byref(risk), risk_obstacle, clamp, work_ptr, work_bytes, sdf_ptr, stream))


def seb_inpaint_workspace_bytes(nx, ny) -> int:
    return load().seb_inpaint_workspace_bytes(nx, ny)


def seb_inpaint_nearest(elev_ptr, nx, ny, max_cells, work_ptr, work_bytes, out_ptr, source_ptr=None, stream=0) -> None:
    _check(load().seb_inpaint_nearest(elev_ptr, nx, ny, max_cells, work_ptr, work_bytes, out_ptr, source_ptr, stream))


def seb_elev_params_default() -> seb_elev_params:
    p = seb_elev_params()
    load().seb_elev_params_default(ctypes.byref(p))
    return p


def seb_elev_workspace_bytes(p: seb_elev_params, max_points) -> int:
    return load().seb_elev_workspace_bytes(ctypes.byref(p), max_points)


def seb_elev_create(p: seb_elev_params, max_points, ws_ptr, nbytes, stream=0):
    h = ctypes.c_void_p()
    _check(load().seb_elev_create(ctypes.byref(p), max_points, ws_ptr, nbytes, stream, ctypes.byref(h)))
    return h.value


def seb_elev_destroy(h) -> None:
    load().seb_elev_destroy(h)


def seb_elev_set_stream(h, stream) -> None:
    _check(load().seb_elev_set_stream(h, stream))


def seb_elev_integrate(h, pose: seb_scan_pose, points_ptr, n) -> None:
    _check(load().seb_elev_integrate(h, ctypes.byref(pose), points_ptr, n))


def seb_elev_view_get(h) -> seb_elev_view:
    v = seb_elev_view()
    _check(load().seb_elev_view_get(h, ctypes.byref(v)))
    return v


def seb_elev_copy_out(h, height_ptr, variance_ptr) -> None:
    _check(load().seb_elev_copy_out(h, height_ptr, variance_ptr))


def seb_query_poses_grad_noalloc(p: seb_params, elev_ptr, origin_i, origin_j, poses_ptr, n, grad_out_ptr, out_ptr,
                                 flags_ptr, grad_pose_ptr, stream=0) -> None:
    """Forward + backward of the pose query without any device allocation (saved state in the
    library's own device array; at most SEB_NOALLOC_MAX_POSES poses per call)."""
    _check(load().seb_query_poses_grad_noalloc(ctypes.byref(p), elev_ptr, origin_i, origin_j, poses_ptr, n,
                                               grad_out_ptr, out_ptr, flags_ptr, grad_pose_ptr, stream))


def seb_sur_workspace_bytes(p: seb_params, max_batch: int) -> int:
    return int(load().seb_sur_workspace_bytes(ctypes.byref(p), max_batch))


def seb_sur_create(p: seb_params, max_batch: int, workspace_ptr: int, nbytes: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().seb_sur_create(ctypes.byref(p), max_batch, workspace_ptr, nbytes, stream, ctypes.byref(h)))
    return h.value


def seb_sur_destroy(handle: int) -> None:
    _check(load().seb_sur_destroy(handle))


def seb_sur_set_stream(handle: int, stream: int) -> None:
    _check(load().seb_sur_set_stream(handle, stream))


def seb_sur_view_get(handle: int) -> seb_sur_view:
    v = seb_sur_view()
    _check(load().seb_sur_view_get(handle, ctypes.byref(v)))
    return v


def seb_sur_set_engine(handle: int, engine: int) -> None:
    _check(load().seb_sur_set_engine(handle, engine))


def seb_sur_init(handle: int, seed: int) -> None:
    _check(load().seb_sur_init(handle, seed))


def seb_sur_gather(handle, elev_ptr, exact_ptr, nx, ny, centres_ptr, n, offset) -> None:
    _check(load().seb_sur_gather(handle, elev_ptr, exact_ptr, nx, ny, centres_ptr, n, offset))


def seb_sur_train_step(handle, batch, lr, step, loss_ptr=0) -> None:
    _check(load().seb_sur_train_step(handle, batch, lr, step, loss_ptr))


def seb_sur_forward(handle, batch) -> None:
    _check(load().seb_sur_forward(handle, batch))


def seb_sur_infer(handle, elev_ptr, step, radius, exact_fallback, out_ptr, flags_ptr, mask_ptr=0) -> None:
    _check(load().seb_sur_infer(handle, elev_ptr, step, radius, exact_fallback, out_ptr, flags_ptr, mask_ptr))


def seb_sur_state_bytes(handle) -> int:
    return int(load().seb_sur_state_bytes(handle))


def seb_sur_save(handle) -> bytes:
    """Checkpoint image of the training state (blocking: synchronises the handle's stream)."""
    n = seb_sur_state_bytes(handle)
    buf = ctypes.create_string_buffer(n)
    _check(load().seb_sur_save(handle, buf, n))
    return buf.raw


def seb_sur_load(handle, image: bytes) -> None:
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    _check(load().seb_sur_load(handle, buf, len(image)))


def seb_sur_step(handle) -> int:
    return int(load().seb_sur_step(handle))


def seb_terrain_bumpy(params_ptr, n, nx, ny, res, seed, out_ptr, stream=0) -> None:
    _check(load().seb_terrain_bumpy(params_ptr, n, nx, ny, res, seed, out_ptr, stream))
