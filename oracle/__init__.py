"""FP64 CPU oracle for SE(2)-grid traversability (SEB-Naver, Sec. III, Sec. V-B, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
are the only callers.  The product library never imports this package, and this package
never imports the product library.  The arithmetic lives in ``seb_oracle.c`` (plain C,
FP64, compiled with ``-ffp-contract=off``); this module only builds it and marshals arrays.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  footprint       pinned (closed-form counts, 90-degree transposition, central symmetry,
                  area bounds, hand-listed sets)
  jacobi3         pinned (numpy.linalg.eigh on random SPD and near-degenerate matrices)
  grid / cells    pinned (tilted-plane closed forms at every yaw, flat ground, yaw + pi,
                  offset invariance, hand-computed covariances on tiny maps, risk branches)
  poses           pinned (grid equality at yaw 0 on cell centres, tilted-plane closed forms
                  at continuous yaws)
  poses_vjp       pinned (FP64 central differences of ``poses``)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

UNKNOWN = 1
OBSTACLE = 2
DEGENERATE = 4
CHANNELS = ("z", "pitch", "roll", "rough", "risk")


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, FP64, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("n_yaw", ctypes.c_int),
        ("res", ctypes.c_double),
        ("shape", ctypes.c_int),
        ("length", ctypes.c_double),
        ("width", ctypes.c_double),
        ("kappa_max", ctypes.c_double),
        ("phi_x_max", ctypes.c_double),
        ("phi_y_max", ctypes.c_double),
        ("w", ctypes.c_double * 3),
        ("n_min", ctypes.c_int),
    ]


@dataclasses.dataclass
class OracleParams:
    """Assessment parameters (Algorithm 1 inputs).  phi limits 0.52 rad follow Sec. VII-B;
    kappa_max, w and the footprint extents are not given by the paper."""

    nx: int
    ny: int
    n_yaw: int
    res: float
    length: float
    width: float
    shape: str = "rect"  # "rect" | "ellipse"
    kappa_max: float = 0.1
    phi_x_max: float = 0.52
    phi_y_max: float = 0.52
    w: tuple = (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)
    n_min: int = 0

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.n_yaw = self.nx, self.ny, self.n_yaw
        p.res = self.res
        p.shape = {"rect": 0, "ellipse": 1}[self.shape]
        p.length, p.width = self.length, self.width
        p.kappa_max, p.phi_x_max, p.phi_y_max = self.kappa_max, self.phi_x_max, self.phi_y_max
        p.w = (ctypes.c_double * 3)(*self.w)
        p.n_min = self.n_min
        return p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i64 = ctypes.c_int64
            lib.orc_footprint.argtypes = [P, ctypes.c_int, ip, ip, ctypes.c_int]
            lib.orc_jacobi3.argtypes = [dp, dp, dp]
            lib.orc_grid.argtypes = [P, dp, i64, i64, dp, u8p, dp, ctypes.c_int]
            lib.orc_cells.argtypes = [P, dp, i64, i64, i32p, i64, dp, u8p, dp, ctypes.c_int]
            lib.orc_cell_detail.argtypes = [P, dp, i64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            lib.orc_poses.argtypes = [P, dp, i64, i64, dp, i64, dp, u8p, ctypes.c_int]
            lib.orc_poses_vjp.argtypes = [P, dp, i64, i64, dp, i64, dp, dp, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _threads(n_threads):
    if n_threads is None:
        try:
            return max(1, len(os.sched_getaffinity(0)))
        except AttributeError:  # pragma: no cover
            return os.cpu_count() or 1
    return n_threads


def _elev(params, elev):
    e = np.ascontiguousarray(elev, dtype=np.float64)
    assert e.shape == (params.ny, params.nx), (e.shape, params.ny, params.nx)
    return e


def footprint(params: OracleParams, k: int) -> np.ndarray:
    """Integer offsets [n][2] (di, dj) of yaw bin k, rows outer, ascending."""
    lib = _load()
    p = params._c()
    n = lib.orc_footprint(ctypes.byref(p), k, None, None, 0)
    di = np.zeros(max(n, 1), np.int32)
    dj = np.zeros(max(n, 1), np.int32)
    lib.orc_footprint(ctypes.byref(p), k, _ptr(di, ctypes.c_int), _ptr(dj, ctypes.c_int), n)
    return np.stack([di[:n], dj[:n]], axis=1)


def jacobi3(A: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors (columns) of a symmetric 3x3 matrix."""
    lib = _load()
    A = np.asarray(A, np.float64)
    a6 = np.array([A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]], np.float64)
    ev = np.zeros(3)
    V = np.zeros(9)
    lib.orc_jacobi3(_ptr(a6, ctypes.c_double), _ptr(ev, ctypes.c_double), _ptr(V, ctypes.c_double))
    return ev, V.reshape(3, 3)


def assess_grid(params: OracleParams, elev, origin=(0, 0), n_threads=None, with_gap=False):
    """Every (c, r, k): returns out [5][n_yaw][ny][nx] (z, pitch, roll, rough, risk), flags
    [n_yaw][ny][nx], and with_gap=True also the relative eigen-gap [n_yaw][ny][nx]."""
    lib = _load()
    e = _elev(params, elev)
    out = np.zeros((5, params.n_yaw, params.ny, params.nx))
    flags = np.zeros((params.n_yaw, params.ny, params.nx), np.uint8)
    gap = np.zeros((params.n_yaw, params.ny, params.nx)) if with_gap else None
    p = params._c()
    rc = lib.orc_grid(ctypes.byref(p), _ptr(e, ctypes.c_double), origin[0], origin[1],
                      _ptr(out, ctypes.c_double), _ptr(flags, ctypes.c_uint8),
                      _ptr(gap, ctypes.c_double) if with_gap else None, _threads(n_threads))
    if rc != 0:
        raise ValueError("oracle: bad parameters")
    return (out, flags, gap) if with_gap else (out, flags)


def assess_cells(params: OracleParams, elev, cells, origin=(0, 0), n_threads=None):
    """Listed cells [n][3] (c, r, k): returns out [n][5], flags [n], eigen-gap [n]."""
    lib = _load()
    e = _elev(params, elev)
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 3)
    n = cells.shape[0]
    out = np.zeros((n, 5))
    flags = np.zeros(n, np.uint8)
    gap = np.zeros(n)
    p = params._c()
    rc = lib.orc_cells(ctypes.byref(p), _ptr(e, ctypes.c_double), origin[0], origin[1],
                       _ptr(cells, ctypes.c_int32), n, _ptr(out, ctypes.c_double),
                       _ptr(flags, ctypes.c_uint8), _ptr(gap, ctypes.c_double), _threads(n_threads))
    if rc != 0:
        raise ValueError("oracle: bad parameters or cell index")
    return out, flags, gap


def cell_detail(params: OracleParams, elev, c, r, k, origin=(0, 0)):
    """One cell: (out[5], flags, dict of intermediate quantities)."""
    lib = _load()
    e = _elev(params, elev)
    out = np.zeros(5)
    d = np.zeros(33)
    p = params._c()
    f = lib.orc_cell_detail(ctypes.byref(p), _ptr(e, ctypes.c_double), origin[0], origin[1], c, r, k,
                            _ptr(out, ctypes.c_double), _ptr(d, ctypes.c_double))
    if f < 0:
        raise ValueError("oracle: bad parameters")
    cov = np.array([[d[4], d[5], d[6]], [d[5], d[7], d[8]], [d[6], d[8], d[9]]])
    det = dict(n=int(d[0]), mean=d[1:4].copy(), cov=cov, evals=d[10:13].copy(),
               evecs=d[13:22].reshape(3, 3).copy(), z_b=d[22:25].copy(), x_b=d[25:28].copy(),
               y_b=d[28:31].copy(), u_norm=d[31], gap=d[32])
    return out, f, det


def query_poses(params: OracleParams, elev, poses, origin=(0, 0), n_threads=None):
    """Continuous poses [n][3] (x, y, yaw): out [n][5], flags [n]."""
    lib = _load()
    e = _elev(params, elev)
    poses = np.ascontiguousarray(poses, np.float64).reshape(-1, 3)
    n = poses.shape[0]
    out = np.zeros((n, 5))
    flags = np.zeros(n, np.uint8)
    p = params._c()
    lib.orc_poses(ctypes.byref(p), _ptr(e, ctypes.c_double), origin[0], origin[1],
                  _ptr(poses, ctypes.c_double), n, _ptr(out, ctypes.c_double),
                  _ptr(flags, ctypes.c_uint8), _threads(n_threads))
    return out, flags


def query_poses_vjp(params: OracleParams, elev, poses, grad_out, origin=(0, 0), n_threads=None):
    """Gradient of sum(grad_out * (z, pitch, roll, rough, risk)) w.r.t. poses: [n][3]."""
    lib = _load()
    e = _elev(params, elev)
    poses = np.ascontiguousarray(poses, np.float64).reshape(-1, 3)
    g = np.ascontiguousarray(grad_out, np.float64).reshape(-1, 5)
    n = poses.shape[0]
    gp = np.zeros((n, 3))
    p = params._c()
    lib.orc_poses_vjp(ctypes.byref(p), _ptr(e, ctypes.c_double), origin[0], origin[1],
                      _ptr(poses, ctypes.c_double), n, _ptr(g, ctypes.c_double),
                      _ptr(gp, ctypes.c_double), _threads(n_threads))
    return gp
