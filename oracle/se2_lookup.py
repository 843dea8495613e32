"""FP64 reference of the trilinear SE(2) grid lookup.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the GPU tests compare libseb's
``seb_se2_lookup`` / ``seb_se2_lookup_vjp`` with this function on the same seeded grids and
poses.  It shares no code with the library.

What it computes (Sec. VI: the planner reads Risk and the signed distance field at continuous
states by trilinear interpolation of the SE(2) grid, with the yaw handled on SO(2)):

* Grid value ``V[k][r][c]`` sits at world ``((o_i + c + 1/2) res, (o_j + r + 1/2) res,
  2 pi k / K)``.  Arrays are ring-indexed like the map's outputs:
  ``V[k][(r + ring_y) mod ny][(c + ring_x) mod nx]``.
* A pose ``(x, y, theta)`` has grid coordinates ``u = x / res - o_i - 1/2``,
  ``v = y / res - o_j - 1/2`` and ``w = theta K / (2 pi)`` reduced to ``[0, K)``.
* It is inside when ``0 <= u <= nx - 1`` and ``0 <= v <= ny - 1``.  The cell is
  ``c0 = min(floor(u), nx - 2)`` and ``r0 = min(floor(v), ny - 2)``; the yaw bins are
  ``k0 = floor(w)`` and ``k1 = (k0 + 1) mod K`` (SO(2) wrap).  The fractions are
  ``a = u - c0``, ``b = v - r0`` and ``t = w - k0``.
* The value is the sum over the 8 corners of ``(1 - a or a)(1 - b or b)(1 - t or t) V``.
  The gradient is the derivative of that same trilinear form, scaled to world units:
  ``(d/du / res, d/dv / res, d/dw K / (2 pi))``.
* Outside: value ``fill``, gradient 0, flag UNKNOWN.  A NaN value also sets UNKNOWN.  A pose
  with a non-finite coordinate or ``|theta| > 1e4`` rad counts as outside (an interface rule of
  the library, not of the paper).

Pins: ``tests/test_lookup_pins.py`` (grid nodes, exact reproduction of multilinear
functions, SO(2) periodicity, central differences, scipy's RegularGridInterpolator).
"""
from __future__ import annotations

import numpy as np

UNKNOWN = 1


def se2_lookup(grid, poses, res, origin=(0, 0), ring=(0, 0), fill=np.nan):
    """grid [K][ny][nx], poses [n][3] (x, y, theta) -> (value [n], grad [n][3], flags [n])."""
    V = np.asarray(grid, np.float64)
    K, ny, nx = V.shape
    P = np.asarray(poses, np.float64)
    x, y, th = P[:, 0], P[:, 1], P[:, 2]
    u = x / res - origin[0] - 0.5
    v = y / res - origin[1] - 0.5
    w = np.where(np.abs(th) <= 1e4, th, 0.0) * K / (2.0 * np.pi)
    w = w - K * np.floor(w / K)
    inside = (u >= 0) & (u <= nx - 1) & (v >= 0) & (v <= ny - 1) & (np.abs(th) <= 1e4)
    uc = np.where(inside, u, 0.0)
    vc = np.where(inside, v, 0.0)
    c0 = np.minimum(np.floor(uc), nx - 2).astype(np.int64)
    r0 = np.minimum(np.floor(vc), ny - 2).astype(np.int64)
    k0 = np.floor(w).astype(np.int64)
    t = w - k0
    wrapped = k0 >= K  # w rounded up to K
    k0 = np.where(wrapped, 0, k0)
    t = np.where(wrapped, 0.0, t)
    k1 = (k0 + 1) % K
    a = uc - c0
    b = vc - r0

    def at(k, r, c):
        return V[k, (r + ring[1]) % ny, (c + ring[0]) % nx]

    val = np.zeros(len(P))
    du = np.zeros(len(P))
    dv = np.zeros(len(P))
    dw = np.zeros(len(P))
    for kk, wt, dwt in ((k0, 1 - t, -1.0), (k1, t, 1.0)):
        for rr, wb, dwb in ((r0, 1 - b, -1.0), (r0 + 1, b, 1.0)):
            for cc, wa, dwa in ((c0, 1 - a, -1.0), (c0 + 1, a, 1.0)):
                f = at(kk, rr, cc)
                val += wa * wb * wt * f
                du += dwa * wb * wt * f
                dv += wa * dwb * wt * f
                dw += wa * wb * dwt * f
    grad = np.stack([du / res, dv / res, dw * K / (2.0 * np.pi)], axis=1)
    val = np.where(inside, val, fill)
    grad = np.where(inside[:, None], grad, 0.0)
    flags = np.where(~inside | np.isnan(val), UNKNOWN, 0).astype(np.uint8)
    return val, grad, flags
