"""FP64 reference of the SE(2) signed distance field of the obstacle set.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the GPU tests compare libseb's
``seb_risk_sdf`` with this function on the same seeded grids.  It shares no code with the
library.

What it computes (Sec. VI: the planner's collision term uses an SDF over SE(2) whose value at a
state is the distance to the edge of the nearest region, negative inside obstacles; the paper
builds it from the risk map):

* Per yaw bin k, the obstacle set O_k is the cells whose risk is at least ``risk_obstacle``
  (1 by default: the explicit obstacles of Algorithm 1, unknown cells included) or NaN (an
  unknown value counts as an obstacle, as unknown cells do in Algorithm 1); the free set F_k
  is every other cell of the window.
* Distances are Euclidean between cell centres in the (x, y) plane of that bin, in metres:
  ``sdf = res * (min_{o in O_k} |p - o| - min_{f in F_k} |p - f|)``.  One of the two terms is
  0, so a free cell gets its distance to the nearest obstacle and an obstacle cell minus its
  distance to the nearest free cell.  An empty set contributes +inf, and the result is clamped
  to ``[-clamp, clamp]``.
* Cells are in the window's logical order; arrays are ring-indexed like the map's outputs
  (the ring wrap is storage, not adjacency).

This is the definition evaluated by brute force (every cell against every cell of the other
set), restricted to the requested cells.  Pins: ``tests/test_sdf_pins.py`` (scipy's exact
Euclidean distance transform, a single obstacle, a half-plane, empty and full sets).
"""
from __future__ import annotations

import numpy as np


def _logical(grid, ring):
    K, ny, nx = grid.shape
    r = (np.arange(ny) + ring[1]) % ny
    c = (np.arange(nx) + ring[0]) % nx
    return grid[:, r[:, None], c[None, :]]


def risk_sdf(risk, res, risk_obstacle=1.0, clamp=np.inf, ring=(0, 0), cells=None):
    """risk [K][ny][nx] (ring-indexed) -> sdf.  With cells=None the whole grid is returned
    ring-indexed [K][ny][nx]; otherwise cells [m][3] = (c, r, k) in logical order and the
    result is [m]."""
    R = _logical(np.asarray(risk, np.float64), ring)
    K, ny, nx = R.shape
    if cells is None:
        kk, rr, cc = np.meshgrid(np.arange(K), np.arange(ny), np.arange(nx), indexing="ij")
        cells = np.stack([cc.ravel(), rr.ravel(), kk.ravel()], 1)
        whole = True
    else:
        cells = np.asarray(cells, np.int64)
        whole = False
    out = np.empty(len(cells))
    for k in np.unique(cells[:, 2]):
        sel = np.nonzero(cells[:, 2] == k)[0]
        obst = ~(R[k] < risk_obstacle)  # NaN: obstacle
        oy, ox = np.nonzero(obst)
        fy, fx = np.nonzero(~obst)
        py = cells[sel, 1].astype(np.float64)
        px = cells[sel, 0].astype(np.float64)

        def nearest(ty, tx):
            if len(ty) == 0:
                return np.full(len(sel), np.inf)
            best = np.full(len(sel), np.inf)
            for s in range(0, len(ty), 4096):  # chunks keep the pair matrix small
                d2 = (py[:, None] - ty[None, s:s + 4096]) ** 2 + (px[:, None] - tx[None, s:s + 4096]) ** 2
                best = np.minimum(best, d2.min(axis=1))
            return np.sqrt(best)

        d = res * (nearest(oy, ox) - nearest(fy, fx))
        out[sel] = np.clip(d, -clamp, clamp)
    if not whole:
        return out
    L = out.reshape(K, ny, nx)
    G = np.empty_like(L)
    r = (np.arange(ny) + ring[1]) % ny
    c = (np.arange(nx) + ring[0]) % nx
    G[:, r[:, None], c[None, :]] = L
    return G
