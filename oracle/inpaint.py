"""FP64 reference of nearest-neighbour inpainting of the elevation map.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the GPU tests compare libseb's
``seb_inpaint_nearest`` with this function on the same seeded maps.  It shares no code with
the library.

What it computes (Sec. V-A: the elevation map is inpainted before the traversability pass;
Sec. VII-B: the compared pipelines fill unknown cells by nearest-neighbour interpolation):

* Every unknown (NaN) cell takes the elevation of the known cell whose centre is nearest in
  Euclidean distance; among equally near known cells, the one with the smallest column index,
  then the smallest row index (logical order) is taken.
* Known cells keep their value.  With ``max_cells > 0``, an unknown cell whose nearest known
  cell is farther than ``max_cells`` cells stays NaN; a map without known cells stays NaN.

The definition is evaluated by brute force (every unknown cell against every known cell).
Pins: ``tests/test_inpaint_pins.py`` (scipy's exact distance transform for the distances,
hand-built ties, a single known cell, the radius, the all-unknown map).
"""
from __future__ import annotations

import numpy as np


def inpaint_nearest(elev, max_cells=0):
    """elev [ny][nx] (NaN = unknown) -> (filled [ny][nx], source [ny][nx][2] = (row, col) of
    the known cell each value came from, -1 where none)."""
    z = np.asarray(elev, np.float64)
    ny, nx = z.shape
    out = z.copy()
    src = np.full((ny, nx, 2), -1, np.int64)
    known = ~np.isnan(z)
    kr, kc = np.nonzero(known)
    src[kr, kc, 0] = kr
    src[kr, kc, 1] = kc
    ur, uc = np.nonzero(~known)
    if len(kr) == 0 or len(ur) == 0:
        return out, src
    # candidates sorted by (col, row) so that the first minimum is the tie-break winner
    order = np.lexsort((kr, kc))
    kr, kc = kr[order], kc[order]
    step = max(1, (1 << 23) // len(kr))  # rows of the pair matrix per chunk (~64 MB)
    for s in range(0, len(ur), step):
        r = ur[s:s + step, None]
        c = uc[s:s + step, None]
        d2 = (r - kr[None, :]) ** 2 + (c - kc[None, :]) ** 2
        best = np.argmin(d2, axis=1)  # first occurrence: smallest (col, row) among the nearest
        bd2 = d2[np.arange(len(best)), best]
        ok = np.ones(len(best), bool) if max_cells <= 0 else bd2 <= max_cells * max_cells
        rr, cc = ur[s:s + step][ok], uc[s:s + step][ok]
        out[rr, cc] = z[kr[best[ok]], kc[best[ok]]]
        src[rr, cc, 0] = kr[best[ok]]
        src[rr, cc, 1] = kc[best[ok]]
    return out, src
