"""FP64 reference of the elevation-map update from a LiDAR scan (Sec. V-A).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the GPU tests compare libseb's
``seb_elev_*`` calls with this module on the same seeded scans.  It shares no code with the
library.

The state is a robot-centred window of nx x ny cells (height h and variance s2 per cell, NaN =
unknown) whose storage is indexed by world cell index mod n, like the assessment map.  One scan
(robot pose, LiDAR extrinsics, covariances, points in the sensor frame) is integrated in the
order of Sec. V-A:

1. Window (Eq. pm): the map frame sits at res * floor(p_B / res); the window origin is that cell
   minus (nx / 2, ny / 2), so the robot stays at the centre.  Cells that were not inside the
   previous window become unknown.
2. Ray casting: for every point whose (x, y) lies in the window, each cell the segment from the
   sensor to the point crosses in (x, y) (the point's own cell excluded) is cleared (unknown) if
   its height exceeds the highest height of the ray over that cell, plus ``clear_margin``.  The
   cells and the ray's entry / exit parameters come from the slab method on every cell of the
   segment's bounding box, and the cells' heights are those before this scan.
3. Points outside the window are ignored; the others are taken to the body frame and kept when
   their body-frame height lies in [z_min, z_max].  A kept point has world height
   z = b3^T (R_B (R_BS p + p_BS) + p_B) and variance (the three Jacobian terms of Sec. V-A)
   s2 = J_S^T Sigma_S J_S + J_R^T Sigma_R J_R + J_B^T Sigma_B J_B with J_S = (R_B R_BS)^T b3,
   J_R = (R_BS p + p_BS)^ R_B^T b3 and J_B = -b3.
4. One-dimensional Kalman fusion per cell, in information form: against the estimate (h, s2)
   from before this scan, a point with (z - h) / sqrt(s2) > gate lies above the gate, one within
   [-gate, gate] inside it, one below is dropped.  If a cell has points above the gate it is
   reset to the fusion of those points (a higher surface); otherwise its estimate is fused with
   the points inside the gate; an unknown cell takes the fusion of all its points.  Fusion:
   1 / s2' = [1 / s2] + sum 1 / s2_i and h' = s2' ([h / s2] + sum z_i / s2_i).

Readings of Sec. V-A behind these steps: the world height uses + p_B (a rigid transform; the
sign reaches the variance only through J_B, which enters squared); the window is the robot's
cell minus half the map size (Eq. (pm)); ray casting clears a crossed cell whose height exceeds
the ray's top over it by more than clear_margin; several points in a cell are fused against the
pre-scan estimate with the Mahalanobis gate above.  Pins are in ``tests/test_elevation_pins.py``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

B3 = np.array([0.0, 0.0, 1.0])


@dataclasses.dataclass
class ElevParams:
    nx: int
    ny: int
    res: float
    z_min: float = -1.0
    z_max: float = 1.0
    gate: float = 2.5
    clear_margin: float = 0.05


@dataclasses.dataclass
class ScanPose:
    R_B: np.ndarray          # body -> world
    p_B: np.ndarray          # body position in the world
    R_BS: np.ndarray         # sensor -> body
    p_BS: np.ndarray         # sensor position in the body frame
    Sigma_S: np.ndarray      # point covariance (sensor model)
    Sigma_R: np.ndarray      # body attitude covariance (right perturbation)
    Sigma_B: np.ndarray      # body position covariance


def skew(q):
    return np.array([[0.0, -q[2], q[1]], [q[2], 0.0, -q[0]], [-q[1], q[0], 0.0]])


def window_origin(p, pose: ScanPose):
    """Eq. (pm): the window's first cell, with the robot's cell at (nx / 2, ny / 2)."""
    return (int(np.floor(pose.p_B[0] / p.res)) - p.nx // 2, int(np.floor(pose.p_B[1] / p.res)) - p.ny // 2)


def point_heights(pose: ScanPose, pts):
    """World points, body-frame heights and height variances of sensor-frame points [n][3]."""
    P = np.asarray(pts, np.float64)
    body = P @ pose.R_BS.T + pose.p_BS
    world = body @ pose.R_B.T + pose.p_B
    JS = (pose.R_B @ pose.R_BS).T @ B3
    RtB = pose.R_B.T @ B3
    s2 = np.empty(len(P))
    for i in range(len(P)):
        JR = skew(body[i]) @ RtB
        s2[i] = JS @ pose.Sigma_S @ JS + JR @ pose.Sigma_R @ JR + B3 @ pose.Sigma_B @ B3
    return world, body[:, 2], s2


class ElevationMap:
    """store_f32: round the stored heights and variances to float32 after every scan, so that
    the next scan's gate and clearing decisions are taken on the values a float32 map holds."""

    def __init__(self, p: ElevParams, store_f32=False):
        self.p = p
        self.store_f32 = store_f32
        self.h = np.full((p.ny, p.nx), np.nan)   # storage: [world j mod ny][world i mod nx]
        self.s2 = np.full((p.ny, p.nx), np.nan)
        self.origin = None

    # logical (window) <-> storage
    def _idx(self, c, r):
        return (self.origin[1] + r) % self.p.ny, (self.origin[0] + c) % self.p.nx

    def logical(self):
        """(h, s2) [ny][nx] in window order."""
        r, c = np.mgrid[0:self.p.ny, 0:self.p.nx]
        pr, pc = self._idx(c, r)
        return self.h[pr, pc], self.s2[pr, pc]

    def _move(self, o):
        p = self.p
        if self.origin is not None:
            r, c = np.mgrid[0:p.ny, 0:p.nx]
            wi, wj = o[0] + c, o[1] + r  # world indices of the new window
            stay = (wi >= self.origin[0]) & (wi < self.origin[0] + p.nx) & (wj >= self.origin[1]) & \
                   (wj < self.origin[1] + p.ny)
            pr, pc = wj % p.ny, wi % p.nx
            self.h[pr[~stay], pc[~stay]] = np.nan
            self.s2[pr[~stay], pc[~stay]] = np.nan
        self.origin = o

    def _raycast(self, sensor, world, inside):
        """Cells to clear: (storage row, col) list, using the heights before this scan."""
        p = self.p
        res = p.res
        clear = set()
        sx, sy, sz = sensor
        for (x, y, z) in world[inside]:
            dx, dy, dz = x - sx, y - sy, z - sz
            # cells of the bounding box, in world indices
            i0, i1 = int(np.floor(min(sx, x) / res)), int(np.floor(max(sx, x) / res))
            j0, j1 = int(np.floor(min(sy, y) / res)), int(np.floor(max(sy, y) / res))
            pi, pj = int(np.floor(x / res)), int(np.floor(y / res))
            for wi in range(i0, i1 + 1):
                # candidate rows of this column: the segment's y-range over the column's x-range,
                # widened by one cell (the slab test below decides every candidate)
                if dx != 0.0:
                    ta, tb = sorted(((wi * res - sx) / dx, ((wi + 1) * res - sx) / dx))
                    ta, tb = max(ta, 0.0), min(tb, 1.0)
                    ya, yb = sorted((sy + dy * ta, sy + dy * tb))
                    jlo, jhi = max(j0, int(np.floor(ya / res)) - 1), min(j1, int(np.floor(yb / res)) + 1)
                else:
                    jlo, jhi = j0, j1
                for wj in range(jlo, jhi + 1):
                    if (wi, wj) == (pi, pj):
                        continue
                    c, r = wi - self.origin[0], wj - self.origin[1]
                    if not (0 <= c < p.nx and 0 <= r < p.ny):
                        continue
                    # slab method: t-interval of the segment inside the cell's (x, y) box
                    lo, hi = 0.0, 1.0
                    for d, s, a in ((dx, sx, wi * res), (dy, sy, wj * res)):
                        b = a + res
                        if d == 0.0:
                            if not (a <= s < b):
                                lo, hi = 1.0, 0.0
                            continue
                        t0, t1 = (a - s) / d, (b - s) / d
                        lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
                    if not hi > lo:
                        continue
                    ray_top = max(sz + dz * lo, sz + dz * hi)  # the ray is linear in t
                    pr, pc = wj % p.ny, wi % p.nx
                    if self.h[pr, pc] > ray_top + p.clear_margin:
                        clear.add((pr, pc))
        return clear

    def integrate(self, pose: ScanPose, pts):
        p = self.p
        o = window_origin(p, pose)
        self._move(o)
        world, zb, s2 = point_heights(pose, pts)
        fin = np.isfinite(world).all(axis=1)
        wi = np.floor(world[:, 0] / p.res)
        wj = np.floor(world[:, 1] / p.res)
        inside = fin & (wi >= o[0]) & (wi < o[0] + p.nx) & (wj >= o[1]) & (wj < o[1] + p.ny)
        sensor = pose.R_B @ pose.p_BS + pose.p_B
        for (pr, pc) in self._raycast(sensor, world, inside):
            self.h[pr, pc] = np.nan
            self.s2[pr, pc] = np.nan
        keep = inside & (zb >= p.z_min) & (zb <= p.z_max)
        acc = {}
        h0, v0 = self.h.copy(), self.s2.copy()  # estimates before this scan's fusion
        for k in np.nonzero(keep)[0]:
            pr, pc = int(wj[k]) % p.ny, int(wi[k]) % p.nx
            a = acc.setdefault((pr, pc), [0.0, 0.0, 0.0, 0.0, 0])  # in-gate w, wz; above w, wz; n above
            z, w = world[k, 2], 1.0 / s2[k]
            if np.isnan(h0[pr, pc]):
                a[0] += w
                a[1] += w * z
                continue
            d = (z - h0[pr, pc]) / np.sqrt(v0[pr, pc])
            if d > p.gate:
                a[2] += w
                a[3] += w * z
                a[4] += 1
            elif d >= -p.gate:
                a[0] += w
                a[1] += w * z
        for (pr, pc), a in acc.items():
            if a[4] > 0:
                self.s2[pr, pc] = 1.0 / a[2]
                self.h[pr, pc] = a[3] / a[2]
            elif a[0] > 0:
                if np.isnan(h0[pr, pc]):
                    W, WZ = a[0], a[1]
                else:
                    W, WZ = a[0] + 1.0 / v0[pr, pc], a[1] + h0[pr, pc] / v0[pr, pc]
                self.s2[pr, pc] = 1.0 / W
                self.h[pr, pc] = WZ / W
        if self.store_f32:
            self.h = self.h.astype(np.float32).astype(np.float64)
            self.s2 = self.s2.astype(np.float32).astype(np.float64)
        return o
