"""Seeded synthetic terrain shaped like the paper's scenes (Sec. VII-A uses procedurally
generated mountains and forests and real LiDAR maps; neither is available here).

Recipes (all elevations in metres, maps row-major ``[ny][nx]`` with x fastest, NaN = unknown):

* ``bumpy_plane``: tilted plane tan(U[0, 15 deg]) * (cos a * x + sin a * y), a ~ U[0, 2 pi),
  plus 8 Gaussian bumps (amplitude U[-0.5, 0.5] m, sigma U[0.3, 1.5] m, centres uniform
  over the map) plus N(0, 0.01 m) noise.  Small map: 100 x 100 at 0.1 m.
* ``fractal_steps_nan``: 6-octave value noise (base wavelength 8 m, lacunarity 2,
  persistence 0.5, scaled to a peak |z| of 0.8 m), 3 step edges along random lines
  (+U[0.05, 0.3] m on one side) and NaN discs of radius U[0.1, 0.5] m added until 5 %
  of the cells are unknown.  Full local map: 400 x 400 at 0.05 m.
* ``fractal_world``: the same recipe on a larger world, from which rolling windows are cut.
* ``random_poses``: x, y uniform inside the map inset by a margin, yaw uniform [0, 2 pi).
"""
from __future__ import annotations

import numpy as np


def tilted_plane(nx, ny, res, alpha, beta, gamma, origin=(0, 0)):
    """z = alpha * x + beta * y + gamma at the cell centres ((o + c + 1/2) * res)."""
    oi, oj = origin
    x = (oi + np.arange(nx) + 0.5) * res
    y = (oj + np.arange(ny) + 0.5) * res
    return (alpha * x[None, :] + beta * y[:, None] + gamma).astype(np.float64)


def bumpy_plane(seed, nx=100, ny=100, res=0.1, n_bumps=8, noise=0.01, dtype=np.float32):
    rng = np.random.default_rng(seed)
    slope = np.tan(np.deg2rad(rng.uniform(0.0, 15.0)))
    az = rng.uniform(0.0, 2 * np.pi)
    x = (np.arange(nx) + 0.5) * res
    y = (np.arange(ny) + 0.5) * res
    X, Y = np.meshgrid(x, y)
    z = slope * (np.cos(az) * X + np.sin(az) * Y)
    w, h = nx * res, ny * res
    for _ in range(n_bumps):
        amp = rng.uniform(-0.5, 0.5)
        sig = rng.uniform(0.3, 1.5)
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        z += amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sig * sig))
    z += rng.normal(0.0, noise, size=z.shape)
    return z.astype(dtype)


def _value_noise(rng, nx, ny, res, wavelength):
    """One octave of value noise: random lattice values with smoothstep interpolation."""
    gx = int(np.ceil(nx * res / wavelength)) + 2
    gy = int(np.ceil(ny * res / wavelength)) + 2
    lat = rng.uniform(-1.0, 1.0, size=(gy, gx))
    u = (np.arange(nx) + 0.5) * res / wavelength
    v = (np.arange(ny) + 0.5) * res / wavelength
    i0 = np.floor(u).astype(np.int64)
    j0 = np.floor(v).astype(np.int64)
    fu = u - i0
    fv = v - j0
    su = fu * fu * (3 - 2 * fu)
    sv = fv * fv * (3 - 2 * fv)
    a = lat[j0][:, i0]
    b = lat[j0][:, i0 + 1]
    c = lat[j0 + 1][:, i0]
    d = lat[j0 + 1][:, i0 + 1]
    top = a + (b - a) * su[None, :]
    bot = c + (d - c) * su[None, :]
    return top + (bot - top) * sv[:, None]


def _fractal(rng, nx, ny, res, octaves=6, base=8.0, lacunarity=2.0, persistence=0.5, peak=0.8):
    z = np.zeros((ny, nx))
    amp, wl = 1.0, base
    for _ in range(octaves):
        z += amp * _value_noise(rng, nx, ny, res, wl)
        amp *= persistence
        wl /= lacunarity
    z *= peak / np.max(np.abs(z))
    return z


def _steps(rng, z, res, n_steps=3):
    ny, nx = z.shape
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * res, (np.arange(ny) + 0.5) * res)
    for _ in range(n_steps):
        px, py = rng.uniform(0, nx * res), rng.uniform(0, ny * res)
        ang = rng.uniform(0, 2 * np.pi)
        side = (X - px) * np.sin(ang) - (Y - py) * np.cos(ang) > 0
        z = z + np.where(side, rng.uniform(0.05, 0.3), 0.0)
    return z


def _nan_discs(rng, z, res, frac=0.05):
    ny, nx = z.shape
    mask = np.zeros_like(z, dtype=bool)
    target = frac * nx * ny
    count = 0
    while count < target:
        r = rng.uniform(0.1, 0.5) / res
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        x0, x1 = max(0, int(cx - r) - 1), min(nx, int(cx + r) + 2)
        y0, y1 = max(0, int(cy - r) - 1), min(ny, int(cy + r) + 2)
        yy, xx = np.mgrid[y0:y1, x0:x1]
        disc = (xx + 0.5 - cx) ** 2 + (yy + 0.5 - cy) ** 2 <= r * r
        count += int((disc & ~mask[y0:y1, x0:x1]).sum())
        mask[y0:y1, x0:x1] |= disc
    z = z.copy()
    z[mask] = np.nan
    return z


def fractal_steps_nan(seed, nx=400, ny=400, res=0.05, nan_frac=0.05, dtype=np.float32):
    rng = np.random.default_rng(seed)
    z = _fractal(rng, nx, ny, res)
    z = _steps(rng, z, res)
    if nan_frac > 0:
        z = _nan_discs(rng, z, res, nan_frac)
    return z.astype(dtype)


def fractal_world(seed, n=2000, res=0.05, nan_frac=0.05, dtype=np.float32):
    """A large world (n x n cells) from which robot-centric windows are cut."""
    return fractal_steps_nan(seed, n, n, res, nan_frac, dtype)


def shift_sequence(seed, n_shifts=50, step=10):
    """Shifts of round(step * (cos phi, sin phi)) cells, phi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0, 2 * np.pi, size=n_shifts)
    return [(int(np.rint(step * np.cos(p))), int(np.rint(step * np.sin(p)))) for p in phi]


def random_poses(seed, n, nx, ny, res, margin_cells, origin=(0, 0), dtype=np.float32):
    """Poses [n, 3] = (x, y, yaw) in world metres, inset by margin_cells from the window edge."""
    rng = np.random.default_rng(seed)
    oi, oj = origin
    x = (oi + rng.uniform(margin_cells, nx - margin_cells, size=n)) * res
    y = (oj + rng.uniform(margin_cells, ny - margin_cells, size=n)) * res
    th = rng.uniform(0.0, 2 * np.pi, size=n)
    return np.stack([x, y, th], axis=1).astype(dtype)


def random_se2_grid(seed, n_yaw, ny, nx, nan_frac=0.0, dtype=np.float32):
    """A [n_yaw][ny][nx] grid of N(0, 1) values with a fraction of NaN entries."""
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(n_yaw, ny, nx))
    if nan_frac > 0:
        g[rng.random(g.shape) < nan_frac] = np.nan
    return g.astype(dtype)


def lookup_poses(seed, n, nx, ny, res, origin=(0, 0), pad_cells=2.0, yaw_range=20.0, dtype=np.float32):
    """Poses [n, 3] spread over the window and pad_cells beyond it (so some fall outside),
    with yaw uniform in [-yaw_range, yaw_range] (several turns, both signs)."""
    rng = np.random.default_rng(seed)
    oi, oj = origin
    x = (oi + 0.5 + rng.uniform(-pad_cells, nx - 1 + pad_cells, size=n)) * res
    y = (oj + 0.5 + rng.uniform(-pad_cells, ny - 1 + pad_cells, size=n)) * res
    th = rng.uniform(-yaw_range, yaw_range, size=n)
    return np.stack([x, y, th], axis=1).astype(dtype)


def obstacle_risk(seed, n_yaw, ny, nx, n_blobs=12, blob_cells=(2, 12), nan_frac=0.0, dtype=np.float32):
    """A [n_yaw][ny][nx] risk grid: U[0, 0.9) everywhere, and risk 1 inside n_blobs discs per
    yaw bin (radius U[blob_cells] cells, centres uniform), plus an optional NaN fraction."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, 0.9, size=(n_yaw, ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx]
    for k in range(n_yaw):
        for _ in range(n_blobs):
            cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
            rad = rng.uniform(*blob_cells)
            r[k][(yy - cy) ** 2 + (xx - cx) ** 2 <= rad * rad] = 1.0
    if nan_frac > 0:
        r[rng.random(r.shape) < nan_frac] = np.nan
    return r.astype(dtype)


def _rot_zyx(yaw, pitch, roll):
    cy, sy, cp, sp, cr, sr = np.cos(yaw), np.sin(yaw), np.cos(pitch), np.sin(pitch), np.cos(roll), np.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
    Ry = np.array([[cp, 0, sp], [0, 1.0, 0], [-sp, 0, cp]])
    Rx = np.array([[1.0, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def lidar_scan(seed, world, res, x, y, yaw=0.0, n_rings=32, n_az=1024, fov_deg=(-15.0, 15.0), max_range=12.0,
               body_height=0.45, p_BS=(0.1, 0.0, 0.25), tilt_deg=2.0, range_noise=0.01):
    """A synthetic spinning-LiDAR scan of a world heightfield [ny][nx] (world cell (i, j) centred
    at ((i + 1/2) res, (j + 1/2) res); NaN cells are not hit).

    The body sits body_height above the terrain at (x, y) with heading yaw and a random tilt of
    up to tilt_deg; the sensor, at p_BS in the body frame with the body's attitude, casts
    n_rings x n_az rays (elevations uniform over fov_deg, azimuths uniform) and each ray stops at
    the first sample, every res / 2, below the terrain (nearest cell), plus N(0, range_noise)
    range noise.  Returns (R_B, p_B, R_BS, p_BS, points [m][3] in the sensor frame, float32)."""
    rng = np.random.default_rng(seed)
    z = np.asarray(world, np.float64)
    ny, nx = z.shape

    def height(px, py):
        i = np.clip(np.floor(px / res).astype(np.int64), 0, nx - 1)
        j = np.clip(np.floor(py / res).astype(np.int64), 0, ny - 1)
        return z[j, i]

    g = height(np.array([x]), np.array([y]))[0]
    g = 0.0 if np.isnan(g) else g
    R_B = _rot_zyx(yaw, *np.deg2rad(rng.uniform(-tilt_deg, tilt_deg, 2)))
    p_B = np.array([x, y, g + body_height])
    R_BS = np.eye(3)
    p_BS = np.asarray(p_BS, np.float64)
    origin = R_B @ p_BS + p_B
    el = np.deg2rad(np.linspace(fov_deg[0], fov_deg[1], n_rings))
    az = np.linspace(0, 2 * np.pi, n_az, endpoint=False)
    E, A = np.meshgrid(el, az, indexing="ij")
    d_s = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    d_w = d_s @ (R_B @ R_BS).T
    steps = np.arange(1, int(max_range / (res / 2)) + 1) * (res / 2)
    pts = origin[None, None, :] + steps[None, :, None] * d_w[:, None, :]
    below = pts[..., 2] <= height(pts[..., 0], pts[..., 1])
    hit = below.any(axis=1)
    first = np.argmax(below, axis=1)
    r = steps[first[hit]] + rng.normal(0.0, range_noise, hit.sum())
    sensor_pts = d_s[hit] * r[:, None]
    return R_B, p_B, R_BS, p_BS, sensor_pts.astype(np.float32)
