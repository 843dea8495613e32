"""Element-wise comparison of the CUDA path with the FP64 oracle (shared by the GPU tests).

Tolerances (FP32 kernel vs FP64 oracle):
  z <= 1e-4 m, pitch/roll <= 1e-4 rad, risk <= 1e-4, roughness <= 3e-5 (risk carries
  w0 / kappa_max = 3.33 x roughness, so 3e-5 keeps risk within 1e-4).
Cells whose oracle value lies within the tolerance of the compared quantity of a risk
threshold (roughness within 3e-5 of kappa_max, |pitch| / |roll| within 1e-4 of phi_x_max /
phi_y_max) may legitimately take the other branch in FP32; they are counted, not failed.
Cells flagged DEGENERATE by either side are excluded from the value checks (their outputs
are NaN by definition); the UNKNOWN bit is an integer decision and must match exactly.

Ill-conditioned cells are checked against a bound that grows with the conditioning, not
skipped.  The kernel's moment sums are FP32, so its covariance carries an error ||dC|| of a few
u tr(C) (u = 2^-24, the unit roundoff).  By the Davis-Kahan sin-theta theorem the normal then
moves by ||dC|| / (lambda_mid - lambda_min) = (a few u) / g radians, g = (lambda_mid -
lambda_min) / trace the oracle's relative eigen-gap, whichever eigen-solve follows (the kernel
redoes small-gap solves in FP64).  The body frame built from the normal (Eqs. 2-3) amplifies a
normal error by about 1 / n_z (|n x x_yaw| = n_z / cos(roll)), and the plane height at the cell
centre moves by the normal's error times the footprint mean's offset (at most the reach R) over
n_z^2.  Hence, per cell, with B = C_GAP u / (g n_z), n_z from the oracle's frame:
  pitch, roll   <= max(1e-4, B)
  z             <= max(1e-4, B R / n_z)
  roughness     <= 3e-5                   (an eigenvalue moves by ||dC|| only: no gap division)
  risk          <= max(1e-4, B (w1 / phi_x + w2 / phi_y) + 1e-4)   where B > 1e-4
and the risk branch may flip where an oracle angle lies within max(1e-4, B) of its limit.
C_GAP = 16: on near-degenerate footprints (gaps down to 3e-8 and normals up to horizontal) the
largest measured |angle error| g n_z / u was about 3.  Cells whose B exceeds 1e-4 are the
ill-conditioned ones: ordinary terrain has g >~ 1e-2 and n_z ~ 1, so B < 1e-4 and the plain
tolerance applies; their number and the largest |error| / bound are reported (`ill`,
`ill_ratio`).
"""
import numpy as np

TOL = {0: 1e-4, 1: 1e-4, 2: 1e-4, 3: 3e-5, 4: 1e-4}
U32 = 2.0 ** -24
C_GAP = 16.0
UNKNOWN, OBSTACLE, DEGENERATE, FP64 = 1, 2, 4, 8


def ill_bound(gap, nz=1.0):
    """Angle bound B (rad) of a cell with relative eigen-gap `gap` and normal z-component `nz`
    (see the module docstring)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return C_GAP * U32 / np.maximum(gap * nz, 1e-300)


def near_threshold(ref, kappa_max=0.1, phi_x=0.52, phi_y=0.52, margin=None, angle_margin=None):
    """ref: [..., 5] oracle outputs -> bool mask of cells whose roughness / |pitch| / |roll|
    lies within its tolerance (or the given margin; angle_margin, a scalar or per-cell array,
    overrides it for the angles) of the matching risk threshold."""
    mk = TOL[3] if margin is None else margin
    ma = TOL[1] if margin is None else margin
    if angle_margin is not None:
        ma = angle_margin
    with np.errstate(invalid="ignore"):
        return ((np.abs(ref[..., 3] - kappa_max) < mk) | (np.abs(np.abs(ref[..., 1]) - phi_x) < ma)
                | (np.abs(np.abs(ref[..., 2]) - phi_y) < ma))


def compare(gpu, gflags, ref, rflags, kappa_max=0.1, phi_x=0.52, phi_y=0.52, tol=None, label="", gap=None,
            reach_m=0.6, w=(1 / 3, 1 / 3, 1 / 3)):
    """gpu/ref: [n, 5]; flags [n]; gap: the oracle's relative eigen-gaps [n] (optional);
    reach_m: the footprint's largest offset in metres (0.6 covers the 0.9 x 0.6 m and
    0.6 x 0.4 m footprints).  Returns a dict of statistics; raises AssertionError on a violation
    outside the stated exclusions."""
    tol = dict(TOL, **(tol or {}))
    gflags = gflags.astype(np.uint8) & 7
    rflags = rflags.astype(np.uint8) & 7
    assert np.array_equal(gflags & UNKNOWN, rflags & UNKNOWN), f"{label}: UNKNOWN bits differ"
    near = near_threshold(ref, kappa_max, phi_x, phi_y)
    degen = ((gflags | rflags) & DEGENERATE) != 0
    n = len(gpu)
    with np.errstate(invalid="ignore"):
        sp, sr = np.sin(ref[:, 1]), np.sin(ref[:, 2])
        nz = np.sqrt(np.clip(1.0 - sp * sp - sr * sr, 1e-12, 1.0))
    ill = np.zeros(n, bool)
    bound = np.zeros(n)
    if gap is not None:
        with np.errstate(invalid="ignore"):
            b = np.where(np.isfinite(gap), ill_bound(gap, nz), 0.0)
            ill = (b > tol[1]) & ((rflags & UNKNOWN) == 0) & ~degen
        bound = np.where(ill, b, 0.0)
        near = near | (ill & near_threshold(ref, kappa_max, phi_x, phi_y, angle_margin=np.maximum(bound, tol[1])))
    assessed = ((rflags & UNKNOWN) == 0) & ~degen
    flag_mismatch = (gflags != rflags) & ~near & ~degen
    if flag_mismatch.any():
        i = np.flatnonzero(flag_mismatch)[:4]
        raise AssertionError(f"{label}: {flag_mismatch.sum()} flag mismatches away from thresholds; "
                             f"idx {i.tolist()} gpu {gpu[i].tolist()} {gflags[i].tolist()} "
                             f"ref {ref[i].tolist()} {rflags[i].tolist()}")
    stats = dict(n=n, assessed=int(assessed.sum()), near=int((near & assessed).sum()),
                 degenerate=int(degen.sum()), ill=int(ill.sum()), ill_ratio=0.0)
    # per-cell tolerance of each channel: the plain tolerance, widened for ill-conditioned cells
    limit = {ch: np.full(n, tol[ch]) for ch in range(5)}
    limit[1] = np.maximum(tol[1], bound)
    limit[2] = np.maximum(tol[2], bound)
    limit[0] = np.maximum(tol[0], bound * reach_m / nz)
    limit[4] = np.maximum(tol[4], np.where(ill, bound * (w[1] / phi_x + w[2] / phi_y) + tol[4], 0.0))
    errors = []
    for ch in range(5):
        sel = assessed & ~(near if ch == 4 else np.zeros_like(near))
        d = np.abs(gpu[sel, ch].astype(np.float64) - ref[sel, ch])
        lim = limit[ch][sel]
        plain = ~ill[sel]
        mx = float(d[plain].max()) if plain.any() else 0.0
        stats[f"max{ch}"] = mx
        stats[f"p99_{ch}"] = float(np.percentile(d[plain], 99)) if plain.any() else 0.0
        if (~plain).any():
            stats[f"ill_max{ch}"] = float(d[~plain].max())
            stats["ill_ratio"] = max(stats["ill_ratio"], float((d[~plain] / lim[~plain]).max()))
        bad = ~(d <= lim)
        if bad.any():
            i = np.flatnonzero(sel)[np.flatnonzero(bad)[:4]]
            errors.append(f"{label}: channel {ch}: {int(bad.sum())} cells above their bound; max |err| "
                          f"{float(d[bad].max()):.3e}; idx {i.tolist()} gpu {gpu[i, ch].tolist()} "
                          f"ref {ref[i, ch].tolist()} gap {None if gap is None else gap[i].tolist()} "
                          f"n_z {nz[i].tolist()}")
    if errors:
        raise AssertionError("\n".join(errors))
    flips = (np.abs(gpu[:, 4] - ref[:, 4]) > limit[4]) & assessed & near
    stats["flips"] = int(flips.sum())
    assert stats["flips"] <= stats["near"]
    if stats["ill"]:
        print(f"{label}: {stats['ill']} ill-conditioned cells checked against C_GAP u / (gap n_z), "
              f"largest |error| / bound {stats['ill_ratio']:.3g}")
    return stats


def grid_to_rows(out, flags, gap=None):
    """[5][K][ny][nx] + [K][ny][nx] -> rows [K*ny*nx, 5] and flags in (k, r, c) order."""
    if gap is None:
        return out.reshape(5, -1).T, flags.reshape(-1)
    return out.reshape(5, -1).T, flags.reshape(-1), gap.reshape(-1)
