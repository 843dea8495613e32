// SE(2)-grid traversability assessment kernels (Algorithm 1 of Sec. V-B for every cell and
// yaw bin), plus the ring-unrolling copy.
//
// Two kernels share the finish (finish_cell).  Both run one CTA per tile of cells and yaw pair
// {k, k + K/2}: the two bins share a footprint, so their moments, normal and roughness are
// computed once, and pitch and roll change sign.  The tile and its footprint halo are staged in
// shared memory (cells outside the window read as NaN = unknown, Sec. V-A).
//   - assess_kernel_sl (every footprint whose staged tile fits): cells in world-aligned blocks of
//     4 columns x 2 rows, one block per thread, sliding row sums on packed FP32 pairs, the tile
//     staged by one TMA copy; see the block comment above the kernel.
//   - assess_kernel (very large footprints): each thread owns 4 adjacent cells of one row and walks
//     the yaw's row runs with a 4-wide register window, so one shared-memory load feeds 4 cells.
//
// Moments are accumulated about a reference height (the sliding kernel: one per block, the
// per-cell kernel: the cell's own elevation, or the first known footprint cell in run order when
// the centre is unknown): S0 = sum z', S1 = sum di z', S2 = sum dj z', S3 = sum z'^2, z' = z - ref.
// The xy moments (N, sum di, ..., sum dj^2) are exact integers: the table's minus those of the
// missing points.  Every cell's arithmetic therefore depends on its neighbourhood only, never on
// the tile position, which makes the rolling update bit-identical to a full rebuild.
//
// Covariance (population, /N, Algorithm 1) from the moments; smallest eigenpair by the
// trigonometric closed form for symmetric 3x3 matrices (O. K. Smith, "Eigenvalues of a
// symmetric 3 x 3 matrix", CACM 4(4), 1961), eigenvector as the largest cross product of
// two rows of Cov - lambda_min I, roughness from the Rayleigh quotient n^T Cov n.  A
// relative eigen-gap below gap_fp64 redoes the eigen-solve in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>
#include <type_traits>

#include "seb_device.cuh"
#include "seb_internal.h"

namespace seb {

// Element tag of SEB_BF16_TILED windows: a BF16 offset from the FP32 base of its 16 x 16 tile.
struct Bf16Tiled {
  __nv_bfloat16 v;
};
template <>
__device__ __forceinline__ float to_f32<Bf16Tiled>(Bf16Tiled v) {
  return __bfloat162float(v.v);
}

namespace {

// Height of in-window cell (gx, gy) of the launch's elevation window.
template <typename E>
__device__ __forceinline__ float load_elev(const Launch& L, int gx, int gy) {
  return to_f32<E>(static_cast<const E*>(L.elev)[(int64_t)gy * L.nx + gx]);
}
template <>
__device__ __forceinline__ float load_elev<Bf16Tiled>(const Launch& L, int gx, int gy) {
  const float base = __ldg(&L.tile_base[((gy + L.base_py) >> 4) * L.base_tx + ((gx + L.base_px) >> 4)]);
  return base + to_f32<Bf16Tiled>(static_cast<const Bf16Tiled*>(L.elev)[(int64_t)gy * L.nx + gx]);
}
// Height from a staged raw element of cell (gx, gy) (out of the window: the raw value is NaN).
template <typename E>
__device__ __forceinline__ float stage_elev(const Launch& L, E raw, int gx, int gy) {
  return to_f32<E>(raw);
}
template <>
__device__ __forceinline__ float stage_elev<Bf16Tiled>(const Launch& L, Bf16Tiled raw, int gx, int gy) {
  const float d = to_f32<Bf16Tiled>(raw);
  if (gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) return d;
  return __ldg(&L.tile_base[((gy + L.base_py) >> 4) * L.base_tx + ((gx + L.base_px) >> 4)]) + d;
}

// Algorithm 1 from the moments on: covariance, normal, roughness, frame (Eqs. 2-3),
// pitch/roll at heading (ct, st), fitted-plane height at the cell centre, risk.
__device__ __noinline__ Cell finish_cell(int N, int MX, int MY, int MXX, int MXY, int MYY, float S0,
                                         float S1, float S2, float S3, float ref, int n_min,
                                         float ct, float st, const Launch& L, int n_full = 0,
                                         float inv_n_full = 0.f) {
  Cell o;
  const float qnan = __int_as_float(0x7fc00000);
  if (N < n_min) {
    o.z = o.pitch = o.roll = o.rough = qnan;
    o.risk = 1.f;
    o.flags = SEB_FLAG_UNKNOWN | SEB_FLAG_OBSTACLE;
    return o;
  }
  const float res = L.res;
  const float fN = (float)N;
  // exact reciprocal (the means use it); a complete footprint takes the table's 1/N, the same
  // correctly rounded value the division gives
  const float iN = N == n_full ? inv_n_full : 1.f / fN;
  const float inv_n2 = iN * iN;
  // N^2 Cov_xy-block numerators are exact integers (int32 when the tables allow it: 64-bit
  // integer conversions run on the FP64 unit).
  float nxx, nxy, nyy;
  if (L.narrow_moments) {
    nxx = (float)(N * MXX - MX * MX);
    nxy = (float)(N * MXY - MX * MY);
    nyy = (float)(N * MYY - MY * MY);
  } else {
    nxx = (float)((long long)N * MXX - (long long)MX * MX);
    nxy = (float)((long long)N * MXY - (long long)MX * MY);
    nyy = (float)((long long)N * MYY - (long long)MY * MY);
  }
  const float fMX = (float)MX, fMY = (float)MY;
  const float rr2 = inv_n2 * res * res, rr1 = inv_n2 * res;
  float c[6];
  c[0] = nxx * rr2;
  c[1] = nxy * rr2;
  c[3] = nyy * rr2;
  c[2] = fmaf(S1, fN, -fMX * S0) * rr1;
  c[4] = fmaf(S2, fN, -fMY * S0) * rr1;
  c[5] = fmaf(S3, fN, -S0 * S0) * inv_n2;
  float n[3], gap;
  min_eigpair_f(c, n, &gap);
  uint32_t flags = 0;
  const float tr = c[0] + c[3] + c[5];
  if (gap < L.gap_fp64) {
    // Small relative eigen-gap: covariance and eigen-solve again in FP64 from the same moments.
    flags |= SEB_FLAG_FP64;
    const double dN = (double)N, i2 = 1.0 / (dN * dN), r = (double)res;
    double cd[6];
    cd[0] = ((double)N * MXX - (double)MX * MX) * i2 * r * r;
    cd[1] = ((double)N * MXY - (double)MX * MY) * i2 * r * r;
    cd[3] = ((double)N * MYY - (double)MY * MY) * i2 * r * r;
    cd[2] = ((double)S1 * dN - (double)MX * (double)S0) * i2 * r;
    cd[4] = ((double)S2 * dN - (double)MY * (double)S0) * i2 * r;
    cd[5] = ((double)S3 * dN - (double)S0 * (double)S0) * i2;
    double nd[3], gd;
    min_eigpair<double>(cd, nd, &gd);
    const double ld = refine_min<double>(cd, nd);
    n[0] = (float)nd[0];
    n[1] = (float)nd[1];
    n[2] = (float)nd[2];
    o.rough = (float)(ld / (cd[0] + cd[3] + cd[5]));
    atomicAdd(&L.counters[0], 1ull);
    if (gd < 1e-12) flags |= SEB_FLAG_DEGENERATE;
  } else {
    // The closed-form eigenvalue is accurate to ~eps * trace; below a relative gap of 0.05 one
    // Rayleigh-quotient refinement keeps the normal within 1e-5 rad.
    const float lam = gap < 0.05f ? refine_min<float>(c, n) : fmaxf(rayleigh<float>(c, n), 0.f);
    o.rough = __fdividef(lam, tr);  // 2-ulp division: far inside the 1e-4 bar
  }
  // Body frame (Eqs. 2-3): u = z_b x x_yaw = (-n_z s, n_z c, n_x s - n_y c),
  // y_b = u / |u|, x_b = y_b x z_b, so b3^T x_b = -n_z (n_x c + n_y s) / |u|.
  const float uz = n[0] * st - n[1] * ct;
  const float un2 = n[2] * n[2] + uz * uz;
  if (!(n[2] > 1e-6f) || !(un2 >= 1e-12f)) flags |= SEB_FLAG_DEGENERATE;
  if (flags & SEB_FLAG_DEGENERATE) {
    o.z = o.pitch = o.roll = qnan;
    o.risk = 1.f;
    o.flags = flags | SEB_FLAG_OBSTACLE;
    atomicAdd(&L.counters[1], 1ull);
    return o;
  }
  const float iun = rsqrtf(un2);
  const float ybz = fminf(fmaxf(uz * iun, -1.f), 1.f);
  const float xbz = fminf(fmaxf(-n[2] * (n[0] * ct + n[1] * st) * iun, -1.f), 1.f);
  o.pitch = asinf(xbz);
  o.roll = asinf(ybz);
  // Plane through the mean with normal n, evaluated at the cell centre (offset 0).
  o.z = ref + S0 * iN + (n[0] * fMX + n[1] * fMY) * iN * res * __fdividef(1.f, n[2]);
  const float ap = fabsf(o.pitch), ar = fabsf(o.roll);
  if (o.rough > L.kappa_max || ap > L.phi_x_max || ar > L.phi_y_max) {
    o.risk = 1.f;
    flags |= SEB_FLAG_OBSTACLE;
  } else {
    o.risk = L.w0 * (o.rough * L.inv_kappa_max) + L.w1 * (ap * L.inv_phi_x_max) + L.w2 * (ar * L.inv_phi_y_max);
  }
  o.flags = flags;
  return o;
}

__device__ __forceinline__ int unpack(uint32_t v, int sh) { return (int)((v >> sh) & 0xffu) - 128; }

// Moments of the kG cells of this thread for yaw pair `pair`, run by run.  A run whose rows
// (over the warp's cells) hold no unknown cell takes the plain path: 4 FP32 operations per
// (point, cell).  Otherwise the masked path replaces unknown heights by 0 with a 0 weight
// (z' = fma(-ref, m, z_known), exactly z - ref for known points) and accumulates the integer
// moments of the missing points, Q = (n, sum di, sum dj, sum di^2, sum di dj, sum dj^2), which
// are later subtracted from the table's.  Both paths give bit-identical moments for a run
// without unknown cells, so the choice (made per warp) never changes a result.
template <bool COMP>
__device__ __forceinline__ void accumulate(const Tables& T, int pair, const float* __restrict__ sc, int sw,
                                           const int* __restrict__ rowflag_warp, int rpw,
                                           const float ref[kG], float S0[kG], float S1[kG], float S2[kG],
                                           float S3[kG], float Q[6][kG]) {
  float C0[kG], C1[kG], C2[kG], C3[kG];  // compensation terms (COMP)
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    S0[g] = S1[g] = S2[g] = S3[g] = 0.f;
    C0[g] = C1[g] = C2[g] = C3[g] = 0.f;
#pragma unroll
    for (int t = 0; t < 6; ++t) Q[t][g] = 0.f;
  }
  const int lane = threadIdx.x & 31;
  const int r0 = T.run_start[pair], r1 = T.run_start[pair + 1];
  for (int q = r0; q < r1; ++q) {
    const uint32_t pk = T.runs[q];
    const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
    int f = 0;
    for (int r = lane; r < rpw; r += 32) f |= rowflag_warp[dj + r];
    const bool masked = __any_sync(0xffffffffu, f);
    const float* p = sc + dj * sw + lo;
    const int len = hi - lo + 1;
    float a[kG], ac[kG], b[kG], bc[kG], s3[kG], s3c[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) a[g] = ac[g] = b[g] = bc[g] = s3[g] = s3c[g] = 0.f;
    if (!masked) {
      float w0 = p[0], w1 = p[1], w2 = p[2];
      float di = (float)lo;
#pragma unroll 2
      for (int i = 0; i < len; ++i) {
        const float w3 = p[i + 3];
        const float wv[kG] = {w0, w1, w2, w3};
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          const float zp = wv[g] - ref[g];
          if (COMP) {
            nadd(a[g], ac[g], zp);
            nadd(b[g], bc[g], __fmul_rn(di, zp));
            nadd(s3[g], s3c[g], __fmul_rn(zp, zp));
          } else {
            a[g] += zp;
            b[g] = fmaf(di, zp, b[g]);
            s3[g] = fmaf(zp, zp, s3[g]);
          }
        }
        w0 = w1;
        w1 = w2;
        w2 = w3;
        di += 1.f;
      }
    } else {
      // window of (known height or 0, known weight, missing weight)
      float z0, z1, z2, m0, m1, m2, x0, x1, x2;
      auto split = [](float v, float& z, float& m, float& x) {
        const bool k = v == v;
        z = k ? v : 0.f;
        m = k ? 1.f : 0.f;
        x = k ? 0.f : 1.f;
      };
      split(p[0], z0, m0, x0);
      split(p[1], z1, m1, x1);
      split(p[2], z2, m2, x2);
      float qn[kG], qx[kG], qxx[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) qn[g] = qx[g] = qxx[g] = 0.f;
      float di = (float)lo;
#pragma unroll 2
      for (int i = 0; i < len; ++i) {
        float z3, m3, x3;
        split(p[i + 3], z3, m3, x3);
        const float zs[kG] = {z0, z1, z2, z3}, ms[kG] = {m0, m1, m2, m3}, xs[kG] = {x0, x1, x2, x3};
        const float di2 = di * di;
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          const float zp = fmaf(-ref[g], ms[g], zs[g]);
          if (COMP) {
            nadd(a[g], ac[g], zp);
            nadd(b[g], bc[g], __fmul_rn(di, zp));
            nadd(s3[g], s3c[g], __fmul_rn(zp, zp));
          } else {
            a[g] += zp;
            b[g] = fmaf(di, zp, b[g]);
            s3[g] = fmaf(zp, zp, s3[g]);
          }
          qn[g] += xs[g];
          qx[g] = fmaf(di, xs[g], qx[g]);
          qxx[g] = fmaf(di2, xs[g], qxx[g]);
        }
        z0 = z1;
        z1 = z2;
        z2 = z3;
        m0 = m1;
        m1 = m2;
        m2 = m3;
        x0 = x1;
        x1 = x2;
        x2 = x3;
        di += 1.f;
      }
      const float fdj = (float)dj;
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        Q[0][g] += qn[g];
        Q[1][g] += qx[g];
        Q[2][g] = fmaf(fdj, qn[g], Q[2][g]);
        Q[3][g] += qxx[g];
        Q[4][g] = fmaf(fdj, qx[g], Q[4][g]);
        Q[5][g] = fmaf(fdj * fdj, qn[g], Q[5][g]);
      }
    }
    const float fdj = (float)dj;
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      if (COMP) {
        const float at = a[g] + ac[g];
        nadd(S0[g], C0[g], at);
        nadd(S1[g], C1[g], b[g] + bc[g]);
        nadd(S2[g], C2[g], __fmul_rn(fdj, at));
        nadd(S3[g], C3[g], s3[g] + s3c[g]);
      } else {
        S0[g] += a[g];
        S1[g] += b[g];
        S2[g] = fmaf(fdj, a[g], S2[g]);
        S3[g] += s3[g];
      }
    }
  }
  if (COMP) {
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      S0[g] += C0[g];
      S1[g] += C1[g];
      S2[g] += C2[g];
      S3[g] += C3[g];
    }
  }
}

template <typename E, bool COMP>
__global__ void __launch_bounds__(kThreads, 2)
    assess_kernel(const __grid_constant__ Tables T, const __grid_constant__ Launch L) {
  extern __shared__ float smem[];
  int* rowflag = reinterpret_cast<int*>(smem);  // per staged row: holds an unknown cell
  float* tile = smem + kMaxStageRows;
  if (blockDim.x != kThreads || blockIdx.y >= (unsigned)T.n_pairs) {
    if (threadIdx.x == 0) atomicOr(L.err, kErrLaunchShape);
    return;
  }
  // Which rectangle and tile this CTA covers, and the rectangle's layout.
  const int b = blockIdx.x;
  if (L.tile_active && !L.tile_active[b]) return;  // uniform per CTA, before any barrier
  int ri = 0;
#pragma unroll 1
  while (ri + 1 < L.n_rects && b >= L.tile_start[ri + 1]) ++ri;
  const Rect R = L.rects[ri];
  const int lg = R.log_tpr;
  const int tw = kG << lg, th = kThreads >> lg;
  const int t = b - L.tile_start[ri];
  const int tx0 = R.tx + (t % L.tiles_x[ri]) * tw;
  const int ty0 = R.ty + (t / L.tiles_x[ri]) * th;
  const int rx = T.rx, ry = T.ry;
  const int sw = stage_w(lg, rx), sh = stage_h(lg, ry);

  for (int i = threadIdx.x; i < sh; i += kThreads) rowflag[i] = 0;
  __syncthreads();
  // Stage tile + halo (outside the window = NaN = unknown).
  const float qnan = __int_as_float(0x7fc00000);
  for (int idx = threadIdx.x; idx < sw * sh; idx += kThreads) {
    const int row = idx / sw, col = idx - row * sw;
    const int gy = ty0 - ry + row, gx = tx0 - rx + col;
    float v = qnan;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) v = load_elev<E>(L, gx, gy);
    if (v != v) rowflag[row] = 1;
    tile[idx] = v;
  }
  __syncthreads();

  const int lx = (threadIdx.x & ((1 << lg) - 1)) * kG;
  const int ly = threadIdx.x >> lg;
  const int rpw = 32 >> lg > 0 ? 32 >> lg : 1;  // cell rows per warp
  const int ly_w0 = (threadIdx.x & ~31) >> lg;
  const int cx = tx0 + lx, cy = ty0 + ly;
  const int pair = blockIdx.y;
  const float* sc = tile + (ry + ly) * sw + rx + lx;  // centre of cell g is sc[g]

  float ref[kG];
#pragma unroll
  for (int g = 0; g < kG; ++g) ref[g] = sc[g];
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    if (ref[g] == ref[g]) continue;
    // Unknown centre: the first known cell of the footprint in run order.
    float r = 0.f;
    bool found = false;
    for (int q = T.run_start[pair]; q < T.run_start[pair + 1] && !found; ++q) {
      const uint32_t pk = T.runs[q];
      const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
      for (int d = lo; d <= hi; ++d) {
        const float v = sc[dj * sw + g + d];
        if (v == v) {
          r = v;
          found = true;
          break;
        }
      }
    }
    ref[g] = r;
  }

  float S0[kG], S1[kG], S2[kG], S3[kG], Q[6][kG];
  accumulate<COMP>(T, pair, sc, sw, rowflag + ry + ly_w0, rpw, ref, S0, S1, S2, S3, Q);

  if (cy >= R.y0 + R.h) return;
  const int k0 = pair, k1 = pair + T.n_pairs;
  const float ct = T.cos_t[pair], st = T.sin_t[pair];
  int pr = cy + L.ring_y;
  if (pr >= L.ny) pr -= L.ny;
  const int64_t chs = (int64_t)L.n_yaw * L.plane;
  const int* mom = T.mom[pair];
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    const int c = cx + g;
    if (c >= R.x0 + R.w) break;
    if (L.store_mask && !L.store_mask[(int64_t)cy * L.nx + c]) continue;
    const Cell o = finish_cell(mom[0] - (int)Q[0][g], mom[1] - (int)Q[1][g], mom[2] - (int)Q[2][g],
                               mom[3] - (int)Q[3][g], mom[4] - (int)Q[4][g], mom[5] - (int)Q[5][g], S0[g], S1[g],
                               S2[g], S3[g], ref[g], T.n_min[pair], ct, st, L);
    int pc = c + L.ring_x;
    if (pc >= L.nx) pc -= L.nx;
    const int64_t i0 = (int64_t)k0 * L.plane + (int64_t)pr * L.nx + pc;
    const int64_t i1 = (int64_t)k1 * L.plane + (int64_t)pr * L.nx + pc;
    float* out = L.out;
    out[i0] = o.z;
    out[i1] = o.z;
    out[chs + i0] = o.pitch;
    out[chs + i1] = -o.pitch;
    out[2 * chs + i0] = o.roll;
    out[2 * chs + i1] = -o.roll;
    out[3 * chs + i0] = o.rough;
    out[3 * chs + i1] = o.rough;
    out[4 * chs + i0] = o.risk;
    out[4 * chs + i1] = o.risk;
    L.flags[i0] = (uint8_t)o.flags;
    L.flags[i1] = (uint8_t)o.flags;
  }
}

// ------------------------------------------------------------------------------------------------
// Plain-precision kernel with sliding row sums on packed FP32 pairs.
//
// Cells are grouped in blocks of 4 columns x 2 rows aligned to the global grid (global column
// = 0 mod 4, global row = 0 mod 2), one block per thread, so that the grouping of a cell never
// depends on the tile or on the window origin.  The two rows of a block are processed as FP32x2
// pairs (__fadd2_rn / __ffma2_rn, each half rounded like the scalar forms) from a staged tile
// of vertical pairs (T[r][c], T[r+1][c]).  All cells of a block are centred on one reference
// height (the block's first known cell, else the first known footprint cell in run order).
// For each row run (dj, lo, hi) only the first column of the block is summed point by point,
// A = sum z', Bx = sum p z', C = sum z'^2 (p = column offset from the block's first column);
// the next columns follow by sliding the run one cell:
//   A_g = A_{g-1} - z'(lo+g-1) + z'(hi+g), Bx_g = Bx_{g-1} - (lo+g-1) z'(lo+g-1) + (hi+g) z'(hi+g),
//   C_g = C_{g-1} - z'(lo+g-1)^2 + z'(hi+g)^2, and sum di z' = Bx_g - g A_g for column g.
// Runs whose rows (over the warp) hold an unknown cell use weights m (z' = fma(-ref, m, z)) and
// slide the moments of the missing points the same way; both paths give bit-identical sums
// for runs without unknown cells.
// Layouts.  Quad layouts (log2 of blocks per row): 3 -> 32 x 64 cells, 2 -> 16 x 128, 5 -> 128 x 16;
// a half-warp holds 4 blocks x 4 block rows, and alternate pair rows are skewed so that its
// 8-byte reads hit 16 distinct slots (32 banks).  Column layouts kColLay + W (W = 3 or 5 blocks
// per row, 80 or 48 block rows) tile the column bands of a rolling shift that are 12 or 20 cells
// wide without computing cells outside them: thread t holds block column t / H, block row t % H,
// so a half-warp reads 16 pair rows 2 apart in one column; an odd row stride (in 8-byte slots) and
// a one-slot skew every 16 rows keep those 16 reads distinct.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return f2(-a.x, -a.y); }

constexpr int kColLay = 16;
__host__ __device__ inline bool sl_col(int lay) { return lay >= kColLay; }
// blocks per row and block rows of a tile
__host__ __device__ inline int sl_bw(int lay) { return sl_col(lay) ? lay - kColLay : 1 << lay; }
__host__ __device__ inline int sl_bh(int lay) {
  return sl_col(lay) ? (kThreads / (lay - kColLay)) & ~15 : kThreads >> lay;
}
__host__ __device__ inline int sl_tw(int lay) { return 4 * sl_bw(lay); }
__host__ __device__ inline int sl_th(int lay) { return 2 * sl_bh(lay); }
// staged row stride in float2 slots (room for the skew) and the skew (r >> ks) & km of a layout
__host__ __device__ inline int sl_sw2(int lay, int rx) {
  const int w = sl_tw(lay) + 2 * rx;
  return sl_col(lay) ? ((w + 1) | 1) : (w + 3 + 7) & ~7;
}
__host__ __device__ inline int sl_skew_shift(int lay) { return sl_col(lay) ? 4 : 1; }
__host__ __device__ inline int sl_skew_mask(int lay) { return sl_col(lay) ? 1 : 3; }
__device__ __forceinline__ int sl_index(int r, int c, int sw2, int ks, int km) { return r * sw2 + c + ((r >> ks) & km); }
constexpr int kSlQ = 6 * 4;  // missing-point moments per thread: [k][g], both rows in one int32

// Tensor maps of the elevation for the TMA staging, one per tile layout (index stage_map()).
constexpr int kStageMaps = 5;
struct StageMaps {
  CUtensorMap map[kStageMaps];
};
__host__ __device__ inline int stage_map(int lay) {
  return lay == 2 ? 0 : lay == 3 ? 1 : lay == 5 ? 2 : lay == kColLay + 3 ? 3 : 4;
}
// Width of the TMA box of a layout: the staged width plus the slack of rounding the box's first
// column down to a multiple of q = 16 bytes / element size, rounded up to a multiple of q.
__host__ __device__ inline int stage_box_w(int lay, int rx, int q) {
  return (sl_tw(lay) + 2 * rx + q - 1 + q - 1) / q * q;
}
constexpr int kStageWaitPolls = 1 << 20;  // bounded wait for the staged tile

// Kahan's compensated step (W. Kahan, "Further remarks on reducing truncation errors", CACM 8(1),
// 1965) on packed pairs: s - c tracks the sum of the added terms (c holds minus the low-order
// part the last additions lost).
__device__ __forceinline__ void kadd2(float2& s, float2& c, float2 x) {
  const float2 y = add2(x, neg2(c));
  const float2 t = add2(s, y);
  c = add2(add2(t, neg2(s)), neg2(y));
  s = t;
}

// COMP (SEB_COMPENSATED): every accumulation over the row runs (the column-0 sums and the slide
// differences) is Kahan-compensated; the sums within one run (at most ~20 terms of one row) stay
// plain FP32.
template <typename E, bool COMP>
__global__ void __launch_bounds__(kThreads, 2)
    assess_kernel_sl(const __grid_constant__ Tables T, const __grid_constant__ Launch L,
                     const __grid_constant__ StageMaps SM) {
  extern __shared__ float smem[];
  int* rowflag = reinterpret_cast<int*>(smem);
  float2* qs = reinterpret_cast<float2*>(smem + kMaxStageRows);  // TMA box scratch: kSlQ x kThreads slots
  float2* pt = qs + kSlQ * kThreads;                             // [sh - 1][sw2] vertical pairs
  // No global memory access before the stream's previous kernel has completed (pdl_entry) ...
  // except in a later launch of one shift batch: its input window was written before the batch
  // began, and the batch's first launch waited for that before any later launch could start, so
  // it stages and computes at once and waits for the previous launch only before its first store.
  if (L.early)
    asm volatile("griddepcontrol.launch_dependents;");
  else
    pdl_entry();
  if (blockDim.x != kThreads || blockIdx.y >= (unsigned)T.n_pairs) {
    if (L.early) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) atomicOr(L.err, kErrLaunchShape);
    return;
  }
  const int b = blockIdx.x;
  int ri = 0;
#pragma unroll 1
  while (ri + 1 < L.n_rects && b >= L.tile_start[ri + 1]) ++ri;
  const Rect R = L.rects[ri];
  const int lay = R.log_tpr;
  const int tw = sl_tw(lay), th = sl_th(lay);
  const int t = b - L.tile_start[ri];
  const int tx0 = R.tx + (t % L.tiles_x[ri]) * tw;
  const int ty0 = R.ty + (t / L.tiles_x[ri]) * th;
  const int rx = T.rx, ry = T.ry;
  const int sw = tw + 2 * rx, sh = th + 2 * ry, sw2 = sl_sw2(lay, rx);
  const int ks = sl_skew_shift(lay), km = sl_skew_mask(lay);
  const int tid = threadIdx.x;

  const float qnan = __int_as_float(0x7fc00000);
  // Each staged value v goes to two vertical pairs: (row, row + 1).x and (row - 1, row).y.
  auto put = [&](int row, int col, float v) {
    if (!SEB_IN_BOUNDS(L.err, row >= 0 && row < sh && row < kMaxStageRows && col >= 0 && col < sw &&
                                  (row < sh - 1 ? sl_index(row, col, sw2, ks, km) : sl_index(row - 1, col, sw2, ks, km)) < L.pairs_alloc))
      return;
    if (v != v) rowflag[row] = 1;
    if (row < sh - 1) pt[sl_index(row, col, sw2, ks, km)].x = v;
    if (row > 0) pt[sl_index(row - 1, col, sw2, ks, km)].y = v;
  };
  const int dr = kThreads / sw, dc = kThreads - dr * sw;  // row-major walk in steps of kThreads cells
  if (L.tma) {
    // Tile + halo in one TMA copy into the CTA's shared memory (Algorithm 1's footprint cells
    // of every cell of the tile; outside the window the map's fill value NaN = unknown, as in
    // Sec. V-A).  The box starts at the staged tile's first column rounded down to 16 bytes and
    // lands in the scratch qs.
    constexpr int q = 16 / (int)sizeof(E);
    const int gx0 = tx0 - rx, gy0 = ty0 - ry;
    const int x0a = gx0 >= 0 ? gx0 / q * q : -((q - 1 - gx0) / q) * q;
    const int ox = gx0 - x0a, bw = stage_box_w(lay, rx, q);
    uint64_t* bar = reinterpret_cast<uint64_t*>(pt + (size_t)(sh - 1) * sw2);
    const uint32_t base = smem_addr(qs);
    const E* box = reinterpret_cast<const E*>(reinterpret_cast<char*>(qs) + (((base + 1023u) & ~1023u) - base));
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, (uint32_t)(bw * sh * (int)sizeof(E)));
      tma_load_2d(const_cast<E*>(box), &SM.map[stage_map(lay)], x0a, gy0, bar);
    }
    for (int i = tid; i < sh; i += kThreads) rowflag[i] = 0;
    const bool ok = mbar_wait_bounded(bar, 0, kStageWaitPolls);
    if (__syncthreads_or(!ok)) {
      // the copy did not land in time: report it, give the copy one more bounded wait (it
      // writes this CTA's shared memory) and leave the tile unassessed
      if (tid == 0) {
        atomicOr(L.err, kErrStageTimeout);
        mbar_wait_bounded(bar, 0, kStageWaitPolls);
      }
      __syncthreads();
      if (L.early) asm volatile("griddepcontrol.wait;" ::: "memory");
      return;
    }
    int row = tid / sw, col = tid - (tid / sw) * sw;
    while (row < sh) {
      if (SEB_IN_BOUNDS(L.err, (size_t)(row * bw + ox + col + 1) * sizeof(E) + (size_t)(reinterpret_cast<const char*>(box) -
                                                                                       reinterpret_cast<char*>(qs)) <=
                                   (size_t)kSlQ * kThreads * sizeof(float2)))
        put(row, col, stage_elev<E>(L, box[row * bw + ox + col], gx0 + col, gy0 + row));
      row += dr;
      col += dc;
      if (col >= sw) {
        col -= sw;
        ++row;
      }
    }
    __syncthreads();  // the box (in qs) is consumed
    if (tid == 0) mbar_inval(bar);
  } else {
    for (int i = tid; i < sh; i += kThreads) rowflag[i] = 0;
    __syncthreads();
    int row = tid / sw, col = tid - (tid / sw) * sw;
    while (row < sh) {
      const int gy = ty0 - ry + row, gx = tx0 - rx + col;
      float v = qnan;
      if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) v = load_elev<E>(L, gx, gy);
      put(row, col, v);
      row += dr;
      col += dc;
      if (col >= sw) {
        col -= sw;
        ++row;
      }
    }
    __syncthreads();
  }

  // block (cb, rp) of this thread: a half-warp holds 4 blocks x 4 pair rows (quad layouts) or one
  // block column x 16 block rows (column layouts; threads past W x H idle on a copy of a block)
  int cb, rp;
  bool idle = false;
  if (sl_col(lay)) {
    const int bh = sl_bh(lay), bw = sl_bw(lay);
    cb = tid / bh;
    rp = tid - cb * bh;
    if (cb >= bw) {
      cb = bw - 1;
      idle = true;
    }
  } else {
    const int c4 = (1 << lay) >> 2;
    cb = (tid & 3) + 4 * ((tid >> 4) % c4);
    rp = ((tid >> 2) & 3) + 4 * ((tid >> 4) / c4);
  }
  const int lx = 4 * cb, ly = 2 * rp;
  const int cx = tx0 + lx, cy = ty0 + ly;
  auto stores = [&](int c, int r) {
    return !idle && c >= R.x0 && c < R.x0 + R.w && r >= R.y0 && r < R.y0 + R.h;
  };
  {
    // a warp without a cell to store (outside the rectangle, or masked out) skips the work;
    // no block-wide barrier follows
    int need = 0;
    for (int h = 0; h < 2; ++h)
      for (int g = 0; g < 4; ++g)
        if (stores(cx + g, cy + h) && (!L.store_mask || L.store_mask[(int64_t)(cy + h) * L.nx + cx + g])) need = 1;
    if (!__any_sync(0xffffffffu, need)) return;
  }
  const int pair = blockIdx.y;
  const int r0 = T.run_start[pair], r1 = T.run_start[pair + 1];
  auto tile_at = [&](int row, int col) {
    return row < sh - 1 ? pt[sl_index(row, col, sw2, ks, km)].x : pt[sl_index(row - 1, col, sw2, ks, km)].y;
  };
  // block reference: first known cell of the block (rows outer), else of the footprint of
  // its first cell in run order, else 0 (then every cell of the block is unknown)
  float ref = qnan;
  for (int h = 0; h < 2 && ref != ref; ++h)
    for (int g = 0; g < 4 && ref != ref; ++g) ref = tile_at(ry + ly + h, rx + lx + g);
  if (ref != ref) {
    for (int q = r0; q < r1 && ref != ref; ++q) {
      const uint32_t pk = T.runs[q];
      const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
      for (int d = lo; d <= hi && ref != ref; ++d) ref = tile_at(ry + ly + dj, rx + lx + d);
    }
    if (ref != ref) ref = 0.f;
  }
  const float2 nref = f2(-ref, -ref), one2 = f2(1.f, 1.f), zero2 = f2(0.f, 0.f);

  // Sums over the runs: column 0 of the block (S0c = sum z', S1c = sum p z', S2c = sum dj z',
  // S3c = sum z'^2) and, for t = 1..3, the sums of what the slide from column t - 1 to column t
  // adds (D0 = z'_in - z'_out, D1 = p_in z'_in - p_out z'_out, D2 = dj D0, D3 = z'_in^2 - z'_out^2).
  // Column g is then column 0 plus the slides 1..g; its x-offsets are di = p - g.
  float2 S0c = zero2, S1c = zero2, S2c = zero2, S3c = zero2;
  float2 D0[3], D1[3], D2[3], D3[3];
  float2 K0 = zero2, K1 = zero2, K2 = zero2, K3 = zero2;  // compensations (COMP)
  float2 E0[3], E1[3], E2[3], E3[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) D0[t] = D1[t] = D2[t] = D3[t] = E0[t] = E1[t] = E2[t] = E3[t] = zero2;
  // Integer moments of the missing points of the 8 cells, Qp[k][g] for column g: k = 0..5 ->
  // (n, sum di, sum dj, sum di^2, sum di dj, sum dj^2).  Both rows of a column share one int32,
  // row 0 + 65536 x row 1 (two's complement): sums of such words are exact as long as every
  // field stays within [-32768, 32767].  Each field is a moment of a subset of the footprint, so
  // it is bounded by (points summed) x reach^2; when a whole footprint can exceed the range, the
  // words are unpacked into int32 sums in the (then free) box scratch every L.q_flush runs.
  int Qp[kSlQ];
#pragma unroll
  for (int i = 0; i < kSlQ; ++i) Qp[i] = 0;
  int* qsi = reinterpret_cast<int*>(qs);  // [2 kSlQ][kThreads] int32 sums, or [kSlQ][kThreads] words
  bool qflushed = false;
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < kSlQ; ++i) {
      const int w = Qp[i], a = (w << 16) >> 16, b = (w - a) >> 16;  // row 0: the sign-extended low half
      qsi[(2 * i) * kThreads + tid] = (qflushed ? qsi[(2 * i) * kThreads + tid] : 0) + a;
      qsi[(2 * i + 1) * kThreads + tid] = (qflushed ? qsi[(2 * i + 1) * kThreads + tid] : 0) + b;
      Qp[i] = 0;
    }
    qflushed = true;
  };

  // the runs in chunks of L.q_flush (all of them when 0); the packed words are flushed between
  // chunks (the same runs in every thread of the CTA)
  const int chunk = L.q_flush > 0 ? L.q_flush : (r1 > r0 ? r1 - r0 : 1);
  for (int q0 = r0; q0 < r1; q0 += chunk) {
  if (q0 > r0) flush();
  const int q1 = q0 + chunk < r1 ? q0 + chunk : r1;
  for (int q = q0; q < q1; ++q) {
    const uint32_t pk = T.runs[q];
    const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
    const int row = ry + ly + dj;
    // The masked path gives bit-identical sums for runs without unknown cells, so the choice is
    // free: band tiles of a rolling shift touch the window edge, where nearly every run holds an
    // unknown cell, and there the per-run vote costs more than it saves.
    const bool masked = L.all_masked || __any_sync(0xffffffffu, rowflag[row] | rowflag[row + 1]);
    const float2* pq = pt + sl_index(row, rx + lx + lo, sw2, ks, km);  // pq[k]: column lo + k of the block
    const int len = hi - lo + 1;
    if (!SEB_IN_BOUNDS(L.err, row >= 0 && row + 1 < sh && rx + lx + lo >= 0 && rx + lx + hi + 3 < sw &&
                                  sl_index(row, rx + lx + hi + 3, sw2, ks, km) < L.pairs_alloc))
      continue;
    const float flo = (float)lo, fhi = (float)hi;
    const float2 dj2 = f2((float)dj, (float)dj);
    auto slide = [&](int t, float2 zo, float2 zi) {
      const float po = flo + (float)t, pi = fhi + (float)(t + 1);
      const float2 d = add2(zi, neg2(zo));
      if (COMP) {
        kadd2(D0[t], E0[t], d);
        kadd2(D2[t], E2[t], __fmul2_rn(dj2, d));
        kadd2(D1[t], E1[t], fma2(f2(pi, pi), zi, __fmul2_rn(f2(-po, -po), zo)));
        kadd2(D3[t], E3[t], fma2(zi, zi, __fmul2_rn(neg2(zo), zo)));
      } else {
        D0[t] = add2(D0[t], d);
        D2[t] = fma2(dj2, d, D2[t]);
        D1[t] = fma2(f2(pi, pi), zi, fma2(f2(-po, -po), zo, D1[t]));
        D3[t] = fma2(zi, zi, fma2(neg2(zo), zo, D3[t]));
      }
    };
    auto column0 = [&](float2 Ab, float2 Bx, float2 Cb) {
      if (COMP) {
        kadd2(S0c, K0, Ab);
        kadd2(S1c, K1, Bx);
        kadd2(S2c, K2, __fmul2_rn(dj2, Ab));
        kadd2(S3c, K3, Cb);
      } else {
        S0c = add2(S0c, Ab);
        S1c = add2(S1c, Bx);
        S2c = fma2(dj2, Ab, S2c);
        S3c = add2(S3c, Cb);
      }
    };
    // Column 0 of the block: A = sum z', C = sum z'^2 and Tb = sum of the running sums of z'
    // = sum (len - k) z'_k, so that sum p z' = (hi + 1) A - Tb with p = lo + k.
    const float h1 = fhi + 1.f;
    const float2 H2 = f2(h1, h1);
    if (!masked) {
      float2 Ab = zero2, Tb = zero2, Cb = zero2;
#pragma unroll 4
      for (int k = 0; k < len; ++k) {
        const float2 zp = add2(pq[k], nref);
        Ab = add2(Ab, zp);
        Tb = add2(Tb, Ab);
        Cb = fma2(zp, zp, Cb);
      }
      column0(Ab, fma2(H2, Ab, neg2(Tb)), Cb);
#pragma unroll
      for (int t = 0; t < 3; ++t) slide(t, add2(pq[t], nref), add2(pq[len + t], nref));
    } else {
      // unknown heights: z' = 0 (the known ones get exactly the plain path's z - ref); the packed
      // word u = [x unknown] + 65536 [y unknown] counts them for both rows at once.  The NaN tests
      // give all-ones / zero masks, so z' and the counts are bitwise ANDs, not selects.
      constexpr int kP = 0x10001;
      auto zof = [&](int k, float2& zp, int& u) {
        const float2 v = pq[k];
        const uint32_t mx = 0u - (uint32_t)(v.x == v.x), my = 0u - (uint32_t)(v.y == v.y);
        const float2 zr = add2(v, nref);
        zp = f2(__uint_as_float(__float_as_uint(zr.x) & mx), __uint_as_float(__float_as_uint(zr.y) & my));
        u = (int)((~mx & 1u) | (~my & 0x10000u));
      };
      // Known weights summed three times over (k1 = sum m, k2 = sum (len - k) m_k,
      // k3 = sum (len - k)(len - k + 1) / 2 m_k, packed like Qp); with u = len - k the missing
      // moments are X1 = len - k1, X2 = sum u x = len (len + 1) / 2 - k2,
      // X3 = len (len + 1)(len + 2) / 6 - k3, and p = hi + 1 - u gives qx = (hi + 1) X1 - X2,
      // qxx = (hi + 1)^2 X1 - 2 (hi + 1) X2 + 2 X3 - X2.
      float2 Ab = zero2, Tb = zero2, Cb = zero2;
      int k1 = 0, k2 = 0, k3 = 0;
#pragma unroll 4
      for (int k = 0; k < len; ++k) {
        const float2 v = pq[k];
        const uint32_t mx = 0u - (uint32_t)(v.x == v.x), my = 0u - (uint32_t)(v.y == v.y);
        const float2 zr = add2(v, nref);
        const float2 zp = f2(__uint_as_float(__float_as_uint(zr.x) & mx), __uint_as_float(__float_as_uint(zr.y) & my));
        Ab = add2(Ab, zp);
        Tb = add2(Tb, Ab);
        Cb = fma2(zp, zp, Cb);
        k1 += (int)((mx & 1u) | (my & 0x10000u));
        k2 += k1;
        k3 += k2;
      }
      column0(Ab, fma2(H2, Ab, neg2(Tb)), Cb);
      const int H = hi + 1;
      const int X1 = len * kP - k1, X2 = (len * (len + 1) / 2) * kP - k2,
                X3 = (len * (len + 1) * (len + 2) / 6) * kP - k3;
      int qn = X1;
      int qx = H * X1 - X2;
      int qxx = H * H * X1 - 2 * H * X2 + 2 * X3 - X2;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (g > 0) {
          float2 zo, zi;
          int xo, xi;
          zof(g - 1, zo, xo);
          zof(len - 1 + g, zi, xi);
          slide(g - 1, zo, zi);
          const int po = lo + g - 1, pi = hi + g;
          qn += xi - xo;
          qx += pi * xi - po * xo;
          qxx += pi * pi * xi - po * po * xo;
        }
        // missing-point moments of column g in its own offsets di = p - g
        const int sdi = qx - g * qn;
        const int sdi2 = qxx - 2 * g * qx + g * g * qn;
        Qp[0 * 4 + g] += qn;
        Qp[1 * 4 + g] += sdi;
        Qp[2 * 4 + g] += dj * qn;
        Qp[3 * 4 + g] += sdi2;
        Qp[4 * 4 + g] += dj * sdi;
        Qp[5 * 4 + g] += dj * dj * qn;
      }
    }
  }
  }
  if (COMP) {  // fold the compensations in: the exact sum is s - c
    S0c = add2(S0c, neg2(K0));
    S1c = add2(S1c, neg2(K1));
    S2c = add2(S2c, neg2(K2));
    S3c = add2(S3c, neg2(K3));
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      D0[t] = add2(D0[t], neg2(E0[t]));
      D1[t] = add2(D1[t], neg2(E1[t]));
      D2[t] = add2(D2[t], neg2(E2[t]));
      D3[t] = add2(D3[t], neg2(E3[t]));
    }
  }
  float2 S0[4], S1[4], S2[4], S3[4];
  {
    float2 a = S0c, bx = S1c, c2 = S2c, c3 = S3c;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g > 0) {
        a = add2(a, D0[g - 1]);
        bx = add2(bx, D1[g - 1]);
        c2 = add2(c2, D2[g - 1]);
        c3 = add2(c3, D3[g - 1]);
      }
      S0[g] = a;
      S1[g] = fma2(f2(-(float)g, -(float)g), a, bx);
      S2[g] = c2;
      S3[g] = c3;
    }
  }

  // the missing-point moments wait for the finish in the (now free) box scratch, out of registers
  if (qflushed) {
    flush();
  } else {
#pragma unroll
    for (int i = 0; i < kSlQ; ++i) qsi[i * kThreads + tid] = Qp[i];
  }

  if (L.early) asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous launch's stores first
  const int k0 = pair, k1 = pair + T.n_pairs;
  const float ct = T.cos_t[pair], st = T.sin_t[pair];
  const int64_t chs = (int64_t)L.n_yaw * L.plane;
  const int* mom = T.mom[pair];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = cy + h;
    int pr = r + L.ring_y;
    if (pr >= L.ny) pr -= L.ny;
    Cell o[4];
    bool keep[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int c = cx + g;
      keep[g] = stores(c, r) && (!L.store_mask || L.store_mask[(int64_t)r * L.nx + c]);
      if (!keep[g]) continue;
      int qv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (qflushed) {
          qv[k] = qsi[(2 * (k * 4 + g) + h) * kThreads + tid];
        } else {
          const int w = qsi[(k * 4 + g) * kThreads + tid], a = (w << 16) >> 16;  // row 0: the low half
          qv[k] = h ? (w - a) >> 16 : a;
        }
      }
      o[g] = finish_cell(mom[0] - qv[0], mom[1] - qv[1], mom[2] - qv[2], mom[3] - qv[3],
                         mom[4] - qv[4], mom[5] - qv[5], h ? S0[g].y : S0[g].x, h ? S1[g].y : S1[g].x,
                         h ? S2[g].y : S2[g].x, h ? S3[g].y : S3[g].x, ref, T.n_min[pair], ct, st, L, mom[0],
                         T.inv_n[pair]);
    }
    int pc = cx + L.ring_x;
    if (pc >= L.nx) pc -= L.nx;
    float* out = L.out;
    if (L.vec4 && keep[0] && keep[1] && keep[2] && keep[3] && (pc & 3) == 0) {
      // the block's 4 cells are 4 consecutive, 16-byte aligned physical cells (nx % 4 == 0,
      // so no ring wrap falls inside it): one 16-byte store per channel and plane
      const int64_t i0 = (int64_t)k0 * L.plane + (int64_t)pr * L.nx + pc;
      const int64_t i1 = (int64_t)k1 * L.plane + (int64_t)pr * L.nx + pc;
      if (!SEB_IN_BOUNDS(L.err, pr >= 0 && pr < L.ny && pc >= 0 && pc + 3 < L.nx && i1 + 3 < chs)) continue;
      auto st4 = [&](int64_t i, float a, float b, float c, float d) {
        *reinterpret_cast<float4*>(out + i) = make_float4(a, b, c, d);
      };
      st4(i0, o[0].z, o[1].z, o[2].z, o[3].z);
      st4(i1, o[0].z, o[1].z, o[2].z, o[3].z);
      st4(chs + i0, o[0].pitch, o[1].pitch, o[2].pitch, o[3].pitch);
      st4(chs + i1, -o[0].pitch, -o[1].pitch, -o[2].pitch, -o[3].pitch);
      st4(2 * chs + i0, o[0].roll, o[1].roll, o[2].roll, o[3].roll);
      st4(2 * chs + i1, -o[0].roll, -o[1].roll, -o[2].roll, -o[3].roll);
      st4(3 * chs + i0, o[0].rough, o[1].rough, o[2].rough, o[3].rough);
      st4(3 * chs + i1, o[0].rough, o[1].rough, o[2].rough, o[3].rough);
      st4(4 * chs + i0, o[0].risk, o[1].risk, o[2].risk, o[3].risk);
      st4(4 * chs + i1, o[0].risk, o[1].risk, o[2].risk, o[3].risk);
      const uint32_t fw = (o[0].flags & 0xffu) | ((o[1].flags & 0xffu) << 8) | ((o[2].flags & 0xffu) << 16) |
                          ((o[3].flags & 0xffu) << 24);  // little-endian: byte g is cell g
      *reinterpret_cast<uint32_t*>(L.flags + i0) = fw;
      *reinterpret_cast<uint32_t*>(L.flags + i1) = fw;
      continue;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (!keep[g]) continue;
      int pcg = pc + g;
      if (pcg >= L.nx) pcg -= L.nx;
      const int64_t i0 = (int64_t)k0 * L.plane + (int64_t)pr * L.nx + pcg;
      const int64_t i1 = (int64_t)k1 * L.plane + (int64_t)pr * L.nx + pcg;
      if (!SEB_IN_BOUNDS(L.err, pr >= 0 && pr < L.ny && pcg >= 0 && pcg < L.nx && i1 < chs)) continue;
      out[i0] = o[g].z;
      out[i1] = o[g].z;
      out[chs + i0] = o[g].pitch;
      out[chs + i1] = -o[g].pitch;
      out[2 * chs + i0] = o[g].roll;
      out[2 * chs + i1] = -o[g].roll;
      out[3 * chs + i0] = o[g].rough;
      out[3 * chs + i1] = o[g].rough;
      out[4 * chs + i0] = o[g].risk;
      out[4 * chs + i1] = o[g].risk;
      L.flags[i0] = (uint8_t)o[g].flags;
      L.flags[i1] = (uint8_t)o[g].flags;
    }
  }
}

__global__ void copy_out_kernel(const Launch L, float* __restrict__ dst, uint8_t* __restrict__ fdst) {
  seb::pdl_entry();
  const int64_t total = (int64_t)L.n_yaw * L.plane;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / L.plane;
    const int64_t rem = i - k * L.plane;
    const int r = (int)(rem / L.nx), c = (int)(rem - (int64_t)r * L.nx);
    int pr = r + L.ring_y, pc = c + L.ring_x;
    if (pr >= L.ny) pr -= L.ny;
    if (pc >= L.nx) pc -= L.nx;
    const int64_t src = k * L.plane + (int64_t)pr * L.nx + pc;
    if (dst)
      for (int ch = 0; ch < SEB_N_CH; ++ch) dst[ch * total + i] = L.out[ch * total + src];
    if (fdst) fdst[i] = L.flags[src];
  }
}

// Tiling of the requested rectangles for assess_kernel (v2 layouts, tiles start at the
// rectangle's corner).
// Both tilings return false if the rectangles would not fit Launch::rects (not reached with the
// at most 4 requested rectangles and 3 rectangles per request; checked all the same).
bool decompose_v2(Launch& L) {
  L.n_rects = 0;
  L.tile_start[0] = 0;
  bool fits = true;
  auto push = [&](int x0, int y0, int w, int h, int lg) {
    if (w <= 0 || h <= 0) return;
    if (L.n_rects >= kMaxRects) {
      fits = false;
      return;
    }
    const int i = L.n_rects++;
    L.rects[i] = Rect{x0, y0, w, h, x0, y0, lg};
    const int tw = kG << lg, th = kThreads >> lg;
    L.tiles_x[i] = (w + tw - 1) / tw;
    L.tile_start[i + 1] = L.tile_start[i] + L.tiles_x[i] * ((h + th - 1) / th);
  };
  for (int k = 0; k < L.n_req; ++k) {
    const Rect q = L.req[k];
    const int wm = q.w >= 32 ? q.w - q.w % 32 : 0, hm = q.h >= 32 ? q.h - q.h % 32 : 0;
    if (wm && hm) {
      push(q.x0, q.y0, wm, hm, 3);
      push(q.x0 + wm, q.y0, q.w - wm, q.h, 1);
      push(q.x0, q.y0 + hm, wm, q.h - hm, 5);
    } else if (q.w < q.h) {
      push(q.x0, q.y0, q.w, q.h, 1);
    } else {
      push(q.x0, q.y0, q.w, q.h, 5);
    }
  }
  return fits;
}

// Tiling for assess_kernel_sl: tile grids start on globally aligned blocks (column = 0 mod 4,
// row = 0 mod 2 in global cells), so a rectangle's grid may start up to 3 columns / 1 row
// before it; those cells are computed but not stored.
bool decompose_sl(Launch& L) {
  L.n_rects = 0;
  L.tile_start[0] = 0;
  bool fits = true;
  auto push = [&](int tx, int ty, int sx0, int sy0, int sx1, int sy1, int lay) {
    if (sx1 <= sx0 || sy1 <= sy0) return;
    if (L.n_rects >= kMaxRects) {
      fits = false;
      return;
    }
    const int i = L.n_rects++;
    L.rects[i] = Rect{sx0, sy0, sx1 - sx0, sy1 - sy0, tx, ty, lay};
    const int tw = sl_tw(lay), th = sl_th(lay);
    L.tiles_x[i] = (sx1 - tx + tw - 1) / tw;
    L.tile_start[i + 1] = L.tile_start[i] + L.tiles_x[i] * ((sy1 - ty + th - 1) / th);
  };
  for (int k = 0; k < L.n_req; ++k) {
    const Rect q = L.req[k];
    const int ax = q.x0 - (((q.x0 + L.phase_x) % 4) + 4) % 4;
    const int ay = q.y0 - (((q.y0 + L.phase_y) % 2) + 2) % 2;
    const int x1 = q.x0 + q.w, y1 = q.y0 + q.h;
    const int W = x1 - ax, H = y1 - ay;
    if (W >= 32 && H >= 64) {
      const int Wm = W - W % 32, Hm = H - H % 64;
      push(ax, ay, q.x0, q.y0, ax + Wm, ay + Hm, 3);
      push(ax + Wm, ay, ax + Wm, q.y0, x1, y1, 2);
      push(ax, ay + Hm, q.x0, ay + Hm, ax + Wm, y1, 5);
    } else if (W < H) {
      // a column band: tiles exactly as wide as the band where it is 3 or 5 blocks wide (a band
      // of up to 8 blocks is cut into at most two such pieces and 4-block ones), layout 2
      // otherwise (at most 3 rectangles per requested one, so kMaxRects holds 4 of them)
      int nb = (W + 3) / 4, x = ax;
      if (nb > 8) {
        push(ax, ay, q.x0, q.y0, x1, y1, 2);
        nb = 0;
      }
      while (nb > 0) {
        const int t = nb <= 5 ? nb : (nb - 3 < 5 ? nb - 3 : 5);
        const int lay = t == 3 ? kColLay + 3 : (t == 5 ? kColLay + 5 : 2);
        const int xe = x + 4 * t < x1 ? x + 4 * t : x1;
        push(x, ay, x > q.x0 ? x : q.x0, q.y0, xe, y1, lay);
        x += 4 * t;
        nb -= t;
      }
    } else {
      push(ax, ay, q.x0, q.y0, x1, y1, 5);
    }
  }
  return fits;
}

size_t pairs_sl(const Tables& T, const Launch& L) {
  size_t pairs = 0;
  for (int i = 0; i < L.n_rects; ++i) {
    const int lay = L.rects[i].log_tpr;
    const size_t s = (size_t)(sl_th(lay) + 2 * T.ry - 1) * sl_sw2(lay, T.rx);
    pairs = s > pairs ? s : pairs;
  }
  return pairs;
}

size_t smem_sl(const Tables& T, const Launch& L) {
  size_t pairs = 0;
  for (int i = 0; i < L.n_rects; ++i) {
    const int lay = L.rects[i].log_tpr;
    const size_t s = (size_t)(sl_th(lay) + 2 * T.ry - 1) * sl_sw2(lay, T.rx);
    pairs = s > pairs ? s : pairs;
  }
  return kMaxStageRows * sizeof(float) + ((size_t)kSlQ * kThreads + pairs) * sizeof(float2) + 16;  // + mbarrier
}

}  // namespace

// Driver entry point of cuTensorMapEncodeTiled (no link against libcuda), looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

namespace {

// Tensor maps for the TMA staging of every layout in the launch; false (plain loads) when the
// elevation's rows are not 16-byte multiples, a box exceeds 256 elements per side or the moment
// scratch it lands in, or the driver has no encoder.
template <typename E>
bool stage_maps(const Tables& T, const Launch& L, StageMaps* M) {
  constexpr int es = (int)sizeof(E), q = 16 / es;
  if (((size_t)L.nx * es) % 16 != 0 || ((uintptr_t)L.elev % 16) != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                         : (sizeof(E) == 2 && std::is_same<E, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  memset(M, 0, sizeof(*M));
  bool used[kStageMaps] = {false, false, false, false, false};
  for (int i = 0; i < L.n_rects; ++i) used[stage_map(L.rects[i].log_tpr)] = true;
  const int lays[kStageMaps] = {2, 3, 5, kColLay + 3, kColLay + 5};
  for (int m = 0; m < kStageMaps; ++m) {
    if (!used[m]) continue;
    const int lay = lays[m];
    const int bw = stage_box_w(lay, T.rx, q), bh = sl_th(lay) + 2 * T.ry;
    if (bw > 256 || bh > 256 || (size_t)bw * bh * es + 1024 > (size_t)kSlQ * kThreads * sizeof(float2)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny};
    const cuuint64_t strides[1] = {(cuuint64_t)L.nx * es};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&M->map[m], dt, 2, const_cast<void*>(L.elev), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// The sliding kernel packs the missing-point moments of a block's two rows into one int32 per
// moment.  Every field is a moment (n, sums of di, dj, di^2, di dj, dj^2) of a subset of one
// footprint, so |field| <= points x reach^2.  Returns the runs after which the packed words must
// be flushed (0: a whole footprint fits int16, never), or -1 when not even one run fits.
int packed_moment_flush(const Tables& T) {
  const long long r = T.rx > T.ry ? T.rx : T.ry, w = r * r > 1 ? r * r : 1;
  long long n_max = 0;
  for (int p = 0; p < T.n_pairs; ++p) n_max = T.mom[p][0] > n_max ? T.mom[p][0] : n_max;
  if (n_max * w <= 32767) return 0;
  const long long per_run = (2 * T.rx + 1) * w;  // a run holds at most 2 rx + 1 points
  return per_run <= 32767 ? (int)(32767 / per_run) : -1;
}

template <typename E, bool COMP>
cudaError_t launch_typed(const Tables& T, const Launch& Lreq, cudaStream_t stream) {
  Launch L = Lreq;
  {
    if (!decompose_sl(L)) return cudaErrorInvalidValue;
    // 16-byte stores of whole cell blocks need 4 | nx (no ring wrap inside a block) and
    // aligned output planes
    L.vec4 = (L.nx % 4 == 0) && ((uintptr_t)L.out % 16 == 0) && ((uintptr_t)L.flags % 4 == 0);
    const size_t smem = smem_sl(T, L);
    L.pairs_alloc = (int32_t)pairs_sl(T, L);
    L.q_flush = packed_moment_flush(T);
    if (smem <= 227 * 1024 && L.q_flush >= 0) {
      if (L.tile_start[L.n_rects] == 0) return cudaSuccess;
      StageMaps M;
      L.tma = stage_maps<E>(T, L, &M) ? 1 : 0;
      if (!L.tma) memset(&M, 0, sizeof(M));
      auto kern = assess_kernel_sl<E, COMP>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      return launch_pdl(kern, dim3(L.tile_start[L.n_rects], T.n_pairs), dim3(kThreads), smem, stream, T, L, M);
    }
    // very large footprints: the per-cell kernel below
  }
  if (!decompose_v2(L)) return cudaErrorInvalidValue;
  if (L.tile_start[L.n_rects] == 0) return cudaSuccess;
  size_t smem = 0;
  for (int i = 0; i < L.n_rects; ++i) {
    const size_t s = (size_t)stage_w(L.rects[i].log_tpr, T.rx) * stage_h(L.rects[i].log_tpr, T.ry);
    smem = s > smem ? s : smem;
  }
  smem = (smem + kMaxStageRows) * sizeof(float);
  auto kern = assess_kernel<E, COMP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(L.tile_start[L.n_rects], T.n_pairs);
  kern<<<grid, kThreads, smem, stream>>>(T, L);
  return cudaGetLastError();
}

}  // namespace


cudaError_t launch_assess(const Tables& T, const Launch& L, int elev_dtype, int precision,
                          cudaStream_t stream) {
  if (L.n_req == 0) return cudaSuccess;
  const bool comp = precision == SEB_COMPENSATED;
  switch (elev_dtype) {
    case SEB_F32:
      return comp ? launch_typed<float, true>(T, L, stream) : launch_typed<float, false>(T, L, stream);
    case SEB_BF16:
      return comp ? launch_typed<__nv_bfloat16, true>(T, L, stream)
                  : launch_typed<__nv_bfloat16, false>(T, L, stream);
    case SEB_BF16_TILED:
      return comp ? launch_typed<Bf16Tiled, true>(T, L, stream) : launch_typed<Bf16Tiled, false>(T, L, stream);
    default:
      return comp ? launch_typed<__half, true>(T, L, stream) : launch_typed<__half, false>(T, L, stream);
  }
}

// SEB_BF16_TILED encoding: one CTA per 16 x 16 world-aligned tile of the window.
__global__ void encode_tiled_kernel(const float* __restrict__ elev, int nx, int ny, int px, int py, int tx_n,
                                    __nv_bfloat16* __restrict__ delta, float* __restrict__ base) {
  __shared__ float lo[256], hi[256];
  seb::pdl_entry();
  const int tx = blockIdx.x, ty = blockIdx.y, t = threadIdx.x;
  const int c = tx * kBaseTile - px + (t & 15), r = ty * kBaseTile - py + (t >> 4);
  const bool in = c >= 0 && c < nx && r >= 0 && r < ny;
  const float z = in ? elev[(int64_t)r * nx + c] : __int_as_float(0x7fc00000);
  const bool known = z == z;
  lo[t] = known ? z : INFINITY;
  hi[t] = known ? z : -INFINITY;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) {
      lo[t] = fminf(lo[t], lo[t + s]);
      hi[t] = fmaxf(hi[t], hi[t + s]);
    }
    __syncthreads();
  }
  const float b = lo[0] <= hi[0] ? 0.5f * lo[0] + 0.5f * hi[0] : 0.f;
  if (t == 0) base[ty * tx_n + tx] = b;
  if (in) delta[(int64_t)r * nx + c] = __float2bfloat16_rn(z - b);
}

cudaError_t launch_copy_out(const Launch& L, float* out_dev, uint8_t* flags_dev, cudaStream_t stream) {
  const int64_t total = (int64_t)L.n_yaw * L.plane;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  return launch_pdl(copy_out_kernel, dim3(blocks), dim3(256), 0, stream, L, out_dev, flags_dev);
}

}  // namespace seb

extern "C" int seb_encode_bf16_tiled(const float* elev, int32_t nx, int32_t ny, int64_t oi, int64_t oj, void* out,
                                     seb_stream_t stream) {
  SEB_RANGE();
  if (!elev || !out || nx < 1 || ny < 1 || ((uintptr_t)out & 255)) {
    seb::set_error("seb_encode_bf16_tiled: NULL pointer, empty window or output not 256-byte aligned");
    return SEB_ERR_INVALID_ARG;
  }
  if ((int64_t)nx * ny > (int64_t)1 << 31) {
    seb::set_error("seb_encode_bf16_tiled: window too large");
    return SEB_ERR_BAD_SHAPE;
  }
  const int px = (int)(((oi % seb::kBaseTile) + seb::kBaseTile) % seb::kBaseTile);
  const int py = (int)(((oj % seb::kBaseTile) + seb::kBaseTile) % seb::kBaseTile);
  const int txn = seb::tiled_tx(nx), tyn = seb::tiled_tx(ny);
  auto* delta = static_cast<__nv_bfloat16*>(out);
  auto* base = reinterpret_cast<float*>(static_cast<uint8_t*>(out) + seb::tiled_base_offset(nx, ny));
  const cudaError_t e = seb::launch_pdl(seb::encode_tiled_kernel, dim3(txn, tyn), dim3(256), 0, (cudaStream_t)stream,
                                        elev, (int)nx, (int)ny, px, py, txn, delta, base);
  if (e != cudaSuccess) {
    seb::set_error("seb_encode_bf16_tiled launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
