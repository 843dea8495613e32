// SE(2)-grid traversability assessment kernel (Algorithm 1 of Sec. V-B for every cell and
// yaw bin), plus the ring-unrolling copy.
//
// One CTA = one 32 x 32 tile of cells x one yaw pair {k, k + K/2} (the two bins share a
// footprint, so their moments, normal and roughness are computed once; pitch and roll
// change sign).  The tile and its footprint halo are staged in shared memory as FP32
// (cells outside the window read as NaN = unknown, Sec. V-A).  Each thread owns 4
// adjacent cells of one row and walks the yaw's row runs with a 4-wide register window,
// so one shared-memory load feeds 4 cells.
//
// Moments are accumulated about a per-cell reference height (the cell's own elevation,
// or the first known footprint cell in run order when the centre is unknown):
//   S0 = sum z', S1 = sum di z', S2 = sum dj z', S3 = sum z'^2,  z' = z - ref,
// with dj folded per run.  The xy moments (N, sum di, ..., sum dj^2) are exact integers:
// the table's when the tile has no unknown cell, else summed from the known mask.  Every
// cell's arithmetic therefore depends on its neighbourhood only, never on the tile
// position, which makes the rolling update bit-identical to a full rebuild.
//
// Covariance (population, /N, Algorithm 1) from the moments; smallest eigenpair by the
// trigonometric closed form for symmetric 3x3 matrices (O. K. Smith, "Eigenvalues of a
// symmetric 3 x 3 matrix", CACM 4(4), 1961), eigenvector as the largest cross product of
// two rows of Cov - lambda_min I, roughness from the Rayleigh quotient n^T Cov n.  A
// relative eigen-gap below gap_fp64 redoes the eigen-solve in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "seb_device.cuh"
#include "seb_internal.h"

namespace seb {
namespace {

// Algorithm 1 from the moments on: covariance, normal, roughness, frame (Eqs. 2-3),
// pitch/roll at heading (ct, st), fitted-plane height at the cell centre, risk.
__device__ __noinline__ Cell finish_cell(int N, int MX, int MY, int MXX, int MXY, int MYY, float S0,
                                         float S1, float S2, float S3, float ref, int n_min,
                                         float ct, float st, const Launch& L) {
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
  const float inv_n2 = 1.f / (fN * fN);
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
  float c[6];
  c[0] = nxx * inv_n2 * res * res;
  c[1] = nxy * inv_n2 * res * res;
  c[3] = nyy * inv_n2 * res * res;
  c[2] = fmaf(S1, fN, -fMX * S0) * inv_n2 * res;
  c[4] = fmaf(S2, fN, -fMY * S0) * inv_n2 * res;
  c[5] = fmaf(S3, fN, -S0 * S0) * inv_n2;
  float n[3], gap;
  min_eigpair<float>(c, n, &gap);
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
    o.rough = refine_min<float>(c, n) / tr;
  }
  // Body frame (Eqs. 2-3): u = z_b x x_yaw = (-n_z s, n_z c, n_x s - n_y c),
  // y_b = u / |u|, x_b = y_b x z_b, so b3^T x_b = -n_z (n_x c + n_y s) / |u|.
  const float uz = n[0] * st - n[1] * ct;
  const float un = sqrtf(n[2] * n[2] + uz * uz);
  if (!(n[2] > 1e-6f) || !(un >= 1e-6f)) flags |= SEB_FLAG_DEGENERATE;
  if (flags & SEB_FLAG_DEGENERATE) {
    o.z = o.pitch = o.roll = qnan;
    o.risk = 1.f;
    o.flags = flags | SEB_FLAG_OBSTACLE;
    atomicAdd(&L.counters[1], 1ull);
    return o;
  }
  const float ybz = fminf(fmaxf(uz / un, -1.f), 1.f);
  const float xbz = fminf(fmaxf(-n[2] * (n[0] * ct + n[1] * st) / un, -1.f), 1.f);
  o.pitch = asinf(xbz);
  o.roll = asinf(ybz);
  // Plane through the mean with normal n, evaluated at the cell centre (offset 0).
  const float mz = S0 / fN;
  o.z = ref + mz + (n[0] * (fMX / fN) + n[1] * (fMY / fN)) * res / n[2];
  const float ap = fabsf(o.pitch), ar = fabsf(o.roll);
  if (o.rough > L.kappa_max || ap > L.phi_x_max || ar > L.phi_y_max) {
    o.risk = 1.f;
    flags |= SEB_FLAG_OBSTACLE;
  } else {
    o.risk = L.w0 * (o.rough / L.kappa_max) + L.w1 * (ap / L.phi_x_max) + L.w2 * (ar / L.phi_y_max);
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
  const int tx0 = R.x0 + (t % L.tiles_x[ri]) * tw;
  const int ty0 = R.y0 + (t / L.tiles_x[ri]) * th;
  const int rx = T.rx, ry = T.ry;
  const int sw = stage_w(lg, rx), sh = stage_h(lg, ry);

  for (int i = threadIdx.x; i < sh; i += kThreads) rowflag[i] = 0;
  __syncthreads();
  // Stage tile + halo (outside the window = NaN = unknown).
  const E* __restrict__ elev = static_cast<const E*>(L.elev);
  const float qnan = __int_as_float(0x7fc00000);
  for (int idx = threadIdx.x; idx < sw * sh; idx += kThreads) {
    const int row = idx / sw, col = idx - row * sw;
    const int gy = ty0 - ry + row, gx = tx0 - rx + col;
    float v = qnan;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) v = to_f32<E>(elev[(int64_t)gy * L.nx + gx]);
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
// Plain-precision kernel on packed FP32 pairs.  Each thread owns a 2 x 2 block of cells; the
// staged tile is stored as vertical pairs (T[r][c], T[r+1][c]) so that one 8-byte shared load
// feeds both rows of a column, and the moment updates run as FP32x2 instructions
// (__fadd2_rn / __ffma2_rn round each half exactly like the scalar forms).  Every cell performs
// the same operations in the same order as assess_kernel, so the results are bit-identical.
// Alternate pair rows are skewed by one element, which keeps a half-warp (8 column pairs x 2
// pair rows) on 32 distinct banks.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ int pair_index(int r, int c, int sw2) { return r * sw2 + c + ((r >> 1) & 1); }

#ifndef SEB_ASSESS_MIN_BLOCKS
#define SEB_ASSESS_MIN_BLOCKS 2  // CTAs per SM the register budget is sized for
#endif
template <typename E>
__global__ void __launch_bounds__(kThreads, SEB_ASSESS_MIN_BLOCKS)
    assess_kernel_x2(const __grid_constant__ Tables T, const __grid_constant__ Launch L) {
  extern __shared__ float smem[];
  int* rowflag = reinterpret_cast<int*>(smem);
  float2* pt = reinterpret_cast<float2*>(smem + kMaxStageRows);  // [sh - 1][sw2] vertical pairs of heights
  // (unknown -> 0), then the matching pairs of known weights, then per-thread missing moments
  float2* pm = pt + (size_t)(kThreads >> 1) * 0;  // placeholder, set below once sh, sw2 are known
  if (blockDim.x != kThreads || blockIdx.y >= (unsigned)T.n_pairs) {
    if (threadIdx.x == 0) atomicOr(L.err, kErrLaunchShape);
    return;
  }
  const int b = blockIdx.x;
  if (L.tile_active && !L.tile_active[b]) return;  // uniform per CTA, before any barrier
  int ri = 0;
#pragma unroll 1
  while (ri + 1 < L.n_rects && b >= L.tile_start[ri + 1]) ++ri;
  const Rect R = L.rects[ri];
  const int lg = R.log_tpr;
  const int tw = kG << lg, th = kThreads >> lg;
  const int t = b - L.tile_start[ri];
  const int tx0 = R.x0 + (t % L.tiles_x[ri]) * tw;
  const int ty0 = R.y0 + (t / L.tiles_x[ri]) * th;
  const int rx = T.rx, ry = T.ry;
  const int sw = tw + 2 * rx, sh = th + 2 * ry;
  const int sw2 = sw + 1;

  const int npair = (sh - 1) * sw2;
  pm = pt + npair;
  float2* qs = pm + npair;  // [6][kThreads] float2 per column of the thread: [g][k][tid]
  for (int i = threadIdx.x; i < sh; i += kThreads) rowflag[i] = 0;
  for (int i = threadIdx.x; i < 12 * kThreads; i += kThreads) qs[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const E* __restrict__ elev = static_cast<const E*>(L.elev);
  for (int idx = threadIdx.x; idx < sw * sh; idx += kThreads) {
    const int row = idx / sw, col = idx - row * sw;
    const int gy = ty0 - ry + row, gx = tx0 - rx + col;
    float v = 0.f, m = 0.f;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
      const float e = to_f32<E>(elev[(int64_t)gy * L.nx + gx]);
      if (e == e) {
        v = e;
        m = 1.f;
      }
    }
    if (m == 0.f) rowflag[row] = 1;
    if (row < sh - 1) {
      const int k = pair_index(row, col, sw2);
      pt[k].x = v;
      pm[k].x = m;
    }
    if (row > 0) {
      const int k = pair_index(row - 1, col, sw2);
      pt[k].y = v;
      pm[k].y = m;
    }
  }
  __syncthreads();

  // 2 x 2 cells per thread: column pair cp, row pair rp (see the bank note above).
  const int cpr = (tw >> 1);                   // column pairs per row
  const int g8 = cpr < 8 ? cpr : 8;
  const int tid = threadIdx.x;
  const int cp = (tid % g8) + g8 * ((tid / (2 * g8)) % (cpr / g8));
  const int rp = ((tid / g8) & 1) + 2 * (tid / (2 * cpr));
  const int lx = 2 * cp, ly = 2 * rp;
  const int cx = tx0 + lx, cy = ty0 + ly;
  if (L.store_mask) {
    // masked-store launch: a warp without a cell to store skips the work (warp-uniform,
    // after the last barrier)
    int need = 0;
    for (int h = 0; h < 2; ++h)
      for (int g = 0; g < 2; ++g) {
        const int c = cx + g, r = cy + h;
        if (c < R.x0 + R.w && r < R.y0 + R.h && L.store_mask[(int64_t)r * L.nx + c]) need = 1;
      }
    if (!__any_sync(0xffffffffu, need)) return;
  }
  const int pair = blockIdx.y;
  const int r0 = T.run_start[pair], r1 = T.run_start[pair + 1];
  const float qnan = __int_as_float(0x7fc00000);
  auto tile_at = [&](int row, int col) {  // staged height (row, col), NaN when unknown
    const int k = row < sh - 1 ? pair_index(row, col, sw2) : pair_index(row - 1, col, sw2);
    const float v = row < sh - 1 ? pt[k].x : pt[k].y, m = row < sh - 1 ? pm[k].x : pm[k].y;
    return m != 0.f ? v : qnan;
  };

  // references: the centre height, else the first known footprint cell in run order
  float ref[2][2];  // [col g][row h]
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float r = tile_at(ry + ly + h, rx + lx + g);
      if (r != r) {
        r = 0.f;
        bool found = false;
        for (int q = r0; q < r1 && !found; ++q) {
          const uint32_t pk = T.runs[q];
          const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
          for (int d = lo; d <= hi; ++d) {
            const float v = tile_at(ry + ly + h + dj, rx + lx + g + d);
            if (v == v) {
              r = v;
              found = true;
              break;
            }
          }
        }
      }
      ref[g][h] = r;
    }
  const float2 nref[2] = {f2(-ref[0][0], -ref[0][1]), f2(-ref[1][0], -ref[1][1])};
  const float2 mref[2] = {nref[0], nref[1]};

  float2 S0[2], S1[2], S2[2], S3[2];
#pragma unroll
  for (int g = 0; g < 2; ++g) S0[g] = S1[g] = S2[g] = S3[g] = f2(0.f, 0.f);
  const int tq = threadIdx.x;
  auto Qs = [&](int k, int g) -> float2& { return qs[(g * 6 + k) * kThreads + tq]; };
  const float2 one2 = f2(1.f, 1.f);
  for (int q = r0; q < r1; ++q) {
    const uint32_t pk = T.runs[q];
    const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
    const int row = ry + ly + dj;  // pair row of this thread for the run
    const bool masked = __any_sync(0xffffffffu, rowflag[row] | rowflag[row + 1]);
    const int base = pair_index(row, rx + lx + lo, sw2);
    const float2* pq = pt + base;
    const float2* pw = pm + base;
    const int len = hi - lo + 1;
    float2 a[2], bb[2], s3[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) a[g] = bb[g] = s3[g] = f2(0.f, 0.f);
    float2 di2 = f2((float)lo, (float)lo);
    if (!masked) {
      float2 w0 = pq[0];
#pragma unroll 4
      for (int i = 0; i < len; ++i) {
        const float2 w1 = pq[i + 1];
        float2 zp = add2(w0, nref[0]);
        a[0] = add2(a[0], zp);
        bb[0] = fma2(di2, zp, bb[0]);
        s3[0] = fma2(zp, zp, s3[0]);
        zp = add2(w1, nref[1]);
        a[1] = add2(a[1], zp);
        bb[1] = fma2(di2, zp, bb[1]);
        s3[1] = fma2(zp, zp, s3[1]);
        w0 = w1;
        di2 = add2(di2, one2);
      }
    } else {
      // unknown heights were staged as 0 with weight 0: z' = fma(-ref, m, z) is exactly
      // z - ref for known points and 0 for unknown ones; x = 1 - m counts the missing points
      float2 z0 = pq[0], m0 = pw[0];
      float2 qn[2], qx[2], qxx[2];
#pragma unroll
      for (int g = 0; g < 2; ++g) qn[g] = qx[g] = qxx[g] = f2(0.f, 0.f);
      const float2 neg1 = f2(-1.f, -1.f);
#pragma unroll 2
      for (int i = 0; i < len; ++i) {
        const float2 z1 = pq[i + 1], m1 = pw[i + 1];
        const float2 d2 = __fmul2_rn(di2, di2);
        const float2 zs[2] = {z0, z1}, ms[2] = {m0, m1};
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const float2 zp = fma2(mref[g], ms[g], zs[g]);
          const float2 x = fma2(neg1, ms[g], one2);
          a[g] = add2(a[g], zp);
          bb[g] = fma2(di2, zp, bb[g]);
          s3[g] = fma2(zp, zp, s3[g]);
          qn[g] = add2(qn[g], x);
          qx[g] = fma2(di2, x, qx[g]);
          qxx[g] = fma2(d2, x, qxx[g]);
        }
        z0 = z1;
        m0 = m1;
        di2 = add2(di2, one2);
      }
      const float fdj = (float)dj;
      const float2 dj2 = f2(fdj, fdj), dj22 = f2(fdj * fdj, fdj * fdj);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        Qs(0, g) = add2(Qs(0, g), qn[g]);
        Qs(1, g) = add2(Qs(1, g), qx[g]);
        Qs(2, g) = fma2(dj2, qn[g], Qs(2, g));
        Qs(3, g) = add2(Qs(3, g), qxx[g]);
        Qs(4, g) = fma2(dj2, qx[g], Qs(4, g));
        Qs(5, g) = fma2(dj22, qn[g], Qs(5, g));
      }
    }
    const float2 dj2 = f2((float)dj, (float)dj);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      S0[g] = add2(S0[g], a[g]);
      S1[g] = add2(S1[g], bb[g]);
      S2[g] = fma2(dj2, a[g], S2[g]);
      S3[g] = add2(S3[g], s3[g]);
    }
  }

  const int k0 = pair, k1 = pair + T.n_pairs;
  const float ct = T.cos_t[pair], st = T.sin_t[pair];
  const int64_t chs = (int64_t)L.n_yaw * L.plane;
  const int* mom = T.mom[pair];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int cyh = cy + h;
    if (cyh >= R.y0 + R.h) break;
    int pr = cyh + L.ring_y;
    if (pr >= L.ny) pr -= L.ny;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int c = cx + g;
      if (c >= R.x0 + R.w) break;
      if (L.store_mask && !L.store_mask[(int64_t)cyh * L.nx + c]) continue;
      float qv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) qv[k] = h ? Qs(k, g).y : Qs(k, g).x;
      const float q0 = qv[0], q1 = qv[1], q2 = qv[2], q3 = qv[3], q4 = qv[4], q5 = qv[5];
      const Cell o = finish_cell(mom[0] - (int)q0, mom[1] - (int)q1, mom[2] - (int)q2, mom[3] - (int)q3,
                                 mom[4] - (int)q4, mom[5] - (int)q5, h ? S0[g].y : S0[g].x, h ? S1[g].y : S1[g].x,
                                 h ? S2[g].y : S2[g].x, h ? S3[g].y : S3[g].x, ref[g][h], T.n_min[pair], ct, st, L);
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
}

__global__ void copy_out_kernel(const Launch L, float* __restrict__ dst, uint8_t* __restrict__ fdst) {
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

template <typename E, bool COMP>
cudaError_t launch_typed(const Tables& T, const Launch& L, cudaStream_t stream) {
  if (!COMP) {
    size_t pairs = 0;
    for (int i = 0; i < L.n_rects; ++i) {
      const int lg = L.rects[i].log_tpr;
      const size_t sw2 = (size_t)(kG << lg) + 2 * T.rx + 1, sh = (size_t)(kThreads >> lg) + 2 * T.ry;
      const size_t s = (sh - 1) * sw2;
      pairs = s > pairs ? s : pairs;
    }
    const size_t smem = kMaxStageRows * sizeof(float) + (2 * pairs + 12 * kThreads) * sizeof(float2);
    auto kern = assess_kernel_x2<E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(L.tile_start[L.n_rects], T.n_pairs);
    kern<<<grid, kThreads, smem, stream>>>(T, L);
    return cudaGetLastError();
  }
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
  if (L.tile_start[L.n_rects] == 0) return cudaSuccess;
  const bool comp = precision == SEB_COMPENSATED;
  switch (elev_dtype) {
    case SEB_F32:
      return comp ? launch_typed<float, true>(T, L, stream) : launch_typed<float, false>(T, L, stream);
    case SEB_BF16:
      return comp ? launch_typed<__nv_bfloat16, true>(T, L, stream)
                  : launch_typed<__nv_bfloat16, false>(T, L, stream);
    default:
      return comp ? launch_typed<__half, true>(T, L, stream) : launch_typed<__half, false>(T, L, stream);
  }
}

cudaError_t launch_copy_out(const Launch& L, float* out_dev, uint8_t* flags_dev, cudaStream_t stream) {
  const int64_t total = (int64_t)L.n_yaw * L.plane;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  copy_out_kernel<<<blocks, 256, 0, stream>>>(L, out_dev, flags_dev);
  return cudaGetLastError();
}

}  // namespace seb
