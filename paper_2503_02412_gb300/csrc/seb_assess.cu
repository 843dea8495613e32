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
  // N^2 Cov_xy-block numerators are exact integers.
  const long long nxx = (long long)N * MXX - (long long)MX * MX;
  const long long nxy = (long long)N * MXY - (long long)MX * MY;
  const long long nyy = (long long)N * MYY - (long long)MY * MY;
  const float fMX = (float)MX, fMY = (float)MY;
  float c[6];
  c[0] = (float)nxx * inv_n2 * res * res;
  c[1] = (float)nxy * inv_n2 * res * res;
  c[3] = (float)nyy * inv_n2 * res * res;
  c[2] = fmaf(S1, fN, -fMX * S0) * inv_n2 * res;
  c[4] = fmaf(S2, fN, -fMY * S0) * inv_n2 * res;
  c[5] = fmaf(S3, fN, -S0 * S0) * inv_n2;
  float n[3], gap;
  min_eigpair<float>(c, n, &gap);
  uint32_t flags = 0;
  const float tr = c[0] + c[3] + c[5];
  float lam;
  if (gap < L.gap_fp64) {
    // Near-degenerate: covariance and eigen-solve again in FP64 from the same moments.
    flags |= SEB_FLAG_FP64;
    const double dN = (double)N, i2 = 1.0 / (dN * dN), r = (double)res;
    double cd[6];
    cd[0] = (double)nxx * i2 * r * r;
    cd[1] = (double)nxy * i2 * r * r;
    cd[3] = (double)nyy * i2 * r * r;
    cd[2] = ((double)S1 * dN - (double)MX * (double)S0) * i2 * r;
    cd[4] = ((double)S2 * dN - (double)MY * (double)S0) * i2 * r;
    cd[5] = ((double)S3 * dN - (double)S0 * (double)S0) * i2;
    double nd[3], gd;
    min_eigpair<double>(cd, nd, &gd);
    const double ld = cd[0] * nd[0] * nd[0] + cd[3] * nd[1] * nd[1] + cd[5] * nd[2] * nd[2] +
                      2.0 * (cd[1] * nd[0] * nd[1] + cd[2] * nd[0] * nd[2] + cd[4] * nd[1] * nd[2]);
    const double trd = cd[0] + cd[3] + cd[5];
    n[0] = (float)nd[0];
    n[1] = (float)nd[1];
    n[2] = (float)nd[2];
    lam = (float)(ld > 0.0 ? ld : 0.0);
    o.rough = (float)((ld > 0.0 ? ld : 0.0) / trd);
    atomicAdd(&L.counters[0], 1ull);
    if (gd < 1e-12) flags |= SEB_FLAG_DEGENERATE;
  } else {
    lam = c[0] * n[0] * n[0] + c[3] * n[1] * n[1] + c[5] * n[2] * n[2] +
          2.f * (c[1] * n[0] * n[1] + c[2] * n[0] * n[2] + c[4] * n[1] * n[2]);
    lam = fmaxf(lam, 0.f);
    o.rough = lam / tr;
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
  (void)lam;
  return o;
}

__device__ __forceinline__ int unpack(uint32_t v, int sh) { return (int)((v >> sh) & 0xffu) - 128; }

// Moments of the 4 cells of this thread for yaw pair `pair`.
template <bool MASKED, bool COMP>
__device__ __forceinline__ void accumulate(const Tables& T, int pair, const float* __restrict__ sc,
                                           int sw, const float ref[kG], float S0[kG], float S1[kG],
                                           float S2[kG], float S3[kG], int N[kG], int MX[kG],
                                           int MY[kG], int MXX[kG], int MXY[kG], int MYY[kG]) {
  float C0[kG], C1[kG], C2[kG], C3[kG];  // compensation terms
  float fN[kG], fMX[kG], fMY[kG], fMXX[kG], fMXY[kG], fMYY[kG];
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    S0[g] = S1[g] = S2[g] = S3[g] = 0.f;
    C0[g] = C1[g] = C2[g] = C3[g] = 0.f;
    fN[g] = fMX[g] = fMY[g] = fMXX[g] = fMXY[g] = fMYY[g] = 0.f;
  }
  const int r0 = T.run_start[pair], r1 = T.run_start[pair + 1];
  for (int q = r0; q < r1; ++q) {
    const uint32_t pk = T.runs[q];
    const int dj = unpack(pk, 0), lo = unpack(pk, 8), hi = unpack(pk, 16);
    const float* p = sc + dj * sw + lo;
    float a[kG], ac[kG], b[kG], bc[kG], s3[kG], s3c[kG], cn[kG], cx[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) a[g] = ac[g] = b[g] = bc[g] = s3[g] = s3c[g] = cn[g] = cx[g] = 0.f;
    float w0 = p[0], w1 = p[1], w2 = p[2];
    float di = (float)lo;
    const int len = hi - lo + 1;
#pragma unroll 2
    for (int i = 0; i < len; ++i) {
      const float w3 = p[i + 3];
      const float wv[kG] = {w0, w1, w2, w3};
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        float zp, m = 1.f;
        if (MASKED) {
          const bool known = wv[g] == wv[g];
          m = known ? 1.f : 0.f;
          zp = fmaf(-ref[g], m, known ? wv[g] : 0.f);
        } else {
          zp = wv[g] - ref[g];
        }
        if (COMP) {
          nadd(a[g], ac[g], zp);
          nadd(b[g], bc[g], __fmul_rn(di, zp));
          nadd(s3[g], s3c[g], __fmul_rn(zp, zp));
        } else {
          a[g] += zp;
          b[g] = fmaf(di, zp, b[g]);
          s3[g] = fmaf(zp, zp, s3[g]);
        }
        if (MASKED) {
          cn[g] += m;
          cx[g] = fmaf(di, m, cx[g]);
          fMXX[g] = fmaf(di * di, m, fMXX[g]);
        }
      }
      w0 = w1;
      w1 = w2;
      w2 = w3;
      di += 1.f;
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
      if (MASKED) {
        fN[g] += cn[g];
        fMX[g] += cx[g];
        fMY[g] = fmaf(fdj, cn[g], fMY[g]);
        fMYY[g] = fmaf(fdj * fdj, cn[g], fMYY[g]);
        fMXY[g] = fmaf(fdj, cx[g], fMXY[g]);
      }
    }
  }
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    if (COMP) {
      S0[g] += C0[g];
      S1[g] += C1[g];
      S2[g] += C2[g];
      S3[g] += C3[g];
    }
    if (MASKED) {
      N[g] = (int)fN[g];
      MX[g] = (int)fMX[g];
      MY[g] = (int)fMY[g];
      MXX[g] = (int)fMXX[g];
      MXY[g] = (int)fMXY[g];
      MYY[g] = (int)fMYY[g];
    } else {
      N[g] = T.mom[pair][0];
      MX[g] = T.mom[pair][1];
      MY[g] = T.mom[pair][2];
      MXX[g] = T.mom[pair][3];
      MXY[g] = T.mom[pair][4];
      MYY[g] = T.mom[pair][5];
    }
  }
}

template <typename E, bool COMP>
__global__ void __launch_bounds__(kThreads, 2)
    assess_kernel(const __grid_constant__ Tables T, const __grid_constant__ Launch L) {
  extern __shared__ float tile[];
  if (blockDim.x != kThreads || blockIdx.y >= (unsigned)T.n_pairs) {
    if (threadIdx.x == 0) atomicOr(L.err, kErrLaunchShape);
    return;
  }
  // Which rectangle and tile this CTA covers.
  const int b = blockIdx.x;
  int ri = 0;
#pragma unroll 1
  while (ri + 1 < L.n_rects && b >= L.tile_start[ri + 1]) ++ri;
  const Rect R = L.rects[ri];
  const int t = b - L.tile_start[ri];
  const int tx0 = R.x0 + (t % L.tiles_x[ri]) * kTileW;
  const int ty0 = R.y0 + (t / L.tiles_x[ri]) * kTileH;
  const int rx = T.rx, ry = T.ry, sw = L.sw, sh = L.sh;

  // Stage tile + halo (outside the window = NaN = unknown).
  const E* __restrict__ elev = static_cast<const E*>(L.elev);
  const float qnan = __int_as_float(0x7fc00000);
  int any_nan = 0;
  for (int idx = threadIdx.x; idx < sw * sh; idx += kThreads) {
    const int row = idx / sw, col = idx - row * sw;
    const int gy = ty0 - ry + row, gx = tx0 - rx + col;
    float v = qnan;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny)
      v = to_f32<E>(elev[(int64_t)gy * L.nx + gx]);
    any_nan |= (v != v);
    tile[idx] = v;
  }
  any_nan = __syncthreads_or(any_nan);

  const int lx = (threadIdx.x & 7) * kG;
  const int ly = threadIdx.x >> 3;
  const int cx = tx0 + lx, cy = ty0 + ly;
  const int pair = blockIdx.y;
  const float* sc = tile + (ry + ly) * sw + rx + lx;  // centre of cell g is sc[g]

  float ref[kG];
#pragma unroll
  for (int g = 0; g < kG; ++g) ref[g] = sc[g];
  if (any_nan) {
    // Unknown centre: the first known cell of the footprint in run order.
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      if (ref[g] == ref[g]) continue;
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
  }

  float S0[kG], S1[kG], S2[kG], S3[kG];
  int N[kG], MX[kG], MY[kG], MXX[kG], MXY[kG], MYY[kG];
  if (any_nan)
    accumulate<true, COMP>(T, pair, sc, sw, ref, S0, S1, S2, S3, N, MX, MY, MXX, MXY, MYY);
  else
    accumulate<false, COMP>(T, pair, sc, sw, ref, S0, S1, S2, S3, N, MX, MY, MXX, MXY, MYY);

  if (cy >= R.y0 + R.h) return;
  const int k0 = pair, k1 = pair + T.n_pairs;
  const float ct = T.cos_t[pair], st = T.sin_t[pair];
  int pr = cy + L.ring_y;
  if (pr >= L.ny) pr -= L.ny;
  const int64_t chs = (int64_t)L.n_yaw * L.plane;
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    const int c = cx + g;
    if (c >= R.x0 + R.w) break;
    const Cell o = finish_cell(N[g], MX[g], MY[g], MXX[g], MXY[g], MYY[g], S0[g], S1[g], S2[g], S3[g],
                               ref[g], T.n_min[pair], ct, st, L);
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
  const size_t smem = (size_t)L.sw * L.sh * sizeof(float);
  auto kern = assess_kernel<E, COMP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(L.tile_start[L.n_rects], T.n_pairs);
  kern<<<grid, kThreads, smem, stream>>>(T, L);
  return cudaGetLastError();
}

}  // namespace

size_t assess_smem_bytes(const Tables& T) {
  int sw = kTileW + 2 * T.rx;
  if ((sw & 1) == 0) ++sw;
  return (size_t)sw * (kTileH + 2 * T.ry) * sizeof(float);
}

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
