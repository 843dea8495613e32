// Learned surrogate of the SE(2) assessment: a small BF16 convolutional network that maps an
// elevation patch to the per-yaw (z - z_cell, pitch, roll, risk) of Algorithm 1, trained on
// the GPU on patches the exact kernel labels, and run fully convolutionally over a map with the
// exact kernel as fallback near unknown cells and step edges.  The paper defines no learned
// model (it names learned traversability as less reliable, Sec. II-A); every prediction is measured
// against the exact kernel.
//
// Network (channel-last, valid convolutions): slope features (dz/dx, dz/dy by central
// differences) -> 4 x [3x3 conv, 32 channels, dilation 1, 2, 4, 8, ReLU] -> 1x1 head to
// 4 x n_pairs outputs.  Receptive field 31 cells: a 48 x 48 elevation crop (46 x 46 features)
// gives the 16 x 16 centre cells.  Weights and stored activations in BF16, accumulation and
// gradients in FP32, FP32 master weights with Adam.  Output channel 4k + q of yaw pair k:
// q = 0 (z - z_cell) x 10 (decimetres), 1 pitch, 2 roll, 3 risk; yaw k + n_pairs is the same
// with pitch and roll negated.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "seb_device.cuh"
#include "seb_internal.h"

namespace {

constexpr int kHid = 32;
constexpr int kInF = 2;
constexpr int kCrop = 48;
constexpr int kFeat = 46;
constexpr int kOutSide = 16;
constexpr int kMargin = 16;  // output cell = crop cell + 16 (features start at crop cell 1, RF 31)
constexpr int kDil[4] = {1, 2, 4, 8};
constexpr int kSide[5] = {46, 44, 40, 32, 16};  // feature side, then after each layer
constexpr float kZScale = 10.f;

typedef __nv_bfloat16 bf16;

__host__ __device__ inline int64_t conv_w(int cin) { return (int64_t)kHid * 9 * cin; }

struct ParamLayout {
  int64_t w[4], b[4], wh, bh, n;
};

ParamLayout param_layout(int nout) {
  ParamLayout P;
  int64_t o = 0;
  int cin = kInF;
  for (int l = 0; l < 4; ++l) {
    P.w[l] = o;
    o += conv_w(cin);
    P.b[l] = o;
    o += kHid;
    cin = kHid;
  }
  P.wh = o;
  o += (int64_t)nout * kHid;
  P.bh = o;
  o += nout;
  P.n = o;
  return P;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (S. Vigna) of (seed, stream, index), Box-Muller.
// ------------------------------------------------------------------------------------------------
__host__ __device__ inline uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__device__ inline float gauss(uint64_t seed, uint64_t idx) {
  const uint64_t h = splitmix(seed ^ splitmix(idx));
  const float u1 = ((float)(uint32_t)(h >> 40) + 1.f) * (1.f / 16777217.f);  // (0, 1]
  const float u2 = (float)(uint32_t)(h & 0xffffffu) * (1.f / 16777216.f);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// ------------------------------------------------------------------------------------------------
// Terrain (the small-map recipe): tilted plane + 8 Gaussian bumps + Gaussian noise.
// params per world: slope (tan), azimuth, noise sigma, unused, then (amp, sigma, cx, cy) x 8.
// ------------------------------------------------------------------------------------------------
constexpr int kTerrainParams = 4 + 8 * 4;

__global__ void terrain_kernel(const float* __restrict__ prm, int n, int nx, int ny, float res, uint64_t seed,
                               float* __restrict__ out) {
  const int64_t total = (int64_t)n * nx * ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(i / ((int64_t)nx * ny));
    const int64_t rem = i - (int64_t)w * nx * ny;
    const int r = (int)(rem / nx), c = (int)(rem - (int64_t)r * nx);
    const float* p = prm + (int64_t)w * kTerrainParams;
    const float x = (c + 0.5f) * res, y = (r + 0.5f) * res;
    float sa, ca;
    sincosf(p[1], &sa, &ca);
    float z = p[0] * (ca * x + sa * y);
    for (int j = 0; j < 8; ++j) {
      const float* q = p + 4 + 4 * j;
      const float dx = x - q[2], dy = y - q[3];
      z += q[0] * expf(-(dx * dx + dy * dy) / (2.f * q[1] * q[1]));
    }
    out[i] = z + p[2] * gauss(seed, (uint64_t)i);
  }
}

// ------------------------------------------------------------------------------------------------
// Training batch: features of a 48 x 48 crop and labels of its 16 x 16 centre.
// ------------------------------------------------------------------------------------------------
__device__ inline float feat_x(const float* e, int64_t ld, int r, int c, float inv2res) {
  const float v = (e[(int64_t)r * ld + c + 1] - e[(int64_t)r * ld + c - 1]) * inv2res;
  return v == v ? v : 0.f;
}
__device__ inline float feat_y(const float* e, int64_t ld, int r, int c, float inv2res) {
  const float v = (e[(int64_t)(r + 1) * ld + c] - e[(int64_t)(r - 1) * ld + c]) * inv2res;
  return v == v ? v : 0.f;
}

__global__ void gather_kernel(const float* __restrict__ elev, const float* __restrict__ exact, int nx, int ny,
                              int n_yaw, const int32_t* __restrict__ centres, int n, float res, int nout,
                              bf16* __restrict__ feat, float* __restrict__ labels, uint32_t* err) {
  const int pi = blockIdx.x;
  if (pi >= n) return;
  const int cx = centres[2 * pi], cy = centres[2 * pi + 1];
  const int x0 = cx - kCrop / 2, y0 = cy - kCrop / 2;
  const float qnan = __int_as_float(0x7fc00000);
  const bool inside = x0 >= 0 && y0 >= 0 && x0 + kCrop <= nx && y0 + kCrop <= ny;
  if (!inside && threadIdx.x == 0) atomicOr(err, 2u);
  bf16* f = feat + (int64_t)pi * kFeat * kFeat * kInF;
  const float inv2res = 0.5f / res;
  for (int i = threadIdx.x; i < kFeat * kFeat; i += blockDim.x) {
    const int r = i / kFeat, c = i - r * kFeat;
    const int er = y0 + 1 + r, ec = x0 + 1 + c;
    f[2 * i] = __float2bfloat16_rn(inside ? feat_x(elev, nx, er, ec, inv2res) : 0.f);
    f[2 * i + 1] = __float2bfloat16_rn(inside ? feat_y(elev, nx, er, ec, inv2res) : 0.f);
  }
  float* lab = labels + (int64_t)pi * kOutSide * kOutSide * nout;
  const int64_t plane = (int64_t)nx * ny, chs = plane * n_yaw;
  const int npairs = nout / 4;
  for (int i = threadIdx.x; i < kOutSide * kOutSide * nout; i += blockDim.x) {
    const int cell = i / nout, ch = i - cell * nout;
    const int k = ch >> 2, q = ch & 3;
    const int r = y0 + kMargin + cell / kOutSide, c = x0 + kMargin + cell % kOutSide;
    float v = qnan;
    if (inside && k < npairs) {
      const int64_t idx = (int64_t)k * plane + (int64_t)r * nx + c;
      if (q == 0)
        v = (exact[idx] - elev[(int64_t)r * nx + c]) * kZScale;
      else if (q == 1)
        v = exact[chs + idx];
      else if (q == 2)
        v = exact[2 * chs + idx];
      else
        v = exact[4 * chs + idx];
    }
    lab[i] = v;
  }
}

// Slope features of a whole map: [ny - 2][nx - 2][2].
__global__ void map_features_kernel(const float* __restrict__ elev, int nx, int ny, float res, bf16* __restrict__ feat) {
  const int W = nx - 2, H = ny - 2;
  const float inv2res = 0.5f / res;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)W * H;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / W), c = (int)(i - (int64_t)r * W);
    feat[2 * i] = __float2bfloat16_rn(feat_x(elev, nx, r + 1, c + 1, inv2res));
    feat[2 * i + 1] = __float2bfloat16_rn(feat_y(elev, nx, r + 1, c + 1, inv2res));
  }
}

// ------------------------------------------------------------------------------------------------
// Convolution layers (SIMT, FP32 accumulation).
// ------------------------------------------------------------------------------------------------
// y[b, i, j, o] = relu(bias[o] + sum_{u, v, c} w[o, u, v, c] x[b, i + u d, j + v d, c]).
template <int CIN>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                       const float* __restrict__ bias, int B, int H, int W, int d,
                                                       bf16* __restrict__ y) {
  __shared__ float ws[9 * CIN * kHid];  // [tap][ci][co]
  for (int i = threadIdx.x; i < 9 * CIN * kHid; i += blockDim.x) {
    const int co = i % kHid, t = i / kHid;  // t = tap * CIN + ci
    const int tap = t / CIN, ci = t % CIN;
    ws[i] = __bfloat162float(w[((int64_t)co * 9 + tap) * CIN + ci]);
  }
  __syncthreads();
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  const int64_t total = (int64_t)B * Ho * Wo;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)Ho * Wo));
    const int rem = (int)(p - (int64_t)b * Ho * Wo);
    const int i = rem / Wo, j = rem - i * Wo;
    float acc[kHid];
#pragma unroll
    for (int o = 0; o < kHid; ++o) acc[o] = bias[o];
    for (int tap = 0; tap < 9; ++tap) {
      const int u = tap / 3, v = tap - u * 3;
      const bf16* xp = x + (((int64_t)b * H + i + u * d) * W + j + v * d) * CIN;
      for (int ci = 0; ci < CIN; ++ci) {
        const float xv = __bfloat162float(xp[ci]);
        const float* wr = ws + (tap * CIN + ci) * kHid;
#pragma unroll
        for (int o = 0; o < kHid; ++o) acc[o] = fmaf(xv, wr[o], acc[o]);
      }
    }
    // 16-byte stores: the 32 outputs of a pixel are 64 contiguous bytes
    uint4* yp = reinterpret_cast<uint4*>(y + p * kHid);
#pragma unroll
    for (int q = 0; q < kHid / 8; ++q) {
      uint4 v;
      __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        h2[t] = __floats2bfloat162_rn(fmaxf(acc[8 * q + 2 * t], 0.f), fmaxf(acc[8 * q + 2 * t + 1], 0.f));
      yp[q] = v;
    }
  }
}

// 1x1 head: pred[p, o] = bh[o] + sum_c wh[o, c] a[p, c]; grid.y chunks the outputs by 16.
__global__ void __launch_bounds__(128) head_fwd_kernel(const bf16* __restrict__ a, const bf16* __restrict__ wh,
                                                       const float* __restrict__ bh, int64_t P, int nout,
                                                       float* __restrict__ pred) {
  const int o0 = blockIdx.y * 16;
  __shared__ float ws[16 * kHid];
  for (int i = threadIdx.x; i < 16 * kHid; i += blockDim.x) {
    const int o = o0 + i / kHid;
    ws[i] = o < nout ? __bfloat162float(wh[(int64_t)o * kHid + i % kHid]) : 0.f;
  }
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float av[kHid];
#pragma unroll
    for (int c = 0; c < kHid; ++c) av[c] = __bfloat162float(a[p * kHid + c]);
    for (int k = 0; k < 16 && o0 + k < nout; ++k) {
      float s = bh[o0 + k];
#pragma unroll
      for (int c = 0; c < kHid; ++c) s = fmaf(ws[k * kHid + c], av[c], s);
      pred[p * nout + o0 + k] = s;
    }
  }
}

// Mean squared error over the finite labels: per-block (sum, count) partials.
__global__ void loss_partials_kernel(const float* __restrict__ pred, const float* __restrict__ lab, int64_t n,
                                     float* __restrict__ partials) {
  float s = 0.f, c = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float l = lab[i];
    if (l == l) {
      const float d = pred[i] - l;
      s = fmaf(d, d, s);
      c += 1.f;
    }
  }
  __shared__ float ss[256], sc[256];
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = ss[0];
    partials[2 * blockIdx.x + 1] = sc[0];
  }
}

// Sums the partials in a fixed order: tot[0] = loss (mean), tot[1] = count.
// One block of 256 threads: thread t sums partials t, t + 256, ... in FP64, then a fixed-order
// tree adds the 256 sums (deterministic: the same order every call).
__global__ void loss_reduce_kernel(const float* __restrict__ partials, int nb, float* __restrict__ tot,
                                   float* __restrict__ loss_out) {
  __shared__ double ss[256], sc[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s += partials[2 * i];
    c += partials[2 * i + 1];
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cc = sc[0] > 0 ? sc[0] : 1.0;
    tot[1] = (float)cc;
    tot[0] = (float)(ss[0] / cc);
    if (loss_out) *loss_out = tot[0];
  }
}

__global__ void dpred_kernel(const float* __restrict__ pred, const float* __restrict__ lab, int64_t n,
                             const float* __restrict__ tot, float* __restrict__ dpred) {
  const float scale = 2.f / tot[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float l = lab[i];
    dpred[i] = l == l ? scale * (pred[i] - l) : 0.f;
  }
}

// Head backward, input side: da[p, c] = sum_o dpred[p, o] wh[o, c].
__global__ void head_bwd_dx_kernel(const float* __restrict__ dpred, const bf16* __restrict__ wh, int64_t P, int nout,
                                   float* __restrict__ da) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float acc[kHid];
#pragma unroll
    for (int c = 0; c < kHid; ++c) acc[c] = 0.f;
    for (int o = 0; o < nout; ++o) {
      const float g = dpred[p * nout + o];
#pragma unroll
      for (int c = 0; c < kHid; ++c) acc[c] = fmaf(g, __bfloat162float(wh[o * kHid + c]), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kHid; ++c) da[p * kHid + c] = acc[c];
  }
}

// Head backward, weight side: per chunk of pixels (staged 64 at a time in shared memory),
// partial dwh[o, c] and dbh[o].
constexpr int kSub = 64;     // pixels staged per shared-memory round
constexpr int kChunkPx = 1024;  // pixels per CTA (one partial per CTA)
constexpr int kHeadChunkPx = 256;  // head weight gradient: pixels per CTA

__global__ void __launch_bounds__(256) head_bwd_dw_kernel(const float* __restrict__ dpred, const bf16* __restrict__ a,
                                                          int64_t P, int nout, int chunk, float* __restrict__ partials) {
  extern __shared__ float sm[];
  float* gs = sm;                 // [kSub][nout]
  float* as = sm + kSub * nout;   // [kSub][kHid]
  const int E = nout * kHid + nout;
  const int per = (E + 255) / 256;
  float acc[24];
  for (int j = 0; j < per && j < 24; ++j) acc[j] = 0.f;
  const int64_t p0 = (int64_t)blockIdx.x * chunk;
  for (int64_t q0 = p0; q0 < p0 + chunk && q0 < P; q0 += kSub) {
    const int np = (int)(P - q0 < kSub ? P - q0 : kSub);
    __syncthreads();
    for (int i = threadIdx.x; i < kSub * nout; i += blockDim.x) gs[i] = i < np * nout ? dpred[q0 * nout + i] : 0.f;
    for (int i = threadIdx.x; i < kSub * kHid; i += blockDim.x)
      as[i] = i < np * kHid ? __bfloat162float(a[q0 * kHid + i]) : 0.f;
    __syncthreads();
    for (int j = 0; j < per && j < 24; ++j) {
      const int e = threadIdx.x + 256 * j;
      if (e >= E) break;
      float s = acc[j];
      if (e < nout * kHid) {
        const int o = e / kHid, c = e - o * kHid;
        for (int p = 0; p < kSub; ++p) s = fmaf(gs[p * nout + o], as[p * kHid + c], s);
      } else {
        const int o = e - nout * kHid;
        for (int p = 0; p < kSub; ++p) s += gs[p * nout + o];
      }
      acc[j] = s;
    }
  }
  float* part = partials + (int64_t)blockIdx.x * E;
  for (int j = 0; j < per && j < 24; ++j) {
    const int e = threadIdx.x + 256 * j;
    if (e < E) part[e] = acc[j];
  }
}

// Conv backward, input side, through the ReLU of this layer's output y:
// dx[b, r, s, c] = sum_{u, v, o} w[o, u, v, c] dz[b, r - u d, s - v d, o], dz = dy * (y > 0).
__global__ void __launch_bounds__(128) conv_bwd_dx_kernel(const float* __restrict__ dy, const bf16* __restrict__ y,
                                                          const bf16* __restrict__ w, int B, int H, int W, int d,
                                                          float* __restrict__ dx) {
  __shared__ float ws[9 * kHid * kHid];  // [tap][o][c]
  for (int i = threadIdx.x; i < 9 * kHid * kHid; i += blockDim.x) {
    const int c = i % kHid, t = i / kHid;  // t = tap * kHid + o
    const int tap = t / kHid, o = t % kHid;
    ws[i] = __bfloat162float(w[((int64_t)o * 9 + tap) * kHid + c]);
  }
  __syncthreads();
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  const int64_t total = (int64_t)B * H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)H * W));
    const int rem = (int)(p - (int64_t)b * H * W);
    const int r = rem / W, s = rem - r * W;
    float acc[kHid];
#pragma unroll
    for (int c = 0; c < kHid; ++c) acc[c] = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
      const int u = tap / 3, v = tap - u * 3;
      const int i = r - u * d, j = s - v * d;
      if (i < 0 || i >= Ho || j < 0 || j >= Wo) continue;
      const int64_t q = ((int64_t)b * Ho + i) * Wo + j;
      for (int o = 0; o < kHid; ++o) {
        const float yo = __bfloat162float(y[q * kHid + o]);
        if (!(yo > 0.f)) continue;
        const float g = dy[q * kHid + o];
        const float* wr = ws + (tap * kHid + o) * kHid;
#pragma unroll
        for (int c = 0; c < kHid; ++c) acc[c] = fmaf(g, wr[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kHid; ++c) dx[p * kHid + c] = acc[c];
  }
}

// Conv backward, weight side: per chunk of output pixels (staged kSub at a time: dz with the
// ReLU mask applied, and the im2col rows of the input), partial dw[o, u, v, c] and db[o].
// Thread t owns output channel o = t / 8 and a contiguous eighth of the 9 * CIN taps.
template <int CIN>
__global__ void __launch_bounds__(256) conv_bwd_dw_kernel(const float* __restrict__ dy, const bf16* __restrict__ y,
                                                          const bf16* __restrict__ x, int B, int H, int W, int d,
                                                          float* __restrict__ partials) {
  constexpr int KW = 9 * CIN;
  constexpr int PER = (KW + 7) / 8;
  __shared__ float dzs[kSub][kHid];
  __shared__ bf16 xs[kSub][KW];
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  const int64_t P = (int64_t)B * Ho * Wo;
  const int o = threadIdx.x >> 3, k0 = (threadIdx.x & 7) * PER;
  float acc[PER], accb = 0.f;
#pragma unroll
  for (int j = 0; j < PER; ++j) acc[j] = 0.f;
  const int64_t p0 = (int64_t)blockIdx.x * kChunkPx;
  for (int64_t q0 = p0; q0 < p0 + kChunkPx && q0 < P; q0 += kSub) {
    __syncthreads();
    for (int i = threadIdx.x; i < kSub * kHid; i += blockDim.x) {
      const int pp = i / kHid, oo = i - pp * kHid;
      const int64_t p = q0 + pp;
      float g = 0.f;
      if (p < P && __bfloat162float(y[p * kHid + oo]) > 0.f) g = dy[p * kHid + oo];
      dzs[pp][oo] = g;
    }
    for (int i = threadIdx.x; i < kSub * KW; i += blockDim.x) {
      const int pp = i / KW, k = i - pp * KW;
      const int64_t p = q0 + pp;
      bf16 v = __float2bfloat16_rn(0.f);
      if (p < P) {
        const int b = (int)(p / ((int64_t)Ho * Wo));
        const int rem = (int)(p - (int64_t)b * Ho * Wo);
        const int i0 = rem / Wo, j0 = rem - i0 * Wo;
        const int tap = k / CIN, c = k - tap * CIN;
        const int u = tap / 3, vv = tap - u * 3;
        v = x[(((int64_t)b * H + i0 + u * d) * W + j0 + vv * d) * CIN + c];
      }
      xs[pp][k] = v;
    }
    __syncthreads();
    for (int pp = 0; pp < kSub; ++pp) {
      const float g = dzs[pp][o];
#pragma unroll
      for (int j = 0; j < PER; ++j)
        if (k0 + j < KW) acc[j] = fmaf(g, __bfloat162float(xs[pp][k0 + j]), acc[j]);
      accb += g;
    }
  }
  constexpr int E = kHid * KW + kHid;
  float* part = partials + (int64_t)blockIdx.x * E;
#pragma unroll
  for (int j = 0; j < PER; ++j)
    if (k0 + j < KW) part[o * KW + k0 + j] = acc[j];
  if ((threadIdx.x & 7) == 0) part[kHid * KW + o] = accb;
}

// Sums per-chunk partials in chunk order (deterministic): out[e] = sum_k partials[k][e].
__global__ void reduce_partials_kernel(const float* __restrict__ partials, int chunks, int E, float* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < chunks; ++k) s += partials[(int64_t)k * E + e];
    out[e] = s;
  }
}

// Adam (D. P. Kingma, J. Ba, 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, bf16* __restrict__ pb, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

// He-normal initialisation of the convolution weights (std sqrt(2 / fan_in)), head weights with
// std sqrt(1 / fan_in), zero biases and Adam moments.
__global__ void init_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, bf16* __restrict__ pb,
                            ParamLayout L, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    float val = 0.f;
    for (int l = 0; l < 4; ++l)
      if (i >= L.w[l] && i < L.b[l]) val = gauss(seed, (uint64_t)i) * sqrtf(2.f / (9.f * (l == 0 ? kInF : kHid)));
    if (i >= L.wh && i < L.bh) val = gauss(seed, (uint64_t)i) * sqrtf(1.f / kHid);
    p[i] = val;
    m[i] = 0.f;
    v[i] = 0.f;
    pb[i] = __float2bfloat16_rn(val);
  }
}

// ------------------------------------------------------------------------------------------------
// Tensor-core convolution (tcgen05, sm_100 family): the 32 -> 32 dilated 3x3 layers as implicit
// GEMMs D[128 pixels][32] = A[128][288] B[288][32] (K = 9 taps x 32 channels), both operands BF16
// and K-major in shared memory in the canonical layout without swizzle (core matrices of 8 rows x
// 16 bytes; K-adjacent core matrices LBO bytes apart, M/N-adjacent ones SBO bytes apart), FP32
// accumulation in tensor memory.
// ------------------------------------------------------------------------------------------------
constexpr int kTcM = 128;
constexpr int kTcK = 9 * kHid;                      // 288
constexpr int kTcKCores = kTcK / 8;                  // 36

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family; swizzle none, base offset 0
  return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = 32.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

// Byte offset of element (row, k) of a K-major operand with nrow_cores core rows:
// layout [k_core][row_core][8 rows][8 elements].
__device__ __forceinline__ uint32_t tc_off(int row, int k, int nrow_cores) {
  return (uint32_t)((((k >> 3) * nrow_cores + (row >> 3)) * 128) + (row & 7) * 16 + (k & 7) * 2);
}

// ------------------------------------------------------------------------------------------------
// Tensor-core backward of the 32 -> 32 layers (tcgen05, the same operand layout and instruction
// descriptor as the forward: BF16, K-major, no swizzle, M = 128, N = 32, FP32 in tensor memory).
// The FP32 gradient dz = dy * (y > 0) enters as two BF16 operands, hi = bf16(dz) and
// lo = bf16(dz - hi), multiplied by the same BF16 weights or activations and accumulated in FP32:
// every product is exact and hi + lo carries dz to about 2^-17, so the tensor-core gradients
// track the FP32 CUDA-core ones.
// ------------------------------------------------------------------------------------------------
struct TcSync {  // one-thread MMA issue, commit and a bounded wait
  uint64_t* bar;
  __device__ void issue(uint32_t tmem_d, uint32_t a0, uint32_t a_lbo, uint32_t b0, uint32_t b_lbo, int ksteps,
                        bool acc_first) const {
    for (int s = 0; s < ksteps; ++s) {
      const uint64_t ad = tc_desc(a0 + s * 2 * a_lbo, a_lbo, 128);
      const uint64_t bd = tc_desc(b0 + s * 2 * b_lbo, b_lbo, 128);
      const uint32_t acc = (s > 0 || acc_first) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tmem_d),
          "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc));
    }
  }
  __device__ void commit() const {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  }
  __device__ bool wait(uint32_t parity) const {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; ++it)
      asm volatile(
          "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n selp.u32 %0, 1, 0, pw;\n}"
          : "=r"(done)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return done != 0;
  }
};

__device__ __forceinline__ uint32_t tmem_alloc_cols(uint32_t* slot, int warp, uint32_t cols) {
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *slot;
}

__device__ __forceinline__ void tmem_free_cols(uint32_t tmem, int warp, uint32_t cols) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 8 BF16 values -> one 16-byte core-matrix row.
__device__ __forceinline__ uint4 pack8(const float v[8]) {
  uint4 o;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
  for (int t = 0; t < 4; ++t) h[t] = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
  return o;
}

// ------------------------------------------------------------------------------------------------
// Tensor-core forward of the 32 -> 32 layers as an implicit GEMM over a 2-D tile of R x C output
// pixels of one image.  The tile's input window, R + 2d rows of Pt = C + 2d pixels (zero outside
// the image), is staged once, as 4 channel groups of [pixel][8 channels] rows of 16 bytes.  Output
// pixel (r, c) of the tile is GEMM row m = r Pt + c (rows with c >= C are computed and dropped),
// and tap (u, v) reads staged pixel m + u d Pt + v d: the A operand of a tap is the staged window
// itself, started that many rows later, so only the descriptor's start address changes from tap
// to tap (16 bytes per pixel) and no pixel is copied per tap.  K-adjacent core matrices are the
// next channel group (LBO = S x 16 bytes), M-adjacent ones the next 8 pixels (SBO = 128).  Up to 4
// M tiles of 128 rows accumulate in 4 x 32 TMEM columns.
// ------------------------------------------------------------------------------------------------
struct ConvTile {
  int C, R, Pt, mt, S;  // tile columns and rows, window pitch (C + 2d), M tiles, group stride in pixels
                        // (Pt (R + 2d) rounded up to 8: each group's window starts 128-byte aligned)
};
constexpr int kCtMaxS = 1328;                       // staged pixels: 4 x 16 bytes each (83 KB)
constexpr int kCtBOff = kCtMaxS * 64;               // weights (32 x 288 BF16) after the window
constexpr int kCtBarOff = kCtBOff + 18 * 1024;
constexpr int kCtSmem = kCtBarOff + 64;             // + barrier and TMEM slot: two CTAs per SM
static_assert(kCtBOff % 1024 == 0, "weights 1 KB aligned");

// Window staging: with a tensor map (use_map), four TMA boxes {8 channels, Pt columns, R + 2d rows,
// 1 image}, one per channel group, land in exactly the [group][pixel][16 bytes] layout above, zero
// outside the image; otherwise 16-byte cp.async copies build the same layout.
template <bool RELU>
__global__ void __launch_bounds__(kTcM, 2) conv_tc_tile_kernel(const __grid_constant__ CUtensorMap xmap, int use_map,
                                                               const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                               const float* __restrict__ bias, int H, int W, int d,
                                                               ConvTile T, int tiles_x, int tiles_y,
                                                               bf16* __restrict__ y, uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint8_t* As = tsm;
  uint8_t* Bs = tsm + kCtBOff;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tsm + kCtBarOff);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + kCtBarOff + 16);
  uint64_t* tbar = reinterpret_cast<uint64_t*>(tsm + kCtBarOff + 32);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  if (blockDim.x != kTcM || T.S > kCtMaxS || T.mt < 1 || T.mt > 4) {
    if (tid == 0) atomicOr(err, 4u);
    return;
  }
  int t = blockIdx.x;
  const int tx = t % tiles_x;
  t /= tiles_x;
  const int ty = t % tiles_y, b = t / tiles_y;
  const int i0 = ty * T.R, j0 = tx * T.C;

  auto cp16 = [](uint8_t* dst, const void* src, uint32_t bytes) {  // bytes 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
  };
  if (use_map && tid == 0) {
    seb::mbar_init(tbar, 1);
    seb::mbar_arrive_expect_tx(tbar, (uint32_t)(T.Pt * (T.R + 2 * d)) * 64u);
    for (int g = 0; g < 4; ++g) seb::tma_load_4d(As + (size_t)g * T.S * 16, &xmap, 8 * g, j0, i0, b, tbar);
  }
  // B: weights [co][tap][ci] -> K-major rows co, k = tap * 32 + ci
  for (int i = tid; i < kHid * kTcKCores; i += kTcM) {
    const int co = i / kTcKCores, kc = i - co * kTcKCores;
    cp16(Bs + tc_off(co, kc * 8, kHid / 8), w + (int64_t)co * kTcK + kc * 8, 16u);
  }
  if (!use_map) {
    // A: window pixel s = rr * Pt + cc, channel group g at (g * S + s) * 16 bytes; four
    // consecutive threads copy one pixel's 64 bytes
    for (int e = tid; e < T.S * 4; e += kTcM) {
      const int s = e >> 2, g = e & 3;
      const int rr = s / T.Pt, cc = s - rr * T.Pt;
      const int gi = i0 + rr, gj = j0 + cc;
      const bool in = gi < H && gj < W;
      const bf16* src = in ? x + (((int64_t)b * H + gi) * W + gj) * kHid + g * 8 : x;
      cp16(As + ((size_t)g * T.S + s) * 16, src, in ? 16u : 0u);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor core
  const uint32_t tmem = tmem_alloc_cols(tslot, warp, 128);    // (its barrier publishes the copies)
  const TcSync sync{mbar};
  // the window's TMA box has landed (bounded wait by the thread that issues the MMAs)
  bool staged = true;
  if (use_map && tid == 0) {
    staged = seb::mbar_wait_bounded(tbar, 0, 1 << 20);
    if (!staged) {
      atomicOr(err, 4u);
      seb::mbar_wait_bounded(tbar, 0, 1 << 20);
    }
  }
  if (tid == 0 && staged) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    const uint32_t a_lbo = (uint32_t)T.S * 16u, b_lbo = (kHid / 8) * 128;
    for (int m = 0; m < T.mt; ++m) {
      for (int s = 0; s < kTcK / 16; ++s) {
        const int tap = s >> 1, u = tap / 3, v = tap - 3 * (tap / 3);
        const uint32_t row = (uint32_t)(m * kTcM + u * d * T.Pt + v * d);
        const uint64_t ad = tc_desc(a0 + (uint32_t)(s & 1) * 2u * a_lbo + row * 16u, a_lbo, 128);
        const uint64_t bd = tc_desc(b0 + s * 2 * b_lbo, b_lbo, 128);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tmem + (uint32_t)(m * kHid)),
            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc));
      }
    }
  }
  if (tid == 0) sync.commit();  // (with no MMA issued, the commit still completes the phase)
  const bool mma_done = sync.wait(0);
  if (!__syncthreads_and(mma_done && staged)) {
    // the copy or the MMAs did not finish in time: report it, give the MMAs one more bounded
    // wait (they write this CTA's tensor memory) and leave the tile unwritten
    if (tid == 0) {
      atomicOr(err, 4u);
      sync.wait(0);
    }
  } else {
    for (int m = 0; m < T.mt; ++m) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * kHid), r);
      const int row = m * kTcM + tid, rr = row / T.Pt, cc = row - rr * T.Pt;
      const int gi = i0 + rr, gj = j0 + cc;
      if (rr < T.R && cc < T.C && gi < Ho && gj < Wo) {
        // 16-byte stores: the 32 outputs of a pixel are 64 contiguous bytes
        uint4* yp = reinterpret_cast<uint4*>(y + (((int64_t)b * Ho + gi) * Wo + gj) * kHid);
#pragma unroll
        for (int q = 0; q < kHid / 8; ++q) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float a = __uint_as_float(r[8 * q + e]) + bias[8 * q + e];
            v[e] = RELU ? fmaxf(a, 0.f) : a;
          }
          yp[q] = pack8(v);
        }
      }
    }
  }
  tmem_free_cols(tmem, warp, 128);
}

// dz = dy * (y > 0) split into BF16 hi = bf16(dz) and lo = bf16(dz - hi), written over dy in
// place: pixel p's 128 bytes become [hi 0..31 | lo 0..31].  One thread per pixel.
__global__ void split_dz_kernel(float* __restrict__ dy, const bf16* __restrict__ y, int64_t P) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float g[kHid];
  const float4* d4 = reinterpret_cast<const float4*>(dy + p * kHid);
  const uint4* y4 = reinterpret_cast<const uint4*>(y + p * kHid);
#pragma unroll
  for (int q = 0; q < kHid / 8; ++q) {
    const float4 a = d4[2 * q], b = d4[2 * q + 1];
    const uint4 yv = y4[q];
    const __nv_bfloat162* y2 = reinterpret_cast<const __nv_bfloat162*>(&yv);
    const float gg[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float ye = e & 1 ? __high2float(y2[e >> 1]) : __low2float(y2[e >> 1]);
      g[8 * q + e] = ye > 0.f ? gg[e] : 0.f;
    }
  }
  uint4* o4 = reinterpret_cast<uint4*>(dy + p * kHid);
#pragma unroll
  for (int q = 0; q < kHid / 8; ++q) {
    float hi[8], lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hi[e] = __bfloat162float(__float2bfloat16_rn(g[8 * q + e]));
      lo[e] = g[8 * q + e] - hi[e];
    }
    o4[q] = pack8(hi);
    o4[kHid / 8 + q] = pack8(lo);
  }
}

// wt[c][tap][o] = w[o][tap][c] (the dgrad operand B in K-major order), one thread per element.
__global__ void transpose_w_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kHid * kTcK) return;
  const int c = i / kTcK, k = i - c * kTcK, tap = k >> 5, o = k & 31;
  wt[i] = w[((int64_t)o * 9 + tap) * kHid + c];
}

// Input side: dx[p][c] = sum_{tap, o} dz[p - tap offset][o] w[o][tap][c] as the implicit GEMM
// D[128 input pixels][32 c] = A[128][288] B[288][32], A the rows (tap, o) of dz (0 outside the
// output), B[k = tap * 32 + o][c] = w[o][tap][c]; once with dz's hi part, then accumulated with
// its lo part.  Writes dx FP32 [B][H][W][32].  Over 2-D tiles, the forward's scheme run
// backwards: dx at input pixel (i, j) sums dz[i - u d][j - v d] over the taps, so a tile of R x C input pixels stages the dz window of rows
// i0 - 2d .. i0 + R - 1 and columns j0 - 2d .. j0 + C - 1 (zero outside the layer's output), and
// tap (u, v) of GEMM row m = r Pt + c reads staged pixel m + (2 - u) d Pt + (2 - v) d.  The window
// is staged twice, the hi then the lo half of the split gradient, into the same shared memory;
// the lo MMAs accumulate onto the hi ones.
__global__ void __launch_bounds__(kTcM, 2) conv_bwd_dx_tile_kernel(const __grid_constant__ CUtensorMap zmap,
                                                                   int use_map, const bf16* __restrict__ dzs,
                                                                   const bf16* __restrict__ wt, int H, int W, int d,
                                                                   ConvTile T, int tiles_x, int tiles_y,
                                                                   float* __restrict__ dx, uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint8_t* As = tsm;
  uint8_t* Bs = tsm + kCtBOff;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tsm + kCtBarOff);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + kCtBarOff + 16);
  uint64_t* tbar = reinterpret_cast<uint64_t*>(tsm + kCtBarOff + 32);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  if (blockDim.x != kTcM || T.S > kCtMaxS || T.mt < 1 || T.mt > 4) {
    if (tid == 0) atomicOr(err, 8u);
    return;
  }
  int t = blockIdx.x;
  const int tx = t % tiles_x;
  t /= tiles_x;
  const int ty = t % tiles_y, b = t / tiles_y;
  const int i0 = ty * T.R, j0 = tx * T.C;
  // B: K-major rows c, k = tap * 32 + o; wt holds w transposed to [c][tap][o] (transpose_w_kernel)
  for (int i = tid; i < kHid * kTcKCores; i += kTcM) {
    const int c = i / kTcKCores, kc = i - c * kTcKCores;
    *reinterpret_cast<uint4*>(Bs + tc_off(c, kc * 8, kHid / 8)) =
        reinterpret_cast<const uint4*>(wt + (int64_t)c * kTcK)[kc];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    if (use_map) seb::mbar_init(tbar, 1);
  }
  const uint32_t tmem = tmem_alloc_cols(tslot, warp, 128);
  const TcSync sync{mbar};
  bool ok = true;
  for (int part = 0; part < 2 && ok; ++part) {  // 0: hi, 1: lo
    if (use_map) {
      // four TMA boxes of the window (channel groups of the hi or the lo half of the split
      // gradient), waited for by the thread that issues the MMAs
      if (tid == 0) {
        seb::mbar_arrive_expect_tx(tbar, (uint32_t)(T.Pt * (T.R + 2 * d)) * 64u);
        for (int g = 0; g < 4; ++g)
          seb::tma_load_4d(As + (size_t)g * T.S * 16, &zmap, kHid * part + 8 * g, j0 - 2 * d, i0 - 2 * d, b, tbar);
        if (!seb::mbar_wait_bounded(tbar, (uint32_t)part, 1 << 20)) {
          atomicOr(err, 8u);
          seb::mbar_wait_bounded(tbar, (uint32_t)part, 1 << 20);
          ok = false;
        }
      }
      ok = __syncthreads_and(ok) != 0;
      if (!ok) break;
    } else {
      for (int e = tid; e < T.S * 4; e += kTcM) {
        const int s = e >> 2, g = e & 3;
        const int rr = s / T.Pt, cc = s - rr * T.Pt;
        const int gi = i0 - 2 * d + rr, gj = j0 - 2 * d + cc;
        const bool in = gi >= 0 && gi < Ho && gj >= 0 && gj < Wo;
        const bf16* src = in ? dzs + (((int64_t)b * Ho + gi) * Wo + gj) * 2 * kHid + part * kHid + g * 8 : dzs;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(As + ((size_t)g * T.S + s) * 16)),
                     "l"(src), "r"(in ? 16u : 0u)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const uint32_t a_lbo = (uint32_t)T.S * 16u, b_lbo = (kHid / 8) * 128;
      for (int m = 0; m < T.mt; ++m) {
        for (int s = 0; s < kTcK / 16; ++s) {
          const int tap = s >> 1, u = tap / 3, v = tap - 3 * (tap / 3);
          const uint32_t row = (uint32_t)(m * kTcM + (2 - u) * d * T.Pt + (2 - v) * d);
          const uint64_t ad = tc_desc(a0 + (uint32_t)(s & 1) * 2u * a_lbo + row * 16u, a_lbo, 128);
          const uint64_t bd = tc_desc(b0 + s * 2 * b_lbo, b_lbo, 128);
          const uint32_t acc = (s > 0 || part > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tmem + (uint32_t)(m * kHid)),
              "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc));
        }
      }
      sync.commit();
    }
    ok = sync.wait((uint32_t)part);
    ok = __syncthreads_and(ok) != 0;  // the next part overwrites the window only after the MMAs read it
  }
  if (!ok) {  // report, give the MMAs in flight one more bounded wait, then free the columns
    if (tid == 0) atomicOr(err, 8u);
    sync.wait(0);
    sync.wait(1);
  } else {
    for (int m = 0; m < T.mt; ++m) {
      uint32_t rr[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * kHid), rr);
      const int row = m * kTcM + tid, r = row / T.Pt, c = row - r * T.Pt;
      const int gi = i0 + r, gj = j0 + c;
      if (r < T.R && c < T.C && gi < H && gj < W) {
        float4* o4 = reinterpret_cast<float4*>(dx + (((int64_t)b * H + gi) * W + gj) * kHid);
#pragma unroll
        for (int q = 0; q < kHid / 4; ++q)
          o4[q] = make_float4(__uint_as_float(rr[4 * q]), __uint_as_float(rr[4 * q + 1]), __uint_as_float(rr[4 * q + 2]),
                              __uint_as_float(rr[4 * q + 3]));
      }
    }
  }
  tmem_free_cols(tmem, warp, 128);
}

// Weight side: dw[o][tap][c] = sum_p dz[p][o] x[p + tap offset][c] and db[o] = sum_p dz[p][o] as
// D[m][o] = sum_k A[m][k] B[o][k] over the CTA's output pixels k (kChunkPx, 128 per round):
// A rows m = tap * 32 + c (three M = 128 tiles; row 288 is all ones, so its D row is db; the rest
// of the third tile is zero), B rows o = dz hi, then dz lo.  One partial [o][tap][c] + [o] per CTA,
// in the layout of conv_bwd_dw_kernel, summed in CTA order by reduce_partials_kernel.
constexpr int kBwTile = kTcM * kTcM * 2;          // one A tile: 128 rows x 128 pixels BF16 (32 KB)
constexpr int kBwBOff = 3 * kBwTile;              // B hi, then B lo: 32 rows x 128 pixels each (8 KB)
constexpr int kBwBarOff = kBwBOff + 2 * kHid * kTcM * 2;
constexpr int kBwSmem = kBwBarOff + 64;  // + barrier and TMEM slot: two CTAs per SM

__global__ void __launch_bounds__(kTcM, 2) conv_bwd_dw_tc_kernel(const bf16* __restrict__ dzs,
                                                                 const bf16* __restrict__ x, int B, int H, int W, int d,
                                                                 float* __restrict__ partials, uint32_t* err) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint8_t* Bh = tsm + kBwBOff;
  uint8_t* Bl = Bh + kHid * kTcM * 2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tsm + kBwBarOff);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + kBwBarOff + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Ho = H - 2 * d, Wo = W - 2 * d;
  const int64_t P = (int64_t)B * Ho * Wo;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
  const uint32_t tmem = tmem_alloc_cols(tslot, warp, 128);  // three 32-column accumulators
  const TcSync sync{mbar};
  bool ok = true;
  const int64_t p0 = (int64_t)blockIdx.x * kChunkPx;
  int round = 0;
  for (int64_t q0 = p0; q0 < p0 + kChunkPx && q0 < P && ok; q0 += kTcM, ++round) {
    // Thread tid stages pixel k = tid of this round: column k of every operand row.  A rows
    // m = tap * 32 + c take x at the pixel's tap offset (16-byte loads of the 32 channels); the
    // ones row 288 is 1 for a pixel of the layer, 0 past the last one; rows 289..383 stay 0.
    // B rows o take dz hi and lo (16-byte loads of the pixel's 32 gradients and activations).
    {
      const int64_t p = q0 + tid;
      const bool valid = p < P;
      int64_t base = 0;
      if (valid) {
        const int b = (int)(p / ((int64_t)Ho * Wo));
        const int rem = (int)(p - (int64_t)b * Ho * Wo);
        const int i = rem / Wo, j = rem - i * Wo;
        base = (((int64_t)b * H + i) * W + j) * kHid;
      }
      bf16* sh = reinterpret_cast<bf16*>(tsm);
      auto a_at = [&](int m) -> bf16& {  // element (m, k = tid) of the three stacked A tiles
        return sh[((m >> 7) * kBwTile + tc_off(m & 127, tid, kTcM / 8)) / 2];
      };
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int u = tap / 3, v = tap - u * 3;
        const uint4* src = reinterpret_cast<const uint4*>(x + base + ((int64_t)u * d * W + v * d) * kHid);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint4 w8 = make_uint4(0u, 0u, 0u, 0u);
          if (valid) w8 = src[q];
          const bf16* e8 = reinterpret_cast<const bf16*>(&w8);
#pragma unroll
          for (int e = 0; e < 8; ++e) a_at(tap * kHid + q * 8 + e) = e8[e];
        }
      }
      a_at(9 * kHid) = __float2bfloat16_rn(valid ? 1.f : 0.f);
      if (round == 0)
        for (int m = 9 * kHid + 1; m < 3 * kTcM; ++m) a_at(m) = __float2bfloat16_rn(0.f);
      bf16* bh = reinterpret_cast<bf16*>(Bh);
      bf16* bl = reinterpret_cast<bf16*>(Bl);
#pragma unroll
      for (int q = 0; q < 8; ++q) {  // hi: q < 4, lo: q >= 4
        uint4 w8 = make_uint4(0u, 0u, 0u, 0u);
        if (valid) w8 = reinterpret_cast<const uint4*>(dzs + p * 2 * kHid)[q];
        const bf16* e8 = reinterpret_cast<const bf16*>(&w8);
        bf16* dst = q < 4 ? bh : bl;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[tc_off((q & 3) * 8 + e, tid, kHid / 8) / 2] = e8[e];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a_lbo = (kTcM / 8) * 128, b_lbo = (kHid / 8) * 128;
      for (int t = 0; t < 3; ++t) {
        const uint32_t a0 = smem_u32(tsm + t * kBwTile);
        sync.issue(tmem + 32 * t, a0, a_lbo, smem_u32(Bh), b_lbo, kTcM / 16, round > 0);
        sync.issue(tmem + 32 * t, a0, a_lbo, smem_u32(Bl), b_lbo, kTcM / 16, true);
      }
      sync.commit();
    }
    ok = sync.wait((uint32_t)(round & 1));
    ok = __syncthreads_and(ok) != 0;  // the next round overwrites A and B only after the MMAs read them
  }
  if (!ok) {  // report, give the MMAs in flight one more bounded wait, then free the columns
    if (tid == 0) atomicOr(err, 8u);
    sync.wait((uint32_t)((round - 1) & 1));
  } else if (round > 0) {
    constexpr int E = kHid * 9 * kHid + kHid;
    float* part = partials + (int64_t)blockIdx.x * E;
    for (int t = 0; t < 3; ++t) {
      uint32_t rr[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * t, rr);
      const int m = t * kTcM + warp * 32 + (tid & 31);
      if (m < 9 * kHid) {
        for (int o = 0; o < kHid; ++o) part[o * 9 * kHid + m] = __uint_as_float(rr[o]);
      } else if (m == 9 * kHid) {
        for (int o = 0; o < kHid; ++o) part[kHid * 9 * kHid + o] = __uint_as_float(rr[o]);
      }
    }
  }
  tmem_free_cols(tmem, warp, 128);
}

// ------------------------------------------------------------------------------------------------
// Inference over a map.
// ------------------------------------------------------------------------------------------------
// act [H4][W4][32] covers cells (r, c) = (i + 16, j + 16); writes out[5][K][ny][nx] and flags for
// those cells: z = elev + pred0 / 10, pitch, roll (negated for k + n_pairs), roughness NaN
// (not predicted), risk clamped to [0, 1]; flags SURROGATE (+ OBSTACLE when risk reaches 1).
__global__ void __launch_bounds__(128) map_head_kernel(const bf16* __restrict__ a, const bf16* __restrict__ wh,
                                                       const float* __restrict__ bh, const float* __restrict__ elev,
                                                       int nx, int ny, int n_yaw, float* __restrict__ out,
                                                       uint8_t* __restrict__ flags) {
  // one thread per cell: its 32 activations once in registers, all 4 x n_pairs outputs
  extern __shared__ float hw[];  // [nout][kHid] weights, then [nout] biases
  const int npairs = n_yaw / 2, nout = 4 * npairs;
  for (int i = threadIdx.x; i < nout * kHid; i += blockDim.x) hw[i] = __bfloat162float(wh[i]);
  for (int i = threadIdx.x; i < nout; i += blockDim.x) hw[nout * kHid + i] = bh[i];
  __syncthreads();
  const int W4 = nx - 2 * kMargin, H4 = ny - 2 * kMargin;
  const int64_t plane = (int64_t)nx * ny, chs = plane * n_yaw;
  const float qnan = __int_as_float(0x7fc00000);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (int64_t)W4 * H4;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / W4), j = (int)(p - (int64_t)i * W4);
    const int64_t cell = (int64_t)(i + kMargin) * nx + j + kMargin;
    float av[kHid];
    const uint4* ap = reinterpret_cast<const uint4*>(a + p * kHid);
#pragma unroll
    for (int q = 0; q < kHid / 8; ++q) {
      const uint4 v = ap[q];
      const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 f = __bfloat1622float2(h2[t]);
        av[8 * q + 2 * t] = f.x;
        av[8 * q + 2 * t + 1] = f.y;
      }
    }
    const float ez = elev[cell];
    for (int k = 0; k < npairs; ++k) {
      float qv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float* w = hw + (4 * k + t) * kHid;
        float s = hw[nout * kHid + 4 * k + t];
#pragma unroll
        for (int c = 0; c < kHid; ++c) s = fmaf(w[c], av[c], s);
        qv[t] = s;
      }
      const float z = ez + qv[0] / kZScale;
      const float risk = fminf(fmaxf(qv[3], 0.f), 1.f);
      const uint8_t f = (uint8_t)(SEB_FLAG_SURROGATE | (risk >= 1.f ? SEB_FLAG_OBSTACLE : 0));
      const int64_t i0 = (int64_t)k * plane + cell, i1 = (int64_t)(k + npairs) * plane + cell;
      out[i0] = z;
      out[i1] = z;
      out[chs + i0] = qv[1];
      out[chs + i1] = -qv[1];
      out[2 * chs + i0] = qv[2];
      out[2 * chs + i1] = -qv[2];
      out[3 * chs + i0] = qnan;
      out[3 * chs + i1] = qnan;
      out[4 * chs + i0] = risk;
      out[4 * chs + i1] = risk;
      flags[i0] = f;
      flags[i1] = f;
    }
  }
}

// Fallback mask: a cell goes to the exact kernel when an unknown cell or a step edge (a
// 4-neighbour height jump above step) lies within Chebyshev distance radius, or when it is
// within the network's margin of the map edge.  tile_active[t] marks 32 x 32 tiles holding
// such a cell.
__global__ void mask_kernel(const float* __restrict__ elev, int nx, int ny, float step, int radius,
                            uint8_t* __restrict__ mask, uint8_t* __restrict__ tile_active, int tiles_x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)nx * ny;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (int64_t)r * nx);
    bool m = r < kMargin || c < kMargin || r >= ny - kMargin || c >= nx - kMargin;
    for (int dr = -radius; dr <= radius && !m; ++dr)
      for (int dc = -radius; dc <= radius && !m; ++dc) {
        const int rr = r + dr, cc = c + dc;
        if (rr < 0 || cc < 0 || rr >= ny || cc >= nx) continue;
        const float z = elev[(int64_t)rr * nx + cc];
        if (z != z) {
          m = true;
          break;
        }
        if (cc + 1 < nx) {
          const float zr = elev[(int64_t)rr * nx + cc + 1];
          if (zr == zr && fabsf(zr - z) > step) m = true;
        }
        if (rr + 1 < ny) {
          const float zd = elev[(int64_t)(rr + 1) * nx + cc];
          if (zd == zd && fabsf(zd - z) > step) m = true;
        }
      }
    mask[i] = m ? 1 : 0;
    if (m) tile_active[(r / 32) * tiles_x + c / 32] = 1;
  }
}

// The same mask by 32 x 32 tiles (radius <= kMaskMaxR): per cell of the tile and its halo the
// source flag (unknown, or a step to the right or below), then the Chebyshev dilation as a
// row pass and a column pass in shared memory.
constexpr int kMaskTile = 32, kMaskMaxR = 8, kMaskExt = kMaskTile + 2 * kMaskMaxR;
__global__ void __launch_bounds__(256) mask_tiled_kernel(const float* __restrict__ elev, int nx, int ny, float step,
                                                         int radius, uint8_t* __restrict__ mask,
                                                         uint8_t* __restrict__ tile_active, int tiles_x) {
  __shared__ uint8_t src[kMaskExt][kMaskExt];
  __shared__ uint8_t hor[kMaskExt][kMaskTile];
  __shared__ int any;
  const int R = radius, E = kMaskTile + 2 * R;
  const int r0 = blockIdx.y * kMaskTile, c0 = blockIdx.x * kMaskTile;
  if (threadIdx.x == 0) any = 0;
  for (int t = threadIdx.x; t < E * E; t += blockDim.x) {
    const int i = t / E, j = t - i * E;
    const int rr = r0 - R + i, cc = c0 - R + j;
    uint8_t f = 0;
    if (rr >= 0 && rr < ny && cc >= 0 && cc < nx) {
      const float z = elev[(int64_t)rr * nx + cc];
      if (z != z) {
        f = 1;
      } else {
        if (cc + 1 < nx) {
          const float zr = elev[(int64_t)rr * nx + cc + 1];
          if (zr == zr && fabsf(zr - z) > step) f = 1;
        }
        if (rr + 1 < ny) {
          const float zd = elev[(int64_t)(rr + 1) * nx + cc];
          if (zd == zd && fabsf(zd - z) > step) f = 1;
        }
      }
    }
    src[i][j] = f;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < E * kMaskTile; t += blockDim.x) {
    const int i = t / kMaskTile, j = t - i * kMaskTile;
    uint8_t h = 0;
    for (int k = 0; k <= 2 * R; ++k) h |= src[i][j + k];
    hor[i][j] = h;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kMaskTile * kMaskTile; t += blockDim.x) {
    const int i = t / kMaskTile, j = t - i * kMaskTile;
    const int r = r0 + i, c = c0 + j;
    if (r >= ny || c >= nx) continue;
    uint8_t m = r < kMargin || c < kMargin || r >= ny - kMargin || c >= nx - kMargin;
    for (int k = 0; k <= 2 * R; ++k) m |= hor[i + k][j];
    mask[(int64_t)r * nx + c] = m;
    if (m) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && any) tile_active[blockIdx.y * tiles_x + blockIdx.x] = 1;
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------------
struct seb_sur {
  seb_params p;
  seb::Tables T;
  int32_t nout, max_batch, chunks_max;
  ParamLayout PL;
  uint8_t* ws;
  size_t bytes;
  cudaStream_t stream;
  // offsets into ws
  seb_sur_view v;
  uint32_t* err;
  int32_t engine;  // SEB_SUR_SIMT | SEB_SUR_TCGEN05 for the 32 -> 32 layers
  int64_t step;    // Adam step of the last seb_sur_train_step (0 after init)
};

namespace {

struct Sizes {
  size_t ctl, master, m, v, grad, wbf, feat, lab, act[4], pred, dpred, dact[4], partials, loss, tot;
  size_t mfeat, mact[4], mask, tiles, total;
};

int chunks_for(int64_t pixels, int chunk) { return (int)((pixels + chunk - 1) / chunk); }

Sizes sizes(const seb_params& p, int nout, int B) {
  Sizes s;
  const ParamLayout PL = param_layout(nout);
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += al(n);
    return at;
  };
  s.ctl = take(256);
  s.master = take(PL.n * 4);
  s.m = take(PL.n * 4);
  s.v = take(PL.n * 4);
  s.grad = take(PL.n * 4);
  s.wbf = take(PL.n * 2);
  s.feat = take((size_t)B * kFeat * kFeat * kInF * 2);
  s.lab = take((size_t)B * kOutSide * kOutSide * nout * 4);
  for (int l = 0; l < 4; ++l) s.act[l] = take((size_t)B * kSide[l + 1] * kSide[l + 1] * kHid * 2);
  s.pred = take((size_t)B * kOutSide * kOutSide * nout * 4);
  s.dpred = take((size_t)B * kOutSide * kOutSide * nout * 4);
  for (int l = 0; l < 4; ++l) s.dact[l] = take((size_t)B * kSide[l + 1] * kSide[l + 1] * kHid * 4);
  const int64_t max_pix = (int64_t)B * kSide[1] * kSide[1];
  const int64_t E = (int64_t)kHid * 9 * kHid + kHid > (int64_t)nout * kHid + nout ? (int64_t)kHid * 9 * kHid + kHid
                                                                                  : (int64_t)nout * kHid + nout;
  s.partials = take((size_t)chunks_for(max_pix, kChunkPx) * E * 4);
  s.loss = take(2 * 4 * 4096);
  s.tot = take(4 * 4);
  const int W = p.nx - 2, H = p.ny - 2;
  s.mfeat = take((size_t)(W > 0 ? W : 0) * (H > 0 ? H : 0) * kInF * 2);
  int w = W, h = H;
  for (int l = 0; l < 4; ++l) {
    w -= 2 * kDil[l];
    h -= 2 * kDil[l];
    s.mact[l] = take((size_t)(w > 0 ? w : 0) * (h > 0 ? h : 0) * kHid * 2);
  }
  s.mask = take((size_t)p.nx * p.ny);
  s.tiles = take((size_t)((p.nx + 31) / 32) * ((p.ny + 31) / 32));
  s.total = o;
  return s;
}

int fail(const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  seb::set_error("%s", buf);
  return SEB_ERR_INVALID_ARG;
}

int cuda_check(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SEB_OK;
  seb::set_error("%s: %s", where, cudaGetErrorString(e));
  return SEB_ERR_CUDA;
}

template <typename T>
T* at(const seb_sur* h, size_t off) {
  return reinterpret_cast<T*>(h->ws + off);
}

}  // namespace

extern "C" {

size_t seb_sur_workspace_bytes(const seb_params* p, int32_t max_batch) {
  SEB_RANGE();
  if (!p || seb::validate_params(*p) != SEB_OK || max_batch < 1) return 0;
  return sizes(*p, 2 * p->n_yaw, max_batch).total;
}

int seb_sur_create(const seb_params* p, int32_t max_batch, void* ws, size_t bytes, seb_stream_t stream, seb_sur** out) {
  SEB_RANGE();
  if (!p || !out || max_batch < 1) return fail("seb_sur_create: NULL argument or batch < 1");
  *out = nullptr;
  int rc = seb::validate_params(*p);
  if (rc) return rc;
  if (p->nx < 2 * kMargin + 1 || p->ny < 2 * kMargin + 1) return fail("seb_sur_create: map smaller than 33 x 33");
  if (p->elev_dtype != SEB_F32) return fail("seb_sur_create: the surrogate reads FP32 elevation");
  if ((int64_t)max_batch * kFeat * kFeat * kHid >= ((int64_t)1 << 31))
    return fail("seb_sur_create: max_batch too large (activation offsets must stay below 2^31)");
  if (!ws || ((uintptr_t)ws & 255)) {
    seb::set_error("surrogate workspace NULL or not 256-byte aligned");
    return SEB_ERR_WORKSPACE;
  }
  const Sizes s = sizes(*p, 2 * p->n_yaw, max_batch);
  if (bytes < s.total) {
    seb::set_error("surrogate workspace too small (%zu < %zu)", bytes, s.total);
    return SEB_ERR_WORKSPACE;
  }
  seb_sur* h = new (std::nothrow) seb_sur;
  if (!h) return fail("out of host memory");
  memset(h, 0, sizeof(*h));
  h->p = *p;
  rc = seb::build_tables(*p, &h->T, nullptr);
  if (rc) {
    delete h;
    return rc;
  }
  h->nout = 2 * p->n_yaw;  // 4 outputs per yaw pair
  h->engine = SEB_SUR_TCGEN05;
  h->max_batch = max_batch;
  h->PL = param_layout(h->nout);
  h->ws = (uint8_t*)ws;
  h->bytes = bytes;
  h->stream = (cudaStream_t)stream;
  h->err = at<uint32_t>(h, s.ctl);
  seb_sur_view& v = h->v;
  v.n_params = h->PL.n;
  v.n_out = h->nout;
  v.max_batch = max_batch;
  v.master = s.master;
  v.adam_m = s.m;
  v.adam_v = s.v;
  v.grad = s.grad;
  v.weights_bf16 = s.wbf;
  v.features = s.feat;
  v.labels = s.lab;
  for (int l = 0; l < 4; ++l) {
    v.act[l] = s.act[l];
    v.dact[l] = s.dact[l];
    v.map_act[l] = s.mact[l];
  }
  v.pred = s.pred;
  v.dpred = s.dpred;
  v.map_features = s.mfeat;
  v.mask = s.mask;
  v.tiles = s.tiles;
  v.partials = s.partials;
  v.loss_partials = s.loss;
  v.totals = s.tot;
  for (int l = 0; l < 4; ++l) {
    v.off_w[l] = h->PL.w[l];
    v.off_b[l] = h->PL.b[l];
  }
  v.off_wh = h->PL.wh;
  v.off_bh = h->PL.bh;
  rc = cuda_check(cudaMemsetAsync(h->err, 0, 256, h->stream), "cudaMemsetAsync(surrogate control)");
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return SEB_OK;
}

int seb_sur_destroy(seb_sur* h) {
  SEB_RANGE();
  if (!h) return SEB_ERR_INVALID_ARG;
  delete h;
  return SEB_OK;
}

int seb_sur_set_stream(seb_sur* h, seb_stream_t s) {
  SEB_RANGE();
  if (!h) return fail("surrogate handle is NULL");
  h->stream = (cudaStream_t)s;
  return SEB_OK;
}

int seb_sur_set_engine(seb_sur* h, int32_t engine) {
  SEB_RANGE();
  if (!h || (engine != SEB_SUR_SIMT && engine != SEB_SUR_TCGEN05)) return fail("seb_sur_set_engine: bad engine");
  h->engine = engine;
  return SEB_OK;
}

int seb_sur_view_get(const seb_sur* h, seb_sur_view* v) {
  SEB_RANGE();
  if (!h || !v) return fail("surrogate handle or view is NULL");
  *v = h->v;
  return SEB_OK;
}

int seb_sur_init(seb_sur* h, uint64_t seed) {
  SEB_RANGE();
  if (!h) return fail("surrogate handle is NULL");
  h->step = 0;
  init_kernel<<<grid_for(h->PL.n, 256), 256, 0, h->stream>>>(at<float>(h, h->v.master), at<float>(h, h->v.adam_m),
                                                             at<float>(h, h->v.adam_v), at<bf16>(h, h->v.weights_bf16),
                                                             h->PL, seed);
  return cuda_check(cudaGetLastError(), "surrogate init");
}

int seb_terrain_bumpy(const float* params_dev, int32_t n, int32_t nx, int32_t ny, float res, uint64_t seed,
                      float* out_dev, seb_stream_t stream) {
  SEB_RANGE();
  if (!params_dev || !out_dev || n < 0 || nx < 1 || ny < 1 || !(res > 0.f)) return fail("seb_terrain_bumpy: bad args");
  if (n == 0) return SEB_OK;
  terrain_kernel<<<grid_for((int64_t)n * nx * ny, 256), 256, 0, (cudaStream_t)stream>>>(params_dev, n, nx, ny, res,
                                                                                        seed, out_dev);
  return cuda_check(cudaGetLastError(), "terrain launch");
}

int seb_sur_gather(seb_sur* h, const float* elev, const float* exact, int32_t nx, int32_t ny, const int32_t* centres,
                   int32_t n, int32_t offset) {
  SEB_RANGE();
  if (!h || !elev || !exact || !centres || n < 0 || offset < 0 || offset + n > h->max_batch)
    return fail("seb_sur_gather: bad args (offset + n must be <= max_batch)");
  if (n == 0) return SEB_OK;
  bf16* feat = at<bf16>(h, h->v.features) + (int64_t)offset * kFeat * kFeat * kInF;
  float* lab = at<float>(h, h->v.labels) + (int64_t)offset * kOutSide * kOutSide * h->nout;
  gather_kernel<<<n, 256, 0, h->stream>>>(elev, exact, nx, ny, h->p.n_yaw, centres, n, h->p.res, h->nout, feat, lab,
                                          h->err);
  return cuda_check(cudaGetLastError(), "gather launch");
}

// Tile of conv_tc_tile_kernel for dilation d and an Ho x Wo output: the column count C (a
// multiple of 8 up to 64, or all of Wo) and the row count R (up to 4 M tiles of 128 rows, the
// window within kCtMaxS pixels) that stage the fewest pixels for the whole output.
static ConvTile conv_tile(int d, int Ho, int Wo) {
  ConvTile best{0, 0, 0, 0, 0};
  double best_score = 1e300;
  for (int c = 8; c <= 64 + 7; c += 8) {
    const int C = c < Wo ? c : Wo;
    const int Pt = C + 2 * d;
    int R = (4 * kTcM) / Pt < Ho ? (4 * kTcM) / Pt : Ho;
    // window pixels per channel group, and one past the last pixel a GEMM row of the M tiles
    // reads (rows past the tile read on into the next group's window, or past the last one)
    auto win = [&](int r) { return (Pt * (r + 2 * d) + 7) / 8 * 8; };
    auto reach = [&](int r) { return (r * Pt + kTcM - 1) / kTcM * kTcM + 2 * d * Pt + 2 * d; };
    while (R > 0 && (win(R) > kCtMaxS || 3 * win(R) + reach(R) > 4 * kCtMaxS)) --R;
    if (R > 0) {
      const double score = (double)((Wo + C - 1) / C) * ((Ho + R - 1) / R) * win(R);
      if (score < best_score) {
        best_score = score;
        best = ConvTile{C, R, Pt, (R * Pt + kTcM - 1) / kTcM, win(R)};
      }
    }
    if (C == Wo) break;
  }
  return best;
}

// 4-D tensor map of a [B][H][W][chans] BF16 buffer whose box {8 channels, Pt columns, rows,
// 1 image} lands in shared memory as [pixel][16 bytes] (zero outside the image); the kernels load
// one box per channel group g (first coordinate 8 g) to build the [group][pixel][16 bytes] window.
// False (the kernels then stage with cp.async) when the driver's encoder is missing or the buffer
// or the box does not meet TMA's rules.
static bool window_map(CUtensorMap* m, const bf16* base, int B, int H, int W, int chans, int Pt, int rows) {
  memset(m, 0, sizeof(*m));
  PFN_cuTensorMapEncodeTiled_v12000 enc = seb::tensor_map_encoder();
  if (!enc || ((uintptr_t)base & 15) != 0 || Pt > 256 || rows > 256) return false;
  const cuuint64_t px = (cuuint64_t)chans * 2;  // bytes per pixel
  const cuuint64_t dims[4] = {(cuuint64_t)chans, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {px, px * W, px * W * H};
  const cuuint32_t box[4] = {8, (cuuint32_t)Pt, (cuuint32_t)rows, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One 3x3 layer l (0..3) on x [B][S][S'][Cin] -> y; the 32 -> 32 layers use the tensor-core
// kernel when the handle's engine says so.
static void conv_layer(seb_sur* h, const bf16* x, int l, int B, int H, int W, bf16* y) {
  const bf16* wb = at<bf16>(h, h->v.weights_bf16);
  const float* master = at<float>(h, h->v.master);
  const int64_t pix = (int64_t)B * (H - 2 * kDil[l]) * (W - 2 * kDil[l]);
  if (l == 0) {
    conv_fwd_kernel<kInF><<<grid_for(pix, 128), 128, 0, h->stream>>>(x, wb + h->PL.w[0], master + h->PL.b[0], B, H,
                                                                      W, kDil[0], y);
  } else if (h->engine == SEB_SUR_TCGEN05) {
    const int d = kDil[l], Ho = H - 2 * d, Wo = W - 2 * d;
    const ConvTile T = conv_tile(d, Ho, Wo);
    const int tx = (Wo + T.C - 1) / T.C, ty = (Ho + T.R - 1) / T.R;
    CUtensorMap xm;
    const int use_map = window_map(&xm, x, B, H, W, kHid, T.Pt, T.R + 2 * d) ? 1 : 0;
    cudaFuncSetAttribute(conv_tc_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCtSmem);
    conv_tc_tile_kernel<true><<<(unsigned)((int64_t)B * ty * tx), kTcM, kCtSmem, h->stream>>>(
        xm, use_map, x, wb + h->PL.w[l], master + h->PL.b[l], H, W, d, T, tx, ty, y, h->err);
  } else {
    conv_fwd_kernel<kHid><<<grid_for(pix, 128), 128, 0, h->stream>>>(x, wb + h->PL.w[l], master + h->PL.b[l], B, H,
                                                                      W, kDil[l], y);
  }
}

static int forward_batch(seb_sur* h, int B) {
  const bf16* wb = at<bf16>(h, h->v.weights_bf16);
  const float* master = at<float>(h, h->v.master);
  const bf16* x = at<bf16>(h, h->v.features);
  for (int l = 0; l < 4; ++l) {
    bf16* y = at<bf16>(h, h->v.act[l]);
    conv_layer(h, x, l, B, kSide[l], kSide[l], y);
    x = y;
  }
  const int64_t P = (int64_t)B * kOutSide * kOutSide;
  head_fwd_kernel<<<dim3(grid_for(P, 128), (h->nout + 15) / 16), 128, 0, h->stream>>>(
      x, wb + h->PL.wh, master + h->PL.bh, P, h->nout, at<float>(h, h->v.pred));
  return cuda_check(cudaGetLastError(), "surrogate forward");
}

int seb_sur_forward(seb_sur* h, int32_t batch) {
  SEB_RANGE();
  if (!h || batch < 1 || batch > h->max_batch) return fail("seb_sur_forward: batch out of range");
  return forward_batch(h, batch);
}

int seb_sur_train_step(seb_sur* h, int32_t B, float lr, int32_t step, float* loss_dev) {
  SEB_RANGE();
  if (!h || B < 1 || B > h->max_batch || step < 1) return fail("seb_sur_train_step: bad batch or step");
  int rc = forward_batch(h, B);
  if (rc) return rc;
  h->step = step;
  cudaStream_t st = h->stream;
  const int nout = h->nout;
  const int64_t P = (int64_t)B * kOutSide * kOutSide;
  const int64_t nl = P * nout;
  float* pred = at<float>(h, h->v.pred);
  float* lab = at<float>(h, h->v.labels);
  float* dpred = at<float>(h, h->v.dpred);
  float* part = at<float>(h, h->v.partials);
  float* grad = at<float>(h, h->v.grad);
  float* tot = at<float>(h, h->v.totals);
  const bf16* wb = at<bf16>(h, h->v.weights_bf16);
  const int nb = grid_for(nl, 256) < 4096 ? grid_for(nl, 256) : 4096;
  loss_partials_kernel<<<nb, 256, 0, st>>>(pred, lab, nl, at<float>(h, h->v.loss_partials));
  loss_reduce_kernel<<<1, 256, 0, st>>>(at<float>(h, h->v.loss_partials), nb, tot, loss_dev);
  dpred_kernel<<<grid_for(nl, 256), 256, 0, st>>>(pred, lab, nl, tot, dpred);
  // head
  head_bwd_dx_kernel<<<grid_for(P, 128), 128, 0, st>>>(dpred, wb + h->PL.wh, P, nout, at<float>(h, h->v.dact[3]));
  {
    // chunks of kHeadChunkPx pixels (4x more CTAs than kChunkPx): the head's P = B * 256 pixels
    // would otherwise give too few CTAs; their partials fit the buffer sized for the first layer
    const int E = nout * kHid + nout;
    const int64_t Emax = (int64_t)kHid * 9 * kHid + kHid > E ? (int64_t)kHid * 9 * kHid + kHid : E;
    const int64_t cap = (int64_t)chunks_for((int64_t)h->max_batch * kSide[1] * kSide[1], kChunkPx) * Emax;
    const int chunk = (int64_t)chunks_for(P, kHeadChunkPx) * E <= cap ? kHeadChunkPx : kChunkPx;
    const int ch = chunks_for(P, chunk);
    if ((E + 255) / 256 > 24) return fail("surrogate head too wide for the weight-gradient kernel");
    const size_t shm = (size_t)kSub * (nout + kHid) * sizeof(float);
    cudaFuncSetAttribute(head_bwd_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    head_bwd_dw_kernel<<<ch, 256, shm, st>>>(dpred, at<bf16>(h, h->v.act[3]), P, nout, chunk, part);
    reduce_partials_kernel<<<grid_for(E, 256), 256, 0, st>>>(part, ch, E, grad + h->PL.wh);
  }
  // conv layers, last to first; dact[l] holds d loss / d (output of layer l)
  for (int l = 3; l >= 0; --l) {
    const int S = kSide[l], So = kSide[l + 1], d = kDil[l];
    const bf16* xin = l == 0 ? at<bf16>(h, h->v.features) : at<bf16>(h, h->v.act[l - 1]);
    const bf16* y = at<bf16>(h, h->v.act[l]);
    const float* dy = at<float>(h, h->v.dact[l]);
    const int64_t Po = (int64_t)B * So * So;
    const int ch = chunks_for(Po, kChunkPx);
    if (l == 0) {
      const int E = kHid * 9 * kInF + kHid;
      conv_bwd_dw_kernel<kInF><<<ch, 256, 0, st>>>(dy, y, xin, B, S, S, d, part);
      reduce_partials_kernel<<<grid_for(E, 256), 256, 0, st>>>(part, ch, E, grad + h->PL.w[0]);
    } else if (h->engine == SEB_SUR_TCGEN05) {
      const int E = kHid * 9 * kHid + kHid;
      // the upstream gradient, masked by this layer's ReLU and split into BF16 hi / lo, over itself
      float* dyw = at<float>(h, h->v.dact[l]);
      split_dz_kernel<<<grid_for(Po, 128), 128, 0, st>>>(dyw, y, Po);
      const bf16* dzs = reinterpret_cast<const bf16*>(dyw);
      cudaFuncSetAttribute(conv_bwd_dw_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwSmem);
      conv_bwd_dw_tc_kernel<<<ch, kTcM, kBwSmem, st>>>(dzs, xin, B, S, S, d, part, h->err);
      reduce_partials_kernel<<<grid_for(E, 256), 256, 0, st>>>(part, ch, E, grad + h->PL.w[l]);
      // the weight partials have been summed: their buffer holds the transposed weights now
      bf16* wt = reinterpret_cast<bf16*>(part);
      transpose_w_kernel<<<grid_for(kHid * kTcK, 256), 256, 0, st>>>(wb + h->PL.w[l], wt);
      const ConvTile T = conv_tile(d, S, S);
      const int tx = (S + T.C - 1) / T.C, ty = (S + T.R - 1) / T.R;
      CUtensorMap zm;
      const int use_map = window_map(&zm, dzs, B, S - 2 * d, S - 2 * d, 2 * kHid, T.Pt, T.R + 2 * d) ? 1 : 0;
      cudaFuncSetAttribute(conv_bwd_dx_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kCtSmem);
      conv_bwd_dx_tile_kernel<<<(unsigned)((int64_t)B * ty * tx), kTcM, kCtSmem, st>>>(
          zm, use_map, dzs, wt, S, S, d, T, tx, ty, at<float>(h, h->v.dact[l - 1]), h->err);
    } else {
      const int E = kHid * 9 * kHid + kHid;
      conv_bwd_dw_kernel<kHid><<<ch, 256, 0, st>>>(dy, y, xin, B, S, S, d, part);
      reduce_partials_kernel<<<grid_for(E, 256), 256, 0, st>>>(part, ch, E, grad + h->PL.w[l]);
      conv_bwd_dx_kernel<<<grid_for((int64_t)B * S * S, 128), 128, 0, st>>>(dy, y, wb + h->PL.w[l], B, S, S, d,
                                                                             at<float>(h, h->v.dact[l - 1]));
    }
  }
  const double c1 = 1.0 - pow(0.9, (double)step), c2 = 1.0 - pow(0.999, (double)step);
  adam_kernel<<<grid_for(h->PL.n, 256), 256, 0, st>>>(at<float>(h, h->v.master), at<float>(h, h->v.adam_m),
                                                      at<float>(h, h->v.adam_v), grad, at<bf16>(h, h->v.weights_bf16),
                                                      h->PL.n, lr, 0.9f, 0.999f, 1e-8f, (float)c1, (float)c2);
  return cuda_check(cudaGetLastError(), "surrogate train step");
}

// Checkpoint image: a 64-byte header, then the FP32 master weights, the Adam first and second
// moments and the BF16 weights, each [n_params].
struct CkptHeader {
  char magic[8];      // "SEBSUR01"
  int64_t n_params;
  int32_t n_out, n_yaw;
  int64_t step;
  uint64_t bytes;     // whole image
  int32_t engine, pad;
  int64_t reserved[2];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

static size_t ckpt_bytes(const seb_sur* h) { return sizeof(CkptHeader) + (size_t)h->PL.n * (3 * 4 + 2); }

size_t seb_sur_state_bytes(const seb_sur* h) { return h ? ckpt_bytes(h) : 0; }

int seb_sur_save(seb_sur* h, void* dst, size_t bytes) {
  SEB_RANGE();
  if (!h || !dst) return fail("seb_sur_save: NULL handle or buffer");
  if (bytes < ckpt_bytes(h)) return fail("seb_sur_save: buffer of %zu bytes < %zu", bytes, ckpt_bytes(h));
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "SEBSUR01", 8);
  hd.n_params = h->PL.n;
  hd.n_out = h->nout;
  hd.n_yaw = h->p.n_yaw;
  hd.step = h->step;
  hd.bytes = ckpt_bytes(h);
  hd.engine = h->engine;
  uint8_t* o = static_cast<uint8_t*>(dst);
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  const size_t n4 = (size_t)h->PL.n * 4, n2 = (size_t)h->PL.n * 2;
  const size_t src[3] = {h->v.master, h->v.adam_m, h->v.adam_v};
  for (int i = 0; i < 3; ++i, o += n4) {
    int rc = cuda_check(cudaMemcpyAsync(o, h->ws + src[i], n4, cudaMemcpyDeviceToHost, h->stream), "seb_sur_save");
    if (rc) return rc;
  }
  int rc = cuda_check(cudaMemcpyAsync(o, h->ws + h->v.weights_bf16, n2, cudaMemcpyDeviceToHost, h->stream),
                      "seb_sur_save");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(h->stream), "seb_sur_save (synchronise)");
}

int seb_sur_load(seb_sur* h, const void* src, size_t bytes) {
  SEB_RANGE();
  if (!h || !src) return fail("seb_sur_load: NULL handle or buffer");
  CkptHeader hd;
  if (bytes < sizeof(hd)) return fail("seb_sur_load: image of %zu bytes has no header", bytes);
  memcpy(&hd, src, sizeof(hd));
  if (memcmp(hd.magic, "SEBSUR01", 8) != 0) return fail("seb_sur_load: not a surrogate checkpoint");
  if (hd.n_params != h->PL.n || hd.n_out != h->nout || hd.n_yaw != h->p.n_yaw)
    return fail("seb_sur_load: checkpoint of %lld parameters / %d outputs / %d yaw bins does not fit this network "
                "(%lld / %d / %d)", (long long)hd.n_params, hd.n_out, hd.n_yaw, (long long)h->PL.n, h->nout,
                h->p.n_yaw);
  if (hd.bytes != ckpt_bytes(h) || bytes < hd.bytes) return fail("seb_sur_load: truncated checkpoint");
  const uint8_t* i = static_cast<const uint8_t*>(src) + sizeof(hd);
  const size_t n4 = (size_t)h->PL.n * 4, n2 = (size_t)h->PL.n * 2;
  const size_t dst[3] = {h->v.master, h->v.adam_m, h->v.adam_v};
  for (int k = 0; k < 3; ++k, i += n4) {
    int rc = cuda_check(cudaMemcpyAsync(h->ws + dst[k], i, n4, cudaMemcpyHostToDevice, h->stream), "seb_sur_load");
    if (rc) return rc;
  }
  int rc = cuda_check(cudaMemcpyAsync(h->ws + h->v.weights_bf16, i, n2, cudaMemcpyHostToDevice, h->stream),
                      "seb_sur_load");
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(h->stream), "seb_sur_load (synchronise)");
  if (rc) return rc;
  h->step = hd.step;
  return SEB_OK;
}

int64_t seb_sur_step(const seb_sur* h) { return h ? h->step : -1; }

int seb_sur_infer(seb_sur* h, const float* elev, float step, int32_t radius, int32_t exact_fallback, float* out,
                  uint8_t* flags, uint8_t* mask_out) {
  SEB_RANGE();
  if (!h || !elev || !out || !flags || radius < 0) return fail("seb_sur_infer: bad args");
  cudaStream_t st = h->stream;
  const int nx = h->p.nx, ny = h->p.ny;
  const bf16* wb = at<bf16>(h, h->v.weights_bf16);
  const float* master = at<float>(h, h->v.master);
  bf16* feat = at<bf16>(h, h->v.map_features);
  map_features_kernel<<<grid_for((int64_t)(nx - 2) * (ny - 2), 256), 256, 0, st>>>(elev, nx, ny, h->p.res, feat);
  const bf16* x = feat;
  int W = nx - 2, H = ny - 2;
  for (int l = 0; l < 4; ++l) {
    bf16* y = at<bf16>(h, h->v.map_act[l]);
    conv_layer(h, x, l, 1, H, W, y);
    W -= 2 * kDil[l];
    H -= 2 * kDil[l];
    x = y;
  }
  {
    const size_t shm = (size_t)h->nout * (kHid + 1) * sizeof(float);
    cudaFuncSetAttribute(map_head_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    map_head_kernel<<<grid_for((int64_t)W * H, 128), 128, shm, st>>>(x, wb + h->PL.wh, master + h->PL.bh, elev, nx,
                                                                      ny, h->p.n_yaw, out, flags);
  }
  uint8_t* mask = mask_out ? mask_out : at<uint8_t>(h, h->v.mask);
  uint8_t* tiles = at<uint8_t>(h, h->v.tiles);
  const int tx = (nx + 31) / 32, ty = (ny + 31) / 32;
  int rc = cuda_check(cudaMemsetAsync(tiles, 0, (size_t)tx * ty, st), "tile flags");
  if (rc) return rc;
  if (radius >= 0 && radius <= kMaskMaxR)
    mask_tiled_kernel<<<dim3((unsigned)tx, (unsigned)ty), 256, 0, st>>>(elev, nx, ny, step, radius, mask, tiles, tx);
  else
    mask_kernel<<<grid_for((int64_t)nx * ny, 256), 256, 0, st>>>(elev, nx, ny, step, radius, mask, tiles, tx);
  rc = cuda_check(cudaGetLastError(), "surrogate inference");
  if (rc || !exact_fallback) return rc;
  seb::Launch L;
  seb::launch_defaults(h->p, h->T, &L);
  L.elev = elev;
  L.out = out;
  L.flags = flags;
  L.err = h->err;
  L.counters = reinterpret_cast<unsigned long long*>(h->err + 2);
  L.store_mask = mask;
  seb::launch_request(L, 0, 0, nx, ny);
  return cuda_check(seb::launch_assess(h->T, L, h->p.elev_dtype, h->p.precision, st), "exact fallback");
}

}  // extern "C"
