// Trilinear lookup of an SE(2) grid at continuous poses, and its adjoint (Sec. VI: the
// planner reads Risk and the signed distance field at continuous states by trilinear
// interpolation of the grid, with the yaw handled on SO(2)).
//
// One thread per pose.  A float pose in metres far from the origin would lose the fraction
// within its cell if its grid coordinate were rounded to a float, and FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU; so each coordinate is formed as an unevaluated
// sum hi + lo of two floats with error-free transformations (the product by FMA, Dekker/Knuth
// two-sum), which carries ~48 bits.  The inside test, the cell index and the fraction are taken
// from that pair exactly.  The 8 corner values are read through the read-only path and the blend
// and its derivative run in FP32.  Poses with a non-finite coordinate or |yaw| > 1e4 rad count
// as outside the window; with n_yaw <= 4096 that keeps every step of the yaw reduction exact.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "seb.h"
#include "seb_internal.h"

namespace {

struct LookupArgs {
  const float* data;
  int nx, ny, K, ring_x, ring_y;
  float ir_h, ir_l;  // 1 / res as a float pair
  float ou_h, ou_l;  // o_i + 1/2
  float ov_h, ov_l;  // o_j + 1/2
  float ys_h, ys_l;  // K / (2 pi)
  float inv_k, inv_res, yaw_unit, fill;
};

// (hi, lo) with hi = fl(hi + lo) and |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void renorm(float& hi, float& lo) {
  const float s = hi + lo;
  lo = lo - (s - hi);
  hi = s;
}

// (hi, lo) + c as a normalised pair (two-sum of hi and c, its error folded into lo).
__device__ __forceinline__ void add_pair(float& hi, float& lo, float c) {
  const float s = hi + c;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (c - bb);
  hi = s;
  lo += e;
  renorm(hi, lo);
}

// x * (h + l) - (oh + ol) as a normalised float pair.
__device__ __forceinline__ void affine2(float x, float h, float l, float oh, float ol, float& hi, float& lo) {
  const float p = x * h;
  const float pe = fmaf(x, l, fmaf(x, h, -p));  // exact error of x h, plus x l
  const float s = p - oh;                        // two-sum of p and -oh
  const float bb = s - p;
  const float e = (p - (s - bb)) + (-oh - bb);
  hi = s;
  lo = e + (pe - ol);
  renorm(hi, lo);
}

// Cell index and fraction of the pair (hi, lo) in [0, n - 1]: i = min(floor(u), n - 2), f = u - i.
__device__ __forceinline__ void split(float hi, float lo, int n, int& i, float& f) {
  float c = floorf(hi);
  if (hi == c && lo < 0.f) c -= 1.f;
  if (c > (float)(n - 2)) c = (float)(n - 2);
  i = (int)c;
  f = (hi - c) + lo;  // hi - c is exact
}

// hi + lo in [0, m] (m a small integer), decided exactly.
__device__ __forceinline__ bool in_range(float hi, float lo, float m) {
  const bool ge0 = hi > 0.f || (hi == 0.f && lo >= 0.f);
  const float d = hi - m;  // exact near the boundary (Sterbenz)
  const bool lem = d < 0.f || (d == 0.f && lo <= 0.f);
  return ge0 && lem;
}

struct Blend {
  float val, da, db, dt;  // value and its derivatives in grid units
};

// Cell, yaw bins and fractions of a pose; false when it is outside the window.
__device__ __forceinline__ bool locate(const LookupArgs& A, const float* pose, int& c0, int& r0, int& k0,
                                       int& k1, float& a, float& b, float& t) {
  const float x = pose[0], y = pose[1], yaw = pose[2];
  if (!(fabsf(yaw) <= 1e4f)) return false;
  float uh, ul, vh, vl;
  affine2(x, A.ir_h, A.ir_l, A.ou_h, A.ou_l, uh, ul);
  affine2(y, A.ir_h, A.ir_l, A.ov_h, A.ov_l, vh, vl);
  if (!(in_range(uh, ul, (float)(A.nx - 1)) && in_range(vh, vl, (float)(A.ny - 1)))) return false;  // NaN: false
  split(uh, ul, A.nx, c0, a);
  split(vh, vl, A.ny, r0, b);
  // w = yaw K / (2 pi) = wh + wl, reduced modulo K.  |yaw| <= 1e4 and K <= 4096 keep |wh| and
  // K q below 2^23, so K q is exact; the subtraction and the range corrections are two-sums.
  float r = yaw * A.ys_h;
  float rl = fmaf(yaw, A.ys_l, fmaf(yaw, A.ys_h, -r));
  renorm(r, rl);
  const float Kf = (float)A.K;
  add_pair(r, rl, -Kf * floorf(r * A.inv_k));
  if (r < 0.f || (r == 0.f && rl < 0.f)) add_pair(r, rl, Kf);
  if (r > Kf || (r == Kf && rl >= 0.f)) add_pair(r, rl, -Kf);
  float kf = floorf(r);
  if (r == kf && rl < 0.f) kf -= 1.f;
  k0 = (int)kf;
  t = (r - kf) + rl;
  if (k0 < 0) {  // only reachable through rounding at w = 0 from below
    k0 = 0;
    t = 0.f;
  } else if (k0 > A.K - 1) {
    k0 = A.K - 1;
    t = 1.f;
  }
  t = fminf(fmaxf(t, 0.f), 1.f);
  k1 = k0 + 1 == A.K ? 0 : k0 + 1;
  return true;
}

__device__ __forceinline__ Blend blend(const LookupArgs& A, int c0, int r0, int k0, int k1, float a, float b,
                                       float t) {
  int pc0 = c0 + A.ring_x, pr0 = r0 + A.ring_y;
  if (pc0 >= A.nx) pc0 -= A.nx;
  if (pr0 >= A.ny) pr0 -= A.ny;
  const int pc1 = pc0 + 1 == A.nx ? 0 : pc0 + 1;
  const int pr1 = pr0 + 1 == A.ny ? 0 : pr0 + 1;
  const int64_t plane = (int64_t)A.nx * A.ny;
  const float* d0 = A.data + (int64_t)k0 * plane;
  const float* d1 = A.data + (int64_t)k1 * plane;
  const int64_t i00 = (int64_t)pr0 * A.nx + pc0, i01 = (int64_t)pr0 * A.nx + pc1;
  const int64_t i10 = (int64_t)pr1 * A.nx + pc0, i11 = (int64_t)pr1 * A.nx + pc1;
  // v[yaw][row][col]
  const float v000 = __ldg(d0 + i00), v001 = __ldg(d0 + i01), v010 = __ldg(d0 + i10), v011 = __ldg(d0 + i11);
  const float v100 = __ldg(d1 + i00), v101 = __ldg(d1 + i01), v110 = __ldg(d1 + i10), v111 = __ldg(d1 + i11);
  const float x00 = v001 - v000, x01 = v011 - v010, x10 = v101 - v100, x11 = v111 - v110;
  const float e00 = fmaf(a, x00, v000), e01 = fmaf(a, x01, v010);
  const float e10 = fmaf(a, x10, v100), e11 = fmaf(a, x11, v110);
  const float y0 = e01 - e00, y1 = e11 - e10;
  const float f0 = fmaf(b, y0, e00), f1 = fmaf(b, y1, e10);
  Blend B;
  B.dt = f1 - f0;
  B.val = fmaf(t, B.dt, f0);
  B.db = fmaf(t, y1 - y0, y0);
  const float g0 = fmaf(b, x01 - x00, x00), g1 = fmaf(b, x11 - x10, x10);
  B.da = fmaf(t, g1 - g0, g0);
  return B;
}

__global__ void __launch_bounds__(256) lookup_kernel(const LookupArgs A, const float* __restrict__ poses, int64_t n,
                                                     float* __restrict__ val, float* __restrict__ grad,
                                                     uint8_t* __restrict__ flags) {
  seb::pdl_entry();
  const float yaw_unit = A.yaw_unit;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c0, r0, k0, k1;
    float a, b, t;
    float v = A.fill, gx = 0.f, gy = 0.f, gt = 0.f;
    uint8_t f = SEB_FLAG_UNKNOWN;
    if (locate(A, poses + 3 * i, c0, r0, k0, k1, a, b, t)) {
      const Blend B = blend(A, c0, r0, k0, k1, a, b, t);
      v = B.val;
      gx = B.da * A.inv_res;
      gy = B.db * A.inv_res;
      gt = B.dt * yaw_unit;
      f = v == v ? 0 : SEB_FLAG_UNKNOWN;
    }
    val[i] = v;
    if (grad) {
      grad[3 * i] = gx;
      grad[3 * i + 1] = gy;
      grad[3 * i + 2] = gt;
    }
    if (flags) flags[i] = f;
  }
}

__global__ void __launch_bounds__(256) lookup_vjp_kernel(const LookupArgs A, const float* __restrict__ poses,
                                                         int64_t n, const float* __restrict__ gval,
                                                         float* __restrict__ gpose) {
  seb::pdl_entry();
  const float yaw_unit = A.yaw_unit;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c0, r0, k0, k1;
    float a, b, t;
    float gx = 0.f, gy = 0.f, gt = 0.f;
    if (locate(A, poses + 3 * i, c0, r0, k0, k1, a, b, t)) {
      const Blend B = blend(A, c0, r0, k0, k1, a, b, t);
      const float g = gval[i];
      gx = g * B.da * A.inv_res;
      gy = g * B.db * A.inv_res;
      gt = g * B.dt * yaw_unit;
    }
    gpose[3 * i] = gx;
    gpose[3 * i + 1] = gy;
    gpose[3 * i + 2] = gt;
  }
}

int check_grid(const seb_grid* g, const char* who) {
  if (!g || !g->data) {
    seb::set_error("%s: grid or its data is NULL", who);
    return SEB_ERR_INVALID_ARG;
  }
  if (g->nx < 2 || g->ny < 2 || g->n_yaw < 1 || g->n_yaw > 4096 || !(g->res > 0.f) || !isfinite(g->res) || g->ring_x < 0 ||
      g->ring_x >= g->nx || g->ring_y < 0 || g->ring_y >= g->ny) {
    seb::set_error("%s: bad grid shape (nx, ny >= 2, 1 <= n_yaw <= 4096, res > 0, 0 <= ring < n)", who);
    return SEB_ERR_BAD_SHAPE;
  }
  return SEB_OK;
}

LookupArgs args_of(const seb_grid* g, float fill) {
  LookupArgs A;
  A.data = g->data;
  A.nx = g->nx;
  A.ny = g->ny;
  A.K = g->n_yaw;
  A.ring_x = g->ring_x;
  A.ring_y = g->ring_y;
  auto pair = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  const double ys = (double)g->n_yaw / (2.0 * 3.14159265358979323846);
  pair(1.0 / (double)g->res, A.ir_h, A.ir_l);
  pair((double)g->origin_i + 0.5, A.ou_h, A.ou_l);
  pair((double)g->origin_j + 0.5, A.ov_h, A.ov_l);
  pair(ys, A.ys_h, A.ys_l);
  A.inv_k = (float)(1.0 / (double)g->n_yaw);
  A.inv_res = (float)(1.0 / (double)g->res);
  A.yaw_unit = (float)ys;
  A.fill = fill;
  return A;
}

int blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

extern "C" int seb_se2_lookup(const seb_grid* g, const float* poses, int64_t n, float fill, float* val, float* grad,
                              uint8_t* flags, seb_stream_t stream) {
  SEB_RANGE();
  int rc = check_grid(g, "seb_se2_lookup");
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!poses || !val))) {
    seb::set_error("seb_se2_lookup: NULL poses/value pointer or negative count");
    return SEB_ERR_INVALID_ARG;
  }
  if (n == 0) return SEB_OK;
  const cudaError_t e = seb::launch_pdl(lookup_kernel, dim3(blocks_for(n)), dim3(256), 0, (cudaStream_t)stream,
                                        args_of(g, fill), poses, n, val, grad, flags);
  if (e != cudaSuccess) {
    seb::set_error("seb_se2_lookup launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}

extern "C" int seb_se2_lookup_vjp(const seb_grid* g, const float* poses, int64_t n, const float* gval, float* gpose,
                                  seb_stream_t stream) {
  SEB_RANGE();
  int rc = check_grid(g, "seb_se2_lookup_vjp");
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!poses || !gval || !gpose))) {
    seb::set_error("seb_se2_lookup_vjp: NULL pointer or negative count");
    return SEB_ERR_INVALID_ARG;
  }
  if (n == 0) return SEB_OK;
  const cudaError_t e = seb::launch_pdl(lookup_vjp_kernel, dim3(blocks_for(n)), dim3(256), 0, (cudaStream_t)stream,
                                        args_of(g, 0.f), poses, n, gval, gpose);
  if (e != cudaSuccess) {
    seb::set_error("seb_se2_lookup_vjp launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
