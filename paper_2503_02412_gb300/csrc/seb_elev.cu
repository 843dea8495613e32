// Elevation-map update from a LiDAR scan (Sec. V-A): robot-centred window (Eq. pm), clearing of
// cells that left it, ray-casting clearing, point filtering, per-point height variance (the
// three Jacobian terms of Sec. V-A) and one-dimensional Kalman fusion per cell with a
// Mahalanobis gate.
//
// Readings (the paper leaves these open): world point = R_B (R_BS p + p_BS) + p_B; the window
// origin is the robot's cell minus (nx / 2, ny / 2); ray casting clears a cell crossed by the
// segment sensor -> point (the point's own cell excluded) whose height exceeds the ray's highest
// height over the cell plus clear_margin; the points of one scan are gated against the cell's
// estimate from before the scan's fusion: points above the gate reset the cell to their fusion
// (a higher surface), points inside are fused with the estimate in information form, points
// below are dropped; an unknown cell takes the fusion of all its points.  The result does not
// depend on the order of the points.
//
// Kernels, per scan: move (clear the cells that entered the window), points (FP64 transform,
// filters, cell, variance: a scan has ~1e4-1e5 points, so FP64 costs little and the cell index
// and the gate decision match an FP64 evaluation), raycast (FP64 Amanatides-Woo walks, 8
// segments per ray; clearing is idempotent, so walks may race), accumulate (FP64 atomics of
// the information sums per cell) and finalize (one thread per cell).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "seb.h"
#include "seb_internal.h"

struct seb_elev {
  seb_elev_params p;
  int64_t max_points;
  cudaStream_t stream;
  float* h;       // [ny][nx], storage index = world index mod n
  float* s2;
  double* acc;    // [4][ny][nx]: in-gate sum w, sum w z; above-gate sum w, sum w z
  int32_t* nup;   // [ny][nx]: points above the gate
  int32_t* cell;  // [max_points]: storage index of a kept point, -1 otherwise
  double* pz;     // [max_points][2]: world height, variance
  uint8_t* inside;// [max_points]: (x, y) inside the window (ray casting)
  double* pw;     // [max_points][3]: world point
  double* rinv;   // [max_points][2]: 1 / dx, 1 / dy of the ray sensor -> point, in cells
  int64_t oi, oj;
  bool valid;
};

namespace {

struct PoseD {
  double R_B[9], p_B[3], R_BS[9], p_BS[3], S_S[9], S_R[9], S_B[9];
};

__device__ __forceinline__ void mv(const double* R, const double* v, double* o) {
  for (int i = 0; i < 3; ++i) o[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
}
__device__ __forceinline__ double quad(const double* S, const double* v) {  // v^T S v
  double r = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r += v[i] * S[3 * i + j] * v[j];
  return r;
}

struct ElevArgs {
  PoseD P;
  int nx, ny;
  double res, inv_res;
  int64_t oi, oj;            // window origin (world cell)
  int64_t old_oi, old_oj;    // previous origin (move kernel)
  int had_window;
  double z_min, z_max, gate, margin;
  double sx, sy, sz;         // sensor position in the world
};

__device__ __forceinline__ int64_t store_idx(const ElevArgs& A, int64_t wi, int64_t wj) {
  int64_t r = wj % A.ny, c = wi % A.nx;
  if (r < 0) r += A.ny;
  if (c < 0) c += A.nx;
  return r * A.nx + c;
}

__global__ void move_kernel(ElevArgs A, float* h, float* s2) {
  seb::pdl_entry();
  const int64_t n = (int64_t)A.nx * A.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / A.nx), c = (int)(t - (int64_t)r * A.nx);
    const int64_t wi = A.oi + c, wj = A.oj + r;
    const bool stay = A.had_window && wi >= A.old_oi && wi < A.old_oi + A.nx && wj >= A.old_oj &&
                      wj < A.old_oj + A.ny;
    if (!stay) {
      const int64_t s = store_idx(A, wi, wj);
      h[s] = __int_as_float(0x7fc00000);
      s2[s] = __int_as_float(0x7fc00000);
    }
  }
}

__global__ void points_kernel(ElevArgs A, const float* __restrict__ pts, int64_t n, int32_t* __restrict__ cell,
                              double* __restrict__ pz, uint8_t* __restrict__ inside, double* __restrict__ pw,
                              double* __restrict__ rinv) {
  seb::pdl_entry();
  double JS[3], RtB[3];
  {
    // J_S = (R_B R_BS)^T b3: the third row of R_B R_BS; R_B^T b3: the third row of R_B
    for (int k = 0; k < 3; ++k) {
      JS[k] = A.P.R_B[6] * A.P.R_BS[k] + A.P.R_B[7] * A.P.R_BS[3 + k] + A.P.R_B[8] * A.P.R_BS[6 + k];
      RtB[k] = A.P.R_B[6 + k];
    }
  }
  const double var_S = quad(A.P.S_S, JS), var_B = A.P.S_B[8];  // J_B = -b3
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double q[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    double b[3], w[3];
    mv(A.P.R_BS, q, b);
    for (int k = 0; k < 3; ++k) b[k] += A.P.p_BS[k];
    mv(A.P.R_B, b, w);
    for (int k = 0; k < 3; ++k) w[k] += A.P.p_B[k];
    pw[3 * i] = w[0];
    pw[3 * i + 1] = w[1];
    pw[3 * i + 2] = w[2];
    const bool fin = isfinite(w[0]) && isfinite(w[1]) && isfinite(w[2]);
    const double fi = floor(w[0] * A.inv_res), fj = floor(w[1] * A.inv_res);
    const bool in = fin && fi >= (double)A.oi && fi < (double)(A.oi + A.nx) && fj >= (double)A.oj &&
                    fj < (double)(A.oj + A.ny);
    inside[i] = in;
    // reciprocals of the ray's extent in cells (0 for an axis it does not move along)
    const double dxc = w[0] * A.inv_res - A.sx * A.inv_res, dyc = w[1] * A.inv_res - A.sy * A.inv_res;
    rinv[2 * i] = dxc != 0.0 ? 1.0 / dxc : 0.0;
    rinv[2 * i + 1] = dyc != 0.0 ? 1.0 / dyc : 0.0;
    const bool keep = in && b[2] >= A.z_min && b[2] <= A.z_max;
    cell[i] = keep ? (int32_t)store_idx(A, (int64_t)fi, (int64_t)fj) : -1;
    if (keep) {
      // J_R = b^ R_B^T b3 (right perturbation of the attitude)
      const double JR[3] = {b[1] * RtB[2] - b[2] * RtB[1], b[2] * RtB[0] - b[0] * RtB[2], b[0] * RtB[1] - b[1] * RtB[0]};
      pz[2 * i] = w[2];
      pz[2 * i + 1] = var_S + quad(A.P.S_R, JR) + var_B;
    }
  }
}

// Walk of the cells crossed by the segment sensor -> point in (x, y) (Amanatides & Woo), in
// world cell units; clears a crossed cell (the point's own excepted) whose height exceeds the
// ray's highest height over it plus the margin.  Each ray's parameter range [0, 1] is split in
// kRaySegs segments walked by separate threads (a scan has only ~1e4 rays): a segment starts at
// the cell holding its start point, with that cell's full entry / exit interval, and stops once
// the next cell is entered at or after its end.  A cell at a segment boundary may be tested by
// both neighbours, never by neither; clearing is idempotent, so that is harmless, and so are
// races between rays.  Four cells per round: indices and ray tops first, then their height loads
// together, then the tests.
constexpr int kRaySegs = 8;

__global__ void raycast_kernel(ElevArgs A, const double* __restrict__ pw, const double* __restrict__ rinv,
                               const uint8_t* __restrict__ inside, int64_t n, float* h, float* s2) {
  seb::pdl_entry();
  const double sx = A.sx * A.inv_res, sy = A.sy * A.inv_res, sz = A.sz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * kRaySegs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / kRaySegs;
    const int seg = (int)(t - i * kRaySegs);
    if (!inside[i]) continue;
    const double ex = pw[3 * i] * A.inv_res, ey = pw[3 * i + 1] * A.inv_res, ez = pw[3 * i + 2];
    const double dx = ex - sx, dy = ey - sy, dz = ez - sz;
    const double ix = rinv[2 * i], iy = rinv[2 * i + 1];  // 1 / dx, 1 / dy (0 when that extent is 0)
    const int stx = dx > 0 ? 1 : (dx < 0 ? -1 : 0), sty = dy > 0 ? 1 : (dy < 0 ? -1 : 0);
    const int64_t ei = (int64_t)floor(ex), ej = (int64_t)floor(ey);
    const double ts = (double)seg / kRaySegs, te = (double)(seg + 1) / kRaySegs;
    const bool up = dz > 0.0;
    int64_t ci = (int64_t)floor(seg == 0 ? sx : sx + dx * ts), cj = (int64_t)floor(seg == 0 ? sy : sy + dy * ts);
    // next boundary crossings and the entry time of the start cell
    double tmx = stx > 0 ? ((double)(ci + 1) - sx) * ix : (stx < 0 ? ((double)ci - sx) * ix : INFINITY);
    double tmy = sty > 0 ? ((double)(cj + 1) - sy) * iy : (sty < 0 ? ((double)cj - sy) * iy : INFINITY);
    const double tdx = stx ? fabs(ix) : INFINITY, tdy = sty ? fabs(iy) : INFINITY;
    double t0 = fmax(0.0, fmax(stx ? tmx - tdx : -INFINITY, sty ? tmy - tdy : -INFINITY));
    const int64_t max_steps = (int64_t)(fabs(dx) + fabs(dy)) + 4;  // cells crossed <= |dx| + |dy| + 2
    constexpr int U = 4;
    bool done = false;
    for (int64_t s = 0; s < max_steps && !done; s += U) {
      int64_t kc[U];
      double top[U];
      bool act[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        act[u] = false;
        if (done) continue;
        const double t1 = fmin(fmin(tmx, tmy), 1.0);
        if (ci == ei && cj == ej) {  // the point's own cell
          done = true;
          continue;
        }
        if (t1 > t0 && ci >= A.oi && ci < A.oi + A.nx && cj >= A.oj && cj < A.oj + A.ny) {
          act[u] = true;
          kc[u] = store_idx(A, ci, cj);
          // the ray's highest height over the cell: at its exit if it climbs, else at its entry
          // (the same double as the larger of the two, since the rounding of sz + dz t is monotone)
          top[u] = sz + dz * (up ? t1 : t0);
        }
        if (t1 >= te) {  // the next cell is entered at or after this segment's end (te <= 1)
          done = true;
          continue;
        }
        if (tmx < tmy) {
          ci += stx;
          t0 = tmx;
          tmx += tdx;
        } else {
          cj += sty;
          t0 = tmy;
          tmy += tdy;
        }
      }
      float hv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) hv[u] = act[u] ? h[kc[u]] : __int_as_float(0x7fc00000);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (act[u] && (double)hv[u] > top[u] + A.margin) {  // NaN compares false
          h[kc[u]] = __int_as_float(0x7fc00000);
          s2[kc[u]] = __int_as_float(0x7fc00000);
        }
      }
    }
  }
}

__global__ void accumulate_kernel(ElevArgs A, const int32_t* __restrict__ cell, const double* __restrict__ pz,
                                  int64_t n, const float* __restrict__ h, const float* __restrict__ s2,
                                  double* __restrict__ acc, int32_t* __restrict__ nup) {
  seb::pdl_entry();
  const int64_t plane = (int64_t)A.nx * A.ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cell[i];
    if (c < 0) continue;
    const double z = pz[2 * i], w = 1.0 / pz[2 * i + 1];
    const float h0 = h[c], v0 = s2[c];
    int slot = 0;  // 0: inside the gate (or an unknown cell), 1: above, -1: dropped
    if (!isnan(h0)) {
      const double d = (z - (double)h0) / sqrt((double)v0);
      slot = d > A.gate ? 1 : (d >= -A.gate ? 0 : -1);
    }
    if (slot < 0) continue;
    atomicAdd(acc + (2 * slot) * plane + c, w);
    atomicAdd(acc + (2 * slot + 1) * plane + c, w * z);
    if (slot == 1) atomicAdd(nup + c, 1);
  }
}

__global__ void finalize_kernel(int64_t plane, float* h, float* s2, double* acc, int32_t* nup) {
  seb::pdl_entry();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < plane; c += (int64_t)gridDim.x * blockDim.x) {
    const double aw = acc[c], awz = acc[plane + c], uw = acc[2 * plane + c], uwz = acc[3 * plane + c];
    const int up = nup[c];
    if (up > 0) {
      h[c] = (float)(uwz / uw);
      s2[c] = (float)(1.0 / uw);
    } else if (aw > 0.0) {
      const float h0 = h[c], v0 = s2[c];
      double W = aw, WZ = awz;
      if (!isnan(h0)) {
        W += 1.0 / (double)v0;
        WZ += (double)h0 / (double)v0;
      }
      h[c] = (float)(WZ / W);
      s2[c] = (float)(1.0 / W);
    }
    acc[c] = acc[plane + c] = acc[2 * plane + c] = acc[3 * plane + c] = 0.0;
    nup[c] = 0;
  }
}

__global__ void copy_out_kernel(ElevArgs A, const float* h, const float* s2, float* ho, float* so) {
  seb::pdl_entry();
  const int64_t n = (int64_t)A.nx * A.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / A.nx), c = (int)(t - (int64_t)r * A.nx);
    const int64_t s = store_idx(A, A.oi + c, A.oj + r);
    if (ho) ho[t] = h[s];
    if (so) so[t] = s2[s];
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t h, s2, acc, nup, cell, pz, inside, pw, rinv, total;
};

Layout layout(const seb_elev_params& p, int64_t np) {
  Layout L;
  const size_t plane = (size_t)p.nx * p.ny;
  size_t o = 0;
  L.h = o;
  o = align256(o + plane * 4);
  L.s2 = o;
  o = align256(o + plane * 4);
  L.acc = o;
  o = align256(o + 4 * plane * 8);
  L.nup = o;
  o = align256(o + plane * 4);
  L.cell = o;
  o = align256(o + (size_t)np * 4);
  L.pz = o;
  o = align256(o + (size_t)np * 16);
  L.inside = o;
  o = align256(o + (size_t)np);
  L.pw = o;
  o = align256(o + (size_t)np * 24);
  L.rinv = o;
  o = align256(o + (size_t)np * 16);
  L.total = o;
  return L;
}

bool params_ok(const seb_elev_params* p) {
  return p && p->nx >= 1 && p->ny >= 1 && p->nx <= 16384 && p->ny <= 16384 && p->res > 0.f && isfinite(p->res) &&
         p->z_min <= p->z_max && p->gate > 0.f;
}

int blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

// The ray walks are few (~1e5 segments) and uneven in length: small blocks spread them over the
// SMs more evenly.
constexpr int kRayThreads = 64;
int ray_blocks(int64_t n) {
  const int64_t b = (n + kRayThreads - 1) / kRayThreads;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

int fail(int code, const char* msg) {
  seb::set_error("%s", msg);
  return code;
}

}  // namespace

extern "C" {

void seb_elev_params_default(seb_elev_params* p) {
  SEB_RANGE();
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = p->ny = 400;
  p->res = 0.05f;
  p->z_min = -1.f;
  p->z_max = 1.f;
  p->gate = 2.5f;
  p->clear_margin = 0.05f;
}

size_t seb_elev_workspace_bytes(const seb_elev_params* p, int64_t max_points) {
  SEB_RANGE();
  if (!params_ok(p) || max_points < 0) return 0;
  return layout(*p, max_points).total;
}

int seb_elev_create(const seb_elev_params* p, int64_t max_points, void* ws, size_t bytes, seb_stream_t stream,
                    seb_elev** out) {
  SEB_RANGE();
  if (!out) return fail(SEB_ERR_INVALID_ARG, "seb_elev_create: out is NULL");
  *out = nullptr;
  if (!params_ok(p) || max_points < 0) return fail(SEB_ERR_INVALID_ARG, "seb_elev_create: bad parameters");
  const Layout L = layout(*p, max_points);
  if (!ws || bytes < L.total || ((uintptr_t)ws & 255))
    return fail(SEB_ERR_WORKSPACE, "seb_elev_create: workspace NULL, too small or not 256-byte aligned");
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ws) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(SEB_ERR_INVALID_ARG, "seb_elev_create: workspace is not device memory");
  }
  seb_elev* e = new (std::nothrow) seb_elev;
  if (!e) return fail(SEB_ERR_INVALID_ARG, "seb_elev_create: out of host memory");
  uint8_t* b = static_cast<uint8_t*>(ws);
  e->p = *p;
  e->max_points = max_points;
  e->stream = (cudaStream_t)stream;
  e->h = reinterpret_cast<float*>(b + L.h);
  e->s2 = reinterpret_cast<float*>(b + L.s2);
  e->acc = reinterpret_cast<double*>(b + L.acc);
  e->nup = reinterpret_cast<int32_t*>(b + L.nup);
  e->cell = reinterpret_cast<int32_t*>(b + L.cell);
  e->pz = reinterpret_cast<double*>(b + L.pz);
  e->inside = b + L.inside;
  e->pw = reinterpret_cast<double*>(b + L.pw);
  e->rinv = reinterpret_cast<double*>(b + L.rinv);
  e->oi = e->oj = 0;
  e->valid = false;
  const size_t plane = (size_t)p->nx * p->ny;
  cudaError_t err = cudaMemsetAsync(e->h, 0xff, plane * 4, e->stream);  // 0xffffffff: a NaN
  if (err == cudaSuccess) err = cudaMemsetAsync(e->s2, 0xff, plane * 4, e->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(e->acc, 0, 4 * plane * 8, e->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(e->nup, 0, plane * 4, e->stream);
  if (err != cudaSuccess) {
    delete e;
    return fail(SEB_ERR_CUDA, "seb_elev_create: clearing the workspace failed");
  }
  *out = e;
  return SEB_OK;
}

int seb_elev_destroy(seb_elev* e) {
  SEB_RANGE();
  delete e;
  return SEB_OK;
}

int seb_elev_set_stream(seb_elev* e, seb_stream_t s) {
  SEB_RANGE();
  if (!e) return fail(SEB_ERR_INVALID_ARG, "seb_elev_set_stream: NULL");
  e->stream = (cudaStream_t)s;
  return SEB_OK;
}

static ElevArgs args_of(const seb_elev* e, const seb_scan_pose* q) {
  ElevArgs A;
  memset(&A, 0, sizeof(A));
  if (q) {
    for (int k = 0; k < 9; ++k) {
      A.P.R_B[k] = q->R_B[k];
      A.P.R_BS[k] = q->R_BS[k];
      A.P.S_S[k] = q->Sigma_S[k];
      A.P.S_R[k] = q->Sigma_R[k];
      A.P.S_B[k] = q->Sigma_B[k];
    }
    for (int k = 0; k < 3; ++k) {
      A.P.p_B[k] = q->p_B[k];
      A.P.p_BS[k] = q->p_BS[k];
    }
  }
  A.nx = e->p.nx;
  A.ny = e->p.ny;
  A.res = e->p.res;
  A.inv_res = 1.0 / (double)e->p.res;
  A.oi = e->oi;
  A.oj = e->oj;
  A.z_min = e->p.z_min;
  A.z_max = e->p.z_max;
  A.gate = e->p.gate;
  A.margin = e->p.clear_margin;
  return A;
}

int seb_elev_integrate(seb_elev* e, const seb_scan_pose* pose, const float* pts, int64_t n) {
  SEB_RANGE();
  if (!e || !pose) return fail(SEB_ERR_INVALID_ARG, "seb_elev_integrate: NULL map or pose");
  if (n < 0 || n > e->max_points || (n > 0 && !pts))
    return fail(SEB_ERR_INVALID_ARG, "seb_elev_integrate: point count outside [0, max_points] or NULL points");
  ElevArgs A = args_of(e, pose);
  // Eq. (pm): window origin from the robot position (FP64 on the host)
  const int64_t oi = (int64_t)floor((double)pose->p_B[0] / (double)e->p.res) - e->p.nx / 2;
  const int64_t oj = (int64_t)floor((double)pose->p_B[1] / (double)e->p.res) - e->p.ny / 2;
  A.old_oi = e->oi;
  A.old_oj = e->oj;
  A.had_window = e->valid;
  A.oi = oi;
  A.oj = oj;
  // sensor position in the world: R_B p_BS + p_B
  double sw[3];
  for (int i = 0; i < 3; ++i)
    sw[i] = A.P.R_B[3 * i] * A.P.p_BS[0] + A.P.R_B[3 * i + 1] * A.P.p_BS[1] + A.P.R_B[3 * i + 2] * A.P.p_BS[2] +
            A.P.p_B[i];
  A.sx = sw[0];
  A.sy = sw[1];
  A.sz = sw[2];
  const cudaStream_t st = e->stream;
  const int64_t plane = (int64_t)e->p.nx * e->p.ny;
  cudaError_t err = seb::launch_pdl(move_kernel, dim3(blocks_for(plane)), dim3(256), 0, st, A, e->h, e->s2);
  if (n > 0 && err == cudaSuccess)
    err = seb::launch_pdl(points_kernel, dim3(blocks_for(n)), dim3(256), 0, st, A, pts, n, e->cell, e->pz, e->inside,
                          e->pw, e->rinv);
  if (n > 0 && err == cudaSuccess)
    err = seb::launch_pdl(raycast_kernel, dim3(ray_blocks(n * kRaySegs)), dim3(kRayThreads), 0, st, A, e->pw, e->rinv,
                          e->inside, n, e->h, e->s2);
  if (n > 0 && err == cudaSuccess)
    err = seb::launch_pdl(accumulate_kernel, dim3(blocks_for(n)), dim3(256), 0, st, A, e->cell, e->pz, n, e->h, e->s2,
                          e->acc, e->nup);
  if (n > 0 && err == cudaSuccess)
    err = seb::launch_pdl(finalize_kernel, dim3(blocks_for(plane)), dim3(256), 0, st, plane, e->h, e->s2, e->acc,
                          e->nup);
  if (err != cudaSuccess) {
    seb::set_error("seb_elev_integrate launch: %s", cudaGetErrorString(err));
    return SEB_ERR_CUDA;
  }
  e->oi = oi;
  e->oj = oj;
  e->valid = true;
  return SEB_OK;
}

int seb_elev_view_get(const seb_elev* e, seb_elev_view* v) {
  SEB_RANGE();
  if (!e || !v) return fail(SEB_ERR_INVALID_ARG, "seb_elev_view_get: NULL");
  v->height = e->h;
  v->variance = e->s2;
  v->ring_x = (int32_t)(((e->oi % e->p.nx) + e->p.nx) % e->p.nx);
  v->ring_y = (int32_t)(((e->oj % e->p.ny) + e->p.ny) % e->p.ny);
  v->origin_i = e->oi;
  v->origin_j = e->oj;
  return SEB_OK;
}

int seb_elev_copy_out(const seb_elev* e, float* height, float* variance) {
  SEB_RANGE();
  if (!e) return fail(SEB_ERR_INVALID_ARG, "seb_elev_copy_out: NULL");
  ElevArgs A = args_of(e, nullptr);
  const cudaError_t lerr = seb::launch_pdl(copy_out_kernel, dim3(blocks_for((int64_t)e->p.nx * e->p.ny)), dim3(256), 0,
                                           e->stream, A, e->h, e->s2, height, variance);
  const cudaError_t err = lerr != cudaSuccess ? lerr : cudaGetLastError();
  if (err != cudaSuccess) {
    seb::set_error("seb_elev_copy_out launch: %s", cudaGetErrorString(err));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}

}  // extern "C"
