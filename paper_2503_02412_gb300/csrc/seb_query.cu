// Continuous-pose query and its hand-written adjoint (a differentiable form of Algorithm 1
// for trajectory samples; the paper's planner instead interpolates the SE(2) grid, Sec. VI-C).
//
// Pose (x, y, theta): the yaw-0 footprint lattice {(di, dj)} (the same membership rule as
// the grid) is rotated by theta and placed at (x, y); each lattice point takes the bilinear
// elevation of the four surrounding cell centres (unknown if any is NaN or outside the
// window).  The known points P_i = (px_i, py_i, z_i), with (px, py) the metric offset from
// (x, y), give mean, population covariance, normal (smallest eigenvector, n_z > 0),
// roughness lambda_min / trace, the frame of Eqs. 2-3, pitch/roll and risk exactly as the
// grid kernel does; z is the fitted-plane height at (x, y):
//   z = mean z + (n_x mean px + n_y mean py) / n_z.
//
// Layout: batches of 65,536 poses or more take one pose per thread, streaming its lattice, so
// a warp runs the eigen-solve, frame and adjoint for 32 poses per pass.  Smaller batches, which
// would not fill the GPU that way, give a group of GL lanes (8 or 32) to each pose: lane l takes
// lattice points l, l + GL, ..., the 10 moment sums are reduced with warp shuffles, and every
// lane of the group then runs the eigen-solve, so no shared memory is needed.
//
// Backward (reverse mode, valid set held fixed): g = d loss / d (z, pitch, roll, rough, risk)
//   - roughness = lambda_min / trace directly; risk: zero on the clamped branches, else w . (kappa/kappa_max, |pitch|/phi_x_max,
//     |roll|/phi_y_max) with sign(0) = 0;
//   - pitch = asin(x_b,z), roll = asin(y_b,z); x_b = y_b x n; y_b = u/|u|, u = n x x_yaw;
//   - z through mean z, mean (px, py) and n;
//   - d lambda_min = n^T dC n; d n = sum_{j != min} v_j v_j^T dC n / (lambda_min - lambda_j);
//   - dC = (1/N) sum (dP_i e_i^T + e_i dP_i^T), e_i = P_i - mean;
//   - dP_i / d(x, y, theta): px = c i - s j, py = s i + c j (metres), so d px / d theta = -py,
//     d py / d theta = px; z_i = bilinear(x + px, y + py) with its cell-wise gradient.
#include <algorithm>
#include <math.h>
#include <string.h>

#include "seb_device.cuh"
#include "seb_internal.h"

namespace seb {
namespace {

constexpr int kPPL = 8;  // lattice points per lane (grouped kernels)
constexpr int64_t kOneLaneMin = 65536;  // batches this large take one pose per thread

struct QState {
  int N;
  float zref;
  float mu[3];  // mean of (px, py, z - zref)
  float C[6];
  float n[3];
  float lam, rough;
  float z, pitch, roll, risk;
  uint32_t flags;
};

template <int GL>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int GL>
__device__ __forceinline__ int group_min(int v) {
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct Pts {
  float px[kPPL], py[kPPL], z[kPPL], gx[kPPL], gy[kPPL];
  bool ok[kPPL];
};

template <typename E, int GL>
__device__ __forceinline__ void gather(const QTab& Q, const QLaunch& L, int lane, float xl, float yl,
                                       float c, float s, Pts& P) {
  const E* __restrict__ elev = static_cast<const E*>(L.elev);
  const float res = L.res, ires = 1.f / L.res;
#pragma unroll
  for (int j = 0; j < kPPL; ++j) {
    const int q = lane + j * GL;
    P.ok[j] = false;
    P.px[j] = P.py[j] = P.z[j] = P.gx[j] = P.gy[j] = 0.f;
    if (q >= Q.n) continue;
    const float di = (float)Q.di[q], dj = (float)Q.dj[q];
    const float ox = c * di - s * dj, oy = s * di + c * dj;  // offset in cells
    const float gxc = xl + ox, gyc = yl + oy;                // grid coordinate
    const float c0 = floorf(gxc), r0 = floorf(gyc);
    P.px[j] = ox * res;
    P.py[j] = oy * res;
    if (!(c0 >= 0.f && r0 >= 0.f && c0 + 1.f <= (float)(L.nx - 1) && r0 + 1.f <= (float)(L.ny - 1))) continue;
    const int ic = (int)c0, ir = (int)r0;
    const int64_t b = (int64_t)ir * L.nx + ic;
    const float z00 = to_f32<E>(elev[b]), z10 = to_f32<E>(elev[b + 1]);
    const float z01 = to_f32<E>(elev[b + L.nx]), z11 = to_f32<E>(elev[b + L.nx + 1]);
    if (!(z00 == z00 && z10 == z10 && z01 == z01 && z11 == z11)) continue;
    const float fx = gxc - c0, fy = gyc - r0;
    P.z[j] = (1.f - fx) * (1.f - fy) * z00 + fx * (1.f - fy) * z10 + (1.f - fx) * fy * z01 + fx * fy * z11;
    P.gx[j] = ((1.f - fy) * (z10 - z00) + fy * (z11 - z01)) * ires;
    P.gy[j] = ((1.f - fx) * (z01 - z00) + fx * (z11 - z10)) * ires;
    P.ok[j] = true;
  }
}

// Eigen-solve, frame and risk of one pose from its moment sums m (N, sum px, sum py, sum z',
// sum px^2, sum px py, sum py^2, sum px z', sum py z', sum z'^2; z' = z - zref).
__device__ __forceinline__ void finish_pose(const QTab& Q, const QLaunch& L, const float m[10], float zref,
                                            float c, float s, QState& S) {
  const float qnan = __int_as_float(0x7fc00000);
  S.N = (int)m[0];
  S.zref = zref;
  S.flags = 0;
  if (S.N < Q.n_min) {
    S.z = S.pitch = S.roll = S.rough = qnan;
    S.risk = 1.f;
    S.flags = SEB_FLAG_UNKNOWN | SEB_FLAG_OBSTACLE;
    for (int t = 0; t < 3; ++t) S.mu[t] = S.n[t] = 0.f;
    for (int t = 0; t < 6; ++t) S.C[t] = 0.f;
    S.lam = 0.f;
    return;
  }
  const float iN = 1.f / m[0];
  S.mu[0] = m[1] * iN;
  S.mu[1] = m[2] * iN;
  S.mu[2] = m[3] * iN;
  S.C[0] = fmaf(-S.mu[0], S.mu[0], m[4] * iN);
  S.C[1] = fmaf(-S.mu[0], S.mu[1], m[5] * iN);
  S.C[2] = fmaf(-S.mu[0], S.mu[2], m[7] * iN);
  S.C[3] = fmaf(-S.mu[1], S.mu[1], m[6] * iN);
  S.C[4] = fmaf(-S.mu[1], S.mu[2], m[8] * iN);
  S.C[5] = fmaf(-S.mu[2], S.mu[2], m[9] * iN);
  float gap;
  min_eigpair<float>(S.C, S.n, &gap);
  const float tr = S.C[0] + S.C[3] + S.C[5];
  if (gap < L.gap_fp64) {
    S.flags |= SEB_FLAG_FP64;
    double cd[6], nd[3], gd;
    for (int t = 0; t < 6; ++t) cd[t] = (double)S.C[t];
    min_eigpair<double>(cd, nd, &gd);
    refine_min<double>(cd, nd);
    for (int t = 0; t < 3; ++t) S.n[t] = (float)nd[t];
    if (gd < 1e-12) S.flags |= SEB_FLAG_DEGENERATE;
  } else {
    refine_min<float>(S.C, S.n);
  }
  const float* n = S.n;
  S.lam = fmaxf(rayleigh<float>(S.C, n), 0.f);
  S.rough = S.lam / tr;
  const float uz = n[0] * s - n[1] * c;
  const float un = sqrtf(n[2] * n[2] + uz * uz);
  if (!(n[2] > 1e-6f) || !(un >= 1e-6f)) S.flags |= SEB_FLAG_DEGENERATE;
  if (S.flags & SEB_FLAG_DEGENERATE) {
    S.z = S.pitch = S.roll = qnan;
    S.risk = 1.f;
    S.flags |= SEB_FLAG_OBSTACLE;
    return;
  }
  S.roll = asinf(fminf(fmaxf(uz / un, -1.f), 1.f));
  S.pitch = asinf(fminf(fmaxf(-n[2] * (n[0] * c + n[1] * s) / un, -1.f), 1.f));
  S.z = S.zref + S.mu[2] + (n[0] * S.mu[0] + n[1] * S.mu[1]) / n[2];
  const float ap = fabsf(S.pitch), ar = fabsf(S.roll);
  if (S.rough > L.kappa_max || ap > L.phi_x_max || ar > L.phi_y_max) {
    S.risk = 1.f;
    S.flags |= SEB_FLAG_OBSTACLE;
  } else {
    S.risk = L.w0 * (S.rough / L.kappa_max) + L.w1 * (ap / L.phi_x_max) + L.w2 * (ar / L.phi_y_max);
  }
}

// Moments, eigen-solve, frame and risk of one pose (every lane of the group gets the result).
template <int GL>
__device__ __forceinline__ void assess_pose(const QTab& Q, const QLaunch& L, int lane, float c, float s,
                                            const Pts& P, QState& S) {
  // Reference height: the known lattice point with the smallest index.
  int first = 1 << 30;
  float zf = 0.f;
#pragma unroll
  for (int j = kPPL - 1; j >= 0; --j)
    if (P.ok[j]) {
      first = lane + j * GL;
      zf = P.z[j];
    }
  const int gfirst = group_min<GL>(first);
  // broadcast zf from the lane that owns gfirst
  const int owner = gfirst % GL;
  const int base = (threadIdx.x & 31) & ~(GL - 1);
  const float zref = __shfl_sync(0xffffffffu, zf, base + (owner < GL ? owner : 0));
  float m[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) m[t] = 0.f;
#pragma unroll
  for (int j = 0; j < kPPL; ++j)
    if (P.ok[j]) {
      const float x = P.px[j], y = P.py[j], z = P.z[j] - zref;
      m[0] += 1.f;
      m[1] += x;
      m[2] += y;
      m[3] += z;
      m[4] = fmaf(x, x, m[4]);
      m[5] = fmaf(x, y, m[5]);
      m[6] = fmaf(y, y, m[6]);
      m[7] = fmaf(x, z, m[7]);
      m[8] = fmaf(y, z, m[8]);
      m[9] = fmaf(z, z, m[9]);
    }
#pragma unroll
  for (int t = 0; t < 10; ++t) m[t] = group_sum<GL>(m[t]);
  finish_pose(Q, L, m, gfirst < (1 << 30) ? zref : 0.f, c, s, S);
}

__device__ __forceinline__ void pose_local(const QLaunch& L, const float* pose, float& xl, float& yl,
                                           float& c, float& s) {
  // Grid coordinate of the pose: cell (col, row) has its centre at ((o + col + 1/2) res).
  // Done in FP64 once per pose so that large world coordinates keep their precision.
  xl = (float)((double)pose[0] / (double)L.res - L.oi - 0.5);
  yl = (float)((double)pose[1] / (double)L.res - L.oj - 0.5);
  sincosf(pose[2], &s, &c);
}

// Pose-level part of the adjoint (known, non-degenerate pose with state S): from the output
// gradient g[5] to the symmetrised covariance adjoint Sm (dL/dP_i = (Sm e_i + mub) / N for point i
// with e_i = P_i - mean) and the direct yaw term of the frame.
__device__ __forceinline__ void pose_adjoint(const QLaunch& L, const QState& S, const float* g, float c, float s,
                                             float Sm[9], float mub[3], float& th_direct) {
  const float g0 = g[0];
  float kb = g[3], pb = g[1], rb = g[2];
  if (!(S.flags & SEB_FLAG_OBSTACLE)) {
    const float sp = S.pitch > 0.f ? 1.f : (S.pitch < 0.f ? -1.f : 0.f);
    const float sr = S.roll > 0.f ? 1.f : (S.roll < 0.f ? -1.f : 0.f);
    kb += g[4] * L.w0 / L.kappa_max;
    pb += g[4] * L.w1 * sp / L.phi_x_max;
    rb += g[4] * L.w2 * sr / L.phi_y_max;
  }
  const float* n = S.n;
  const float uz = n[0] * s - n[1] * c;
  const float un = sqrtf(n[2] * n[2] + uz * uz);
  const float yb[3] = {-n[2] * s / un, n[2] * c / un, uz / un};
  float xb[3];
  cross(yb, n, xb);
  const float xbb[3] = {0.f, 0.f, pb * rsqrtf(fmaxf(1.f - xb[2] * xb[2], 1e-30f))};
  float ybb[3] = {0.f, 0.f, rb * rsqrtf(fmaxf(1.f - yb[2] * yb[2], 1e-30f))};
  float nb[3] = {0.f, 0.f, 0.f}, t3[3];
  cross(n, xbb, t3);  // x_b = y_b x n
  for (int t = 0; t < 3; ++t) ybb[t] += t3[t];
  cross(xbb, yb, t3);
  for (int t = 0; t < 3; ++t) nb[t] += t3[t];
  const float yd = yb[0] * ybb[0] + yb[1] * ybb[1] + yb[2] * ybb[2];
  float ub[3];
  for (int t = 0; t < 3; ++t) ub[t] = (ybb[t] - yb[t] * yd) / un;
  const float xy[3] = {c, s, 0.f};
  cross(xy, ub, t3);  // u = n x x_yaw
  for (int t = 0; t < 3; ++t) nb[t] += t3[t];
  float xyb[3];
  cross(ub, n, xyb);
  th_direct = -s * xyb[0] + c * xyb[1];
  // z = mean z + (n_x mean px + n_y mean py) / n_z
  const float h = n[0] * S.mu[0] + n[1] * S.mu[1];
  nb[0] += g0 * S.mu[0] / n[2];
  nb[1] += g0 * S.mu[1] / n[2];
  nb[2] -= g0 * h / (n[2] * n[2]);
  mub[0] = g0 * n[0] / n[2];
  mub[1] = g0 * n[1] / n[2];
  mub[2] = g0;
  // kappa = lambda_min / trace
  const float tr = S.C[0] + S.C[3] + S.C[5];
  const float lamb = kb / tr, trb = -kb * S.lam / (tr * tr);
  float Cb[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Cb[3 * a + b] = lamb * n[a] * n[b] + (a == b ? trb : 0.f);
  // eigenvector part: the other two eigenpairs
  float l[3];
  eigvals3<float>(S.C, l);
  float vmax[3], vmid[3];
  if (null_vector<float>(S.C, l[2], vmax)) {
    cross(n, vmax, vmid);
    const float nm = rsqrtf(vmid[0] * vmid[0] + vmid[1] * vmid[1] + vmid[2] * vmid[2]);
    for (int t = 0; t < 3; ++t) vmid[t] *= nm;
    // re-orthogonalise v_max against n and v_mid
    cross(vmid, n, vmax);
    const float* vs[2] = {vmid, vmax};
    const float ls[2] = {l[1], l[2]};
    for (int jv = 0; jv < 2; ++jv) {
      const float* v = vs[jv];
      const float coef = (v[0] * nb[0] + v[1] * nb[1] + v[2] * nb[2]) / (S.lam - ls[jv]);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Cb[3 * a + b] += coef * v[a] * n[b];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Sm[3 * a + b] = Cb[3 * a + b] + Cb[3 * b + a];
}

// Outputs and the per-pose state the backward reuses.
__device__ __forceinline__ void store_pose(const QLaunch& L, int64_t i, const QState& S) {
  float* o = L.out + 5 * i;
  o[0] = S.z;
  o[1] = S.pitch;
  o[2] = S.roll;
  o[3] = S.rough;
  o[4] = S.risk;
  L.flags[i] = (uint8_t)S.flags;
  if (L.saved) {
    float* v = L.saved + (int64_t)SEB_QUERY_SAVED * i;
    v[0] = (float)S.N;
    v[1] = S.zref;
    v[2] = S.mu[0];
    v[3] = S.mu[1];
    v[4] = S.mu[2];
    for (int t = 0; t < 6; ++t) v[5 + t] = S.C[t];
    v[11] = S.n[0];
    v[12] = S.n[1];
    v[13] = S.n[2];
    v[14] = S.lam;
    v[15] = __uint_as_float(S.flags);
  }
}

__device__ __forceinline__ void load_pose(const QLaunch& L, int64_t i, float c, float s, QState& S) {
  const float* v = L.saved + (int64_t)SEB_QUERY_SAVED * i;
  S.N = (int)v[0];
  S.zref = v[1];
  S.mu[0] = v[2];
  S.mu[1] = v[3];
  S.mu[2] = v[4];
  for (int t = 0; t < 6; ++t) S.C[t] = v[5 + t];
  S.n[0] = v[11];
  S.n[1] = v[12];
  S.n[2] = v[13];
  S.lam = v[14];
  S.flags = __float_as_uint(v[15]);
  if (!(S.flags & (SEB_FLAG_UNKNOWN | SEB_FLAG_DEGENERATE))) {
    const float* n = S.n;
    const float uz = n[0] * s - n[1] * c;
    const float un = sqrtf(n[2] * n[2] + uz * uz);
    S.roll = asinf(fminf(fmaxf(uz / un, -1.f), 1.f));
    S.pitch = asinf(fminf(fmaxf(-n[2] * (n[0] * c + n[1] * s) / un, -1.f), 1.f));
    S.rough = S.lam / (S.C[0] + S.C[3] + S.C[5]);
  }
}

// One lattice point of a pose, in two steps: lattice_fetch computes the metric offset and
// issues the loads of the four bilinear corners; lattice_eval gives the bilinear height and its
// gradient, false when the point is unknown (a NaN or out-of-window corner).  Splitting them lets
// a thread issue the loads of several points before it uses any.
struct LatTap {
  float px, py, fx, fy, z00, z10, z01, z11;
  bool in;
};

template <typename E>
__device__ __forceinline__ void lattice_fetch(const QTab& Q, const QLaunch& L, const E* __restrict__ elev, int q,
                                              float xl, float yl, float c, float s, LatTap& t) {
  const float di = (float)Q.di[q], dj = (float)Q.dj[q];
  const float ox = c * di - s * dj, oy = s * di + c * dj;
  const float gxc = xl + ox, gyc = yl + oy;
  const float c0 = floorf(gxc), r0 = floorf(gyc);
  t.px = ox * L.res;
  t.py = oy * L.res;
  t.fx = gxc - c0;
  t.fy = gyc - r0;
  t.in = c0 >= 0.f && r0 >= 0.f && c0 + 1.f <= (float)(L.nx - 1) && r0 + 1.f <= (float)(L.ny - 1);
  if (t.in) {
    const int64_t b = (int64_t)(int)r0 * L.nx + (int)c0;
    t.z00 = to_f32<E>(elev[b]);
    t.z10 = to_f32<E>(elev[b + 1]);
    t.z01 = to_f32<E>(elev[b + L.nx]);
    t.z11 = to_f32<E>(elev[b + L.nx + 1]);
  }
}

__device__ __forceinline__ bool lattice_eval(const LatTap& t, const QLaunch& L, float& z, float& gx, float& gy) {
  if (!t.in) return false;
  const float z00 = t.z00, z10 = t.z10, z01 = t.z01, z11 = t.z11;
  if (!(z00 == z00 && z10 == z10 && z01 == z01 && z11 == z11)) return false;
  const float fx = t.fx, fy = t.fy, ires = 1.f / L.res;
  z = (1.f - fx) * (1.f - fy) * z00 + fx * (1.f - fy) * z10 + (1.f - fx) * fy * z01 + fx * fy * z11;
  gx = ((1.f - fy) * (z10 - z00) + fy * (z11 - z01)) * ires;
  gy = ((1.f - fx) * (z01 - z00) + fx * (z11 - z10)) * ires;
  return true;
}

template <typename E>
__device__ __forceinline__ bool lattice_point(const QTab& Q, const QLaunch& L, int q, float xl, float yl, float c,
                                              float s, float& px, float& py, float& z, float& gx, float& gy) {
  LatTap t;
  lattice_fetch<E>(Q, L, static_cast<const E*>(L.elev), q, xl, yl, c, s, t);
  px = t.px;
  py = t.py;
  return lattice_eval(t, L, z, gx, gy);
}

// Lattice points whose corner loads a one-pose-per-thread kernel keeps in flight at once (the
// forward stream and the adjoint stream; measured on 1 M poses: the adjoint's larger state
// leaves room for 2).
constexpr int kQB = 4, kQBB = 2;
constexpr int kQBS = 2;  // the same for the forward with the window in shared memory (lower latency)

// Moments of one pose by one thread, streaming its lattice in order (sums centred on the first
// known point, as the grouped kernels do, but added in lattice order).
template <typename E, int QB>
__device__ __forceinline__ void stream_moments(const QTab& Q, const QLaunch& L, const E* __restrict__ elev, float xl,
                                               float yl, float c, float s, float m[10], float& zref) {
  for (int t = 0; t < 10; ++t) m[t] = 0.f;
  zref = 0.f;
  bool have = false;
  for (int q0 = 0; q0 < Q.n; q0 += QB) {
    LatTap t[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      t[u].in = false;
      if (q0 + u < Q.n) lattice_fetch<E>(Q, L, elev, q0 + u, xl, yl, c, s, t[u]);
    }
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      float z, gx, gy;
      if (!lattice_eval(t[u], L, z, gx, gy)) continue;
      const float x = t[u].px, y = t[u].py;
      if (!have) {
        zref = z;
        have = true;
      }
      z -= zref;
      m[0] += 1.f;
      m[1] += x;
      m[2] += y;
      m[3] += z;
      m[4] = fmaf(x, x, m[4]);
      m[5] = fmaf(x, y, m[5]);
      m[6] = fmaf(y, y, m[6]);
      m[7] = fmaf(x, z, m[7]);
      m[8] = fmaf(y, z, m[8]);
      m[9] = fmaf(z, z, m[9]);
    }
  }
}

// One pose per thread, for large batches: a warp then runs the eigen-solve, frame and adjoint
// for 32 poses per pass (a group of GL lanes per pose runs them for 32 / GL).  `elev` is the
// window in global memory, or its copy in the CTA's shared memory.
template <typename E, int QB = kQB>
__device__ __forceinline__ void fwd1_pose(const QTab& Q, const QLaunch& L, const E* __restrict__ elev, int64_t i) {
  float xl, yl, c, s;
  pose_local(L, L.poses + 3 * i, xl, yl, c, s);
  float m[10], zref;
  stream_moments<E, QB>(Q, L, elev, xl, yl, c, s, m, zref);
  QState S;
  finish_pose(Q, L, m, zref, c, s, S);
  store_pose(L, i, S);
}

template <typename E>
__device__ __forceinline__ void bwd1_pose(const QTab& Q, const QLaunch& L, const E* __restrict__ elev, int64_t i) {
  float xl, yl, c, s;
  pose_local(L, L.poses + 3 * i, xl, yl, c, s);
  QState S;
  if (L.saved) {
    load_pose(L, i, c, s, S);
  } else {
    float m[10], zref;
    stream_moments<E, kQBB>(Q, L, elev, xl, yl, c, s, m, zref);
    finish_pose(Q, L, m, zref, c, s, S);
  }
  float gpx = 0.f, gpy = 0.f, gth = 0.f;
  if (!(S.flags & (SEB_FLAG_UNKNOWN | SEB_FLAG_DEGENERATE))) {
    float Sm[9], mub[3], th_direct;
    pose_adjoint(L, S, L.gout + 5 * i, c, s, Sm, mub, th_direct);
    const float iN = 1.f / (float)S.N;
    for (int q0 = 0; q0 < Q.n; q0 += kQBB) {
      LatTap t[kQBB];
#pragma unroll
      for (int u = 0; u < kQBB; ++u) {
        t[u].in = false;
        if (q0 + u < Q.n) lattice_fetch<E>(Q, L, elev, q0 + u, xl, yl, c, s, t[u]);
      }
#pragma unroll
      for (int u = 0; u < kQBB; ++u) {
        float z, gx, gy;
        if (!lattice_eval(t[u], L, z, gx, gy)) continue;
        const float px = t[u].px, py = t[u].py;
        const float e0 = px - S.mu[0], e1 = py - S.mu[1], e2 = (z - S.zref) - S.mu[2];
        const float bx = (Sm[0] * e0 + Sm[1] * e1 + Sm[2] * e2 + mub[0]) * iN;
        const float by = (Sm[3] * e0 + Sm[4] * e1 + Sm[5] * e2 + mub[1]) * iN;
        const float bz = (Sm[6] * e0 + Sm[7] * e1 + Sm[8] * e2 + mub[2]) * iN;
        gpx = fmaf(bz, gx, gpx);
        gpy = fmaf(bz, gy, gpy);
        gth += -bx * py + by * px + bz * (-gx * py + gy * px);
      }
    }
    gth += th_direct;
  }
  L.gpose[3 * i] = gpx;
  L.gpose[3 * i + 1] = gpy;
  L.gpose[3 * i + 2] = gth;
}

template <typename E>
__global__ void __launch_bounds__(256) query_fwd1_kernel(const __grid_constant__ QTab Q,
                                                         const __grid_constant__ QLaunch L) {
  seb::pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  fwd1_pose<E>(Q, L, static_cast<const E*>(L.elev), i);
}

template <typename E>
__global__ void __launch_bounds__(256) query_bwd1_kernel(const __grid_constant__ QTab Q,
                                                         const __grid_constant__ QLaunch L) {
  seb::pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  bwd1_pose<E>(Q, L, static_cast<const E*>(L.elev), i);
}

// The same with the whole window copied into the CTA's shared memory first: the ~140 bilinear
// corner loads of a pose then come from shared memory instead of L1 / L2.  Persistent: each CTA
// copies the window once and loops over poses.  It pays while three CTAs fit on an SM (a window
// of up to kQMapSmem bytes: 100 x 100 FP32, or 180 x 180 BF16 at 0.1 m); with one CTA per SM
// the lost occupancy costs more than the loads save, so larger windows stay in global memory.
constexpr size_t kQMapSmem = 72 * 1024;
template <typename E, bool BWD>
__global__ void __launch_bounds__(256, 3) query1_smem_kernel(const __grid_constant__ QTab Q,
                                                          const __grid_constant__ QLaunch L) {
  extern __shared__ __align__(16) unsigned char qsm[];
  E* map = reinterpret_cast<E*>(qsm);
  seb::pdl_entry();
  const E* g = static_cast<const E*>(L.elev);
  const int64_t cells = (int64_t)L.nx * L.ny;
  int64_t k0 = 0;
  if (((uintptr_t)g & 15) == 0) {  // 16-byte copies, then the tail element by element
    const int64_t n16 = cells * (int64_t)sizeof(E) / 16;
    for (int64_t k = threadIdx.x; k < n16; k += blockDim.x)
      reinterpret_cast<uint4*>(map)[k] = __ldg(reinterpret_cast<const uint4*>(g) + k);
    k0 = n16 * 16 / (int64_t)sizeof(E);
  }
  for (int64_t k = k0 + threadIdx.x; k < cells; k += blockDim.x) map[k] = g[k];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (BWD)
      bwd1_pose<E>(Q, L, map, i);
    else
      fwd1_pose<E, kQBS>(Q, L, map, i);
  }
}

template <typename E, int GL>
__global__ void __launch_bounds__(256) query_fwd_kernel(const __grid_constant__ QTab Q,
                                                        const __grid_constant__ QLaunch L) {
  seb::pdl_entry();
  const int gpb = 256 / GL;
  const int64_t i = (int64_t)blockIdx.x * gpb + threadIdx.x / GL;
  const int lane = threadIdx.x & (GL - 1);
  const bool live = i < L.n;
  const int64_t ii = live ? i : L.n - 1;  // dead groups mirror the last pose (no store)
  float xl, yl, c, s;
  pose_local(L, L.poses + 3 * ii, xl, yl, c, s);
  Pts P;
  gather<E, GL>(Q, L, lane, xl, yl, c, s, P);
  QState S;
  assess_pose<GL>(Q, L, lane, c, s, P, S);
  if (!live || lane != 0) return;
  store_pose(L, i, S);
}

template <typename E, int GL>
__global__ void __launch_bounds__(256) query_bwd_kernel(const __grid_constant__ QTab Q,
                                                        const __grid_constant__ QLaunch L) {
  seb::pdl_entry();
  const int gpb = 256 / GL;
  const int64_t i = (int64_t)blockIdx.x * gpb + threadIdx.x / GL;
  const int lane = threadIdx.x & (GL - 1);
  const bool live = i < L.n;
  const int64_t ii = live ? i : L.n - 1;
  float xl, yl, c, s;
  pose_local(L, L.poses + 3 * ii, xl, yl, c, s);
  Pts P;
  gather<E, GL>(Q, L, lane, xl, yl, c, s, P);
  QState S;
  if (L.saved)
    load_pose(L, ii, c, s, S);
  else
    assess_pose<GL>(Q, L, lane, c, s, P, S);
  float gpx = 0.f, gpy = 0.f, gth = 0.f;
  if (!(S.flags & (SEB_FLAG_UNKNOWN | SEB_FLAG_DEGENERATE))) {
    float Sm[9], mub[3], th_direct;
    pose_adjoint(L, S, L.gout + 5 * ii, c, s, Sm, mub, th_direct);
    const float iN = 1.f / (float)S.N;
#pragma unroll
    for (int j = 0; j < kPPL; ++j) {
      if (!P.ok[j]) continue;
      const float e0 = P.px[j] - S.mu[0], e1 = P.py[j] - S.mu[1], e2 = (P.z[j] - S.zref) - S.mu[2];
      const float bx = (Sm[0] * e0 + Sm[1] * e1 + Sm[2] * e2 + mub[0]) * iN;
      const float by = (Sm[3] * e0 + Sm[4] * e1 + Sm[5] * e2 + mub[1]) * iN;
      const float bz = (Sm[6] * e0 + Sm[7] * e1 + Sm[8] * e2 + mub[2]) * iN;
      gpx = fmaf(bz, P.gx[j], gpx);
      gpy = fmaf(bz, P.gy[j], gpy);
      gth += -bx * P.py[j] + by * P.px[j] + bz * (-P.gx[j] * P.py[j] + P.gy[j] * P.px[j]);
    }
    if (lane == 0) gth += th_direct;  // pose-level term, counted once per group
  }
  // Reductions outside the branch: every lane of the warp reaches the same shuffles.
  gpx = group_sum<GL>(gpx);
  gpy = group_sum<GL>(gpy);
  gth = group_sum<GL>(gth);
  if (!live || lane != 0) return;
  L.gpose[3 * i] = gpx;
  L.gpose[3 * i + 1] = gpy;
  L.gpose[3 * i + 2] = gth;
}

template <typename E>
cudaError_t launch_q(const QTab& Q, const QLaunch& L, bool backward, cudaStream_t st) {
  if (L.n == 0) return cudaSuccess;
  if (L.n >= kOneLaneMin) {  // enough poses to fill the GPU with one pose per thread
    const int64_t blocks = (L.n + 255) / 256;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const size_t map_bytes = (size_t)L.nx * L.ny * sizeof(E);
    if (map_bytes <= kQMapSmem) {  // the window fits in shared memory: persistent CTAs
      auto kern = backward ? query1_smem_kernel<E, true> : query1_smem_kernel<E, false>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)map_bytes);
      int dev = 0, sms = 0, per_sm = 0;
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, map_bytes);
      if (e != cudaSuccess) return e;
      if (per_sm > 0) {
        const int64_t grid = std::min<int64_t>(blocks, (int64_t)sms * per_sm);
        seb::launch_pdl(kern, dim3((unsigned)grid), dim3(256), map_bytes, st, Q, L);
        return cudaGetLastError();
      }
    }
    if (backward)
      seb::launch_pdl(query_bwd1_kernel<E>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
    else
      seb::launch_pdl(query_fwd1_kernel<E>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
    return cudaGetLastError();
  }
  const int GL = Q.n <= 8 * kPPL ? 8 : 32;
  const int gpb = 256 / GL;
  const int64_t blocks = (L.n + gpb - 1) / gpb;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  if (GL == 8) {
    if (backward)
      seb::launch_pdl(query_bwd_kernel<E, 8>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
    else
      seb::launch_pdl(query_fwd_kernel<E, 8>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
  } else {
    if (backward)
      seb::launch_pdl(query_bwd_kernel<E, 32>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
    else
      seb::launch_pdl(query_fwd_kernel<E, 32>, dim3((unsigned)blocks), dim3(256), 0, st, Q, L);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_query(const QTab& Q, const QLaunch& L, int elev_dtype, bool backward, cudaStream_t st) {
  switch (elev_dtype) {
    case SEB_F32: return launch_q<float>(Q, L, backward, st);
    case SEB_BF16: return launch_q<__nv_bfloat16>(Q, L, backward, st);
    default: return launch_q<__half>(Q, L, backward, st);
  }
}

int query_setup(const seb_params& p, const void* elev, int64_t oi, int64_t oj, const float* poses, int64_t n,
                QTab* Q, QLaunch* L) {
  int rc = validate_params(p);
  if (rc) return rc;
  if (p.elev_dtype == SEB_BF16_TILED) {
    set_error("the continuous query reads FP32, BF16 or FP16 elevation, not SEB_BF16_TILED windows");
    return SEB_ERR_INVALID_ARG;
  }
  Tables T;  // on the stack: the allocation-free query shares this path
  rc = build_tables(p, &T, nullptr);
  if (rc) return rc;
  rc = build_lattice(T, Q);
  if (rc) return rc;
  if (Q->n > 32 * kPPL) {
    set_error("footprint lattice exceeds %d points", 32 * kPPL);
    return SEB_ERR_BAD_SHAPE;
  }
  memset(L, 0, sizeof(*L));
  L->elev = elev;
  L->nx = p.nx;
  L->ny = p.ny;
  L->res = p.res;
  L->oi = (double)oi;
  L->oj = (double)oj;
  L->poses = poses;
  L->n = n;
  L->kappa_max = p.kappa_max;
  L->phi_x_max = p.phi_x_max;
  L->phi_y_max = p.phi_y_max;
  L->w0 = p.w[0];
  L->w1 = p.w[1];
  L->w2 = p.w[2];
  L->gap_fp64 = p.gap_fp64;
  return SEB_OK;
}

}  // namespace seb

using namespace seb;

extern "C" int seb_query_poses(const seb_params* p, const void* elev, int64_t oi, int64_t oj,
                               const float* poses, int64_t n, float* out, uint8_t* flags, float* saved,
                               seb_stream_t stream) {
  SEB_RANGE();
  if (!p || !elev || (n > 0 && (!poses || !out || !flags)) || n < 0) {
    set_error("seb_query_poses: NULL pointer or negative count");
    return SEB_ERR_INVALID_ARG;
  }
  QTab Q;
  QLaunch L;
  const int rc = query_setup(*p, elev, oi, oj, poses, n, &Q, &L);
  if (rc) return rc;
  L.out = out;
  L.flags = flags;
  L.saved = saved;
  cudaError_t e = launch_query(Q, L, p->elev_dtype, false, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error("seb_query_poses launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}

extern "C" int seb_query_poses_backward(const seb_params* p, const void* elev, int64_t oi, int64_t oj,
                                        const float* poses, const float* saved, const float* gout, float* gpose,
                                        int64_t n, seb_stream_t stream) {
  SEB_RANGE();
  if (!p || !elev || (n > 0 && (!poses || !gout || !gpose)) || n < 0) {
    set_error("seb_query_poses_backward: NULL pointer or negative count");
    return SEB_ERR_INVALID_ARG;
  }
  QTab Q;
  QLaunch L;
  const int rc = query_setup(*p, elev, oi, oj, poses, n, &Q, &L);
  if (rc) return rc;
  L.saved = const_cast<float*>(saved);
  L.gout = gout;
  L.gpose = gpose;
  cudaError_t e = launch_query(Q, L, p->elev_dtype, true, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error("seb_query_poses_backward launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
