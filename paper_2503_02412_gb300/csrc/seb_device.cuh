// Device helpers shared by the libseb kernels: element widening, compensated summation
// and the closed-form symmetric 3x3 eigen-solver.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace seb {

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) {
  return __half2float(v);
}

// Neumaier's compensated summation step (A. Neumaier, ZAMM 54, 1974).
__device__ __forceinline__ void nadd(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

struct Cell {
  float z, pitch, roll, rough, risk;
  uint32_t flags;
};

template <typename F>
__device__ __forceinline__ void cross(const F a[3], const F b[3], F o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Smallest eigenpair of the symmetric matrix (xx, xy, xz, yy, yz, zz).  Returns the unit
// eigenvector with n_z >= 0 in n and the relative gap (lambda_mid - lambda_min) / trace.
// Smith's form: q = tr/3, B = A - qI, p = sqrt(tr(B^2)/6), r = det(B)/(2 p^3),
// phi = acos(r)/3; eigenvalues q + 2p cos(phi + 2 pi j / 3), j = 0 (max), 1 (min), 2 (mid);
// hence lambda_mid - lambda_min = 2 sqrt(3) p sin(phi).
template <typename F>
__device__ __forceinline__ F min_eigpair(const F c[6], F n[3], F* gap_rel) {
  const F tr = c[0] + c[3] + c[5];
  const F q = tr / F(3);
  const F bxx = c[0] - q, byy = c[3] - q, bzz = c[5] - q;
  const F off = c[1] * c[1] + c[2] * c[2] + c[4] * c[4];
  const F p2 = (bxx * bxx + byy * byy + bzz * bzz + F(2) * off) / F(6);
  n[0] = n[1] = F(0);
  n[2] = F(1);
  if (!(p2 > F(0)) || !(tr > F(0))) {
    *gap_rel = F(0);
    return q;
  }
  const F p = sqrt(p2);
  const F det = bxx * (byy * bzz - c[4] * c[4]) - c[1] * (c[1] * bzz - c[4] * c[2]) +
                c[2] * (c[1] * c[4] - byy * c[2]);
  F r = det / (F(2) * p2 * p);
  r = r < F(-1) ? F(-1) : (r > F(1) ? F(1) : r);
  const F phi = acos(r) / F(3);
  const F lmin = q + F(2) * p * cos(phi + F(2.0943951023931954923));
  *gap_rel = F(3.4641016151377545870) * p * sin(phi) / tr;
  const F r0[3] = {c[0] - lmin, c[1], c[2]};
  const F r1[3] = {c[1], c[3] - lmin, c[4]};
  const F r2[3] = {c[2], c[4], c[5] - lmin};
  F v01[3], v02[3], v12[3];
  cross(r0, r1, v01);
  cross(r0, r2, v02);
  cross(r1, r2, v12);
  const F d01 = v01[0] * v01[0] + v01[1] * v01[1] + v01[2] * v01[2];
  const F d02 = v02[0] * v02[0] + v02[1] * v02[1] + v02[2] * v02[2];
  const F d12 = v12[0] * v12[0] + v12[1] * v12[1] + v12[2] * v12[2];
  const F* v = v01;
  F d = d01;
  if (d02 > d) {
    v = v02;
    d = d02;
  }
  if (d12 > d) {
    v = v12;
    d = d12;
  }
  if (!(d > F(0))) {
    *gap_rel = F(0);
    return lmin;
  }
  const F inv = F(1) / sqrt(d);
  const F sgn = v[2] < F(0) ? F(-1) : F(1);
  n[0] = v[0] * inv * sgn;
  n[1] = v[1] * inv * sgn;
  n[2] = v[2] * inv * sgn;
  return lmin;
}


// All three eigenvalues by the same closed form: lambda_j = q + 2p cos(phi + 2 pi j / 3),
// j = 0 (largest), 1 (smallest), 2 (middle).  l[0] <= l[1] <= l[2] on return.
template <typename F>
__device__ __forceinline__ void eigvals3(const F c[6], F l[3]) {
  const F tr = c[0] + c[3] + c[5];
  const F q = tr / F(3);
  const F bxx = c[0] - q, byy = c[3] - q, bzz = c[5] - q;
  const F off = c[1] * c[1] + c[2] * c[2] + c[4] * c[4];
  const F p2 = (bxx * bxx + byy * byy + bzz * bzz + F(2) * off) / F(6);
  if (!(p2 > F(0))) {
    l[0] = l[1] = l[2] = q;
    return;
  }
  const F p = sqrt(p2);
  const F det = bxx * (byy * bzz - c[4] * c[4]) - c[1] * (c[1] * bzz - c[4] * c[2]) +
                c[2] * (c[1] * c[4] - byy * c[2]);
  F r = det / (F(2) * p2 * p);
  r = r < F(-1) ? F(-1) : (r > F(1) ? F(1) : r);
  const F phi = acos(r) / F(3);
  l[2] = q + F(2) * p * cos(phi);
  l[0] = q + F(2) * p * cos(phi + F(2.0943951023931954923));
  l[1] = q + F(2) * p * cos(phi - F(2.0943951023931954923));
}

// Unit null vector of (A - lambda I) from the largest cross product of two of its rows.
template <typename F>
__device__ __forceinline__ bool null_vector(const F c[6], F lambda, F v[3]) {
  const F r0[3] = {c[0] - lambda, c[1], c[2]};
  const F r1[3] = {c[1], c[3] - lambda, c[4]};
  const F r2[3] = {c[2], c[4], c[5] - lambda};
  F a[3], b[3], d[3];
  cross(r0, r1, a);
  cross(r0, r2, b);
  cross(r1, r2, d);
  const F na = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const F nb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const F nd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const F* s = a;
  F m = na;
  if (nb > m) {
    s = b;
    m = nb;
  }
  if (nd > m) {
    s = d;
    m = nd;
  }
  if (!(m > F(0))) return false;
  const F inv = F(1) / sqrt(m);
  v[0] = s[0] * inv;
  v[1] = s[1] * inv;
  v[2] = s[2] * inv;
  return true;
}

// Rayleigh quotient n^T A n of a unit vector.
template <typename F>
__device__ __forceinline__ F rayleigh(const F c[6], const F n[3]) {
  return c[0] * n[0] * n[0] + c[3] * n[1] * n[1] + c[5] * n[2] * n[2] +
         F(2) * (c[1] * n[0] * n[1] + c[2] * n[0] * n[2] + c[4] * n[1] * n[2]);
}

// One Rayleigh-quotient refinement of the smallest eigenpair: the null vector of
// (A - n^T A n I) replaces n (kept when the rows are degenerate), oriented to n_z >= 0.
// Returns the refined n^T A n, clamped at 0.  Near a double smallest eigenvalue the
// closed-form eigenvalue loses accuracy (acos at r ~ -1); the quotient of the first vector
// is accurate to the square of its angle error, and the refined vector follows it.
template <typename F>
__device__ __forceinline__ F refine_min(const F c[6], F n[3]) {
  F v[3];
  if (null_vector<F>(c, rayleigh<F>(c, n), v)) {
    const F sgn = v[2] < F(0) ? F(-1) : F(1);
    n[0] = v[0] * sgn;
    n[1] = v[1] * sgn;
    n[2] = v[2] * sgn;
  }
  const F l = rayleigh<F>(c, n);
  return l > F(0) ? l : F(0);
}

// FP32 smallest eigenpair with the same closed form, arranged for throughput: one acos and
// one sincos (cos(phi + 2 pi / 3) = -cos(phi) / 2 - sqrt(3) sin(phi) / 2), and a reciprocal
// square root for the normalisation.  Returns the relative gap in *gap_rel.
__device__ __forceinline__ void min_eigpair_f(const float c[6], float n[3], float* gap_rel) {
  const float tr = c[0] + c[3] + c[5];
  const float q = tr * (1.f / 3.f);
  const float bxx = c[0] - q, byy = c[3] - q, bzz = c[5] - q;
  const float off = c[1] * c[1] + c[2] * c[2] + c[4] * c[4];
  const float p2 = (bxx * bxx + byy * byy + bzz * bzz + 2.f * off) * (1.f / 6.f);
  n[0] = n[1] = 0.f;
  n[2] = 1.f;
  *gap_rel = 0.f;
  if (!(p2 > 0.f) || !(tr > 0.f)) return;
  const float p = sqrtf(p2);
  const float det = bxx * (byy * bzz - c[4] * c[4]) - c[1] * (c[1] * bzz - c[4] * c[2]) +
                    c[2] * (c[1] * c[4] - byy * c[2]);
  float r = __fdividef(det, 2.f * p2 * p);  // clamped below; a 2-ulp quotient is ample
  r = fminf(fmaxf(r, -1.f), 1.f);
  float sp, cp;
  sincosf(acosf(r) * (1.f / 3.f), &sp, &cp);
  const float lmin = q + 2.f * p * (-0.5f * cp - 0.86602540378443865f * sp);
  *gap_rel = __fdividef(3.4641016151377546f * p * sp, tr);
  const float r0[3] = {c[0] - lmin, c[1], c[2]};
  const float r1[3] = {c[1], c[3] - lmin, c[4]};
  const float r2[3] = {c[2], c[4], c[5] - lmin};
  float a[3], b[3], d[3];
  cross(r0, r1, a);
  cross(r0, r2, b);
  cross(r1, r2, d);
  const float na = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  const float nb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const float nd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const float* v = a;
  float m = na;
  if (nb > m) {
    v = b;
    m = nb;
  }
  if (nd > m) {
    v = d;
    m = nd;
  }
  if (!(m > 0.f)) {
    *gap_rel = 0.f;
    return;
  }
  const float inv = (v[2] < 0.f ? -1.f : 1.f) * rsqrtf(m);
  n[0] = v[0] * inv;
  n[1] = v[1] * inv;
  n[2] = v[2] * inv;
}

// Tensor memory access (TMA) staging: one thread issues a 2-D tiled bulk copy of a box of a
// tensor map into the CTA's own shared memory (no multicast) and an mbarrier counts its bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Arrives once on the barrier and announces `bytes` of transaction for the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n selp.u32 %0, 1, 0, pw;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier: false when `limit` polls ran out (each poll
// already suspends the thread for a hardware-chosen time while the phase is incomplete).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Box of a 2-D tensor map at element coordinates (x, y) -> shared memory (128-byte aligned);
// x * element size must be a multiple of 16 bytes; y may be negative or beyond the tensor
// (out-of-bounds elements read as the map's fill value).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Box of a 4-D tensor map at element coordinates {c0..c3} -> shared memory (128-byte aligned);
// c0 * element size must be a multiple of 16 bytes, the others may be negative or beyond the
// tensor (out-of-bounds elements read as zero).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace seb
