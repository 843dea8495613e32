// Signed distance field of the obstacle set of an SE(2) risk grid (Sec. VI: the planner's
// collision term reads an SDF over SE(2) whose value is the distance to the edge of the
// nearest region, negative inside obstacles; the paper builds it from the risk map).
//
// Per yaw bin k, obstacles are the cells with risk >= risk_obstacle (NaN counts as an
// obstacle); every other cell is free.  sdf = res * (distance to the nearest obstacle centre -
// distance to the nearest free centre), clamped to [-clamp, clamp]: a free cell gets its
// distance to the obstacles, an obstacle cell minus its distance to the free cells.  Distances
// are taken in the window's logical order (the ring wrap is storage, not adjacency), and the
// result is stored ring-indexed like the input, so the same seb_grid fields describe it.
//
// Exact Euclidean distances, separable: d^2(i, j) = min_j' g(i, j')^2 + (j - j')^2, with
// g(i, j') the distance in rows to the nearest feature of column j'.  Nothing farther than
// W = ceil(clamp / res) + 1 cells can fall under the clamp, so W bounds both passes.
//   1. cols_kernel: sweeps every column down and up (linear time), split in 8 row segments (16 on
//      small grids) swept by separate warps and joined through their first / last obstacle and
//      free rows, and stores per cell the distance in rows to the nearest obstacle and to the nearest free cell
//      of its column (uint16 each, 0xFFFF = none within W).  Loads are issued 8 rows at a time.
//   2. rows_kernel: a block per (bin, row) stages that row's squared column distances in shared
//      memory, padded with "no feature" sentinels; every cell takes the minimum of
//      g(j')^2 + (j - j')^2 over |j - j'| = 0, 1, 2, ..., four offsets per step, and stops when
//      (j - j')^2 alone reaches the best value.  The squared distances are exact 32-bit integers;
//      while W <= 179, rows16_kernel runs the same search on packed 16-bit pairs.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "seb.h"
#include "seb_internal.h"

namespace {

constexpr uint32_t kNone = 0xFFFFu;
constexpr int kMaxSide = 16384;
constexpr int kBatch = 8;      // column-pass loads in flight per thread
constexpr int kRowThreads = 256;
constexpr size_t kPadSmemMax = 96 * 1024;  // padded row pass up to this much shared memory
constexpr int32_t kFar = 1 << 30;  // "no feature": above any W^2 (W <= 16384), kFar + W^2 < 2^31

struct SdfArgs {
  const float* risk;
  float* sdf;
  uint32_t* work;  // [K][ny][nx] logical: (g_obstacle << 16) | g_free
  int nx, ny, K, ring_x, ring_y;
  int W;           // search bound in cells (<= 16383)
  float thr, res, clamp;
};

__device__ __forceinline__ int64_t phys(const SdfArgs& A, int k, int i, int j) {
  int r = i + A.ring_y, c = j + A.ring_x;
  if (r >= A.ny) r -= A.ny;
  if (c >= A.nx) c -= A.nx;
  return ((int64_t)k * A.ny + r) * A.nx + c;
}

// SEGS row segments (warps) per column stripe: more of them when the grid has few stripes.
template <int SEGS>
__global__ void __launch_bounds__(32 * SEGS) cols_kernel(const SdfArgs A) {
  seb::pdl_entry();
  // a block per (bin, 32-column stripe): lane = column, warp = one of SEGS row segments.  Each
  // warp sweeps its segment down (distances to the nearest obstacle / free cell at or above,
  // within the segment) and records the segment's first and last obstacle / free rows; after a
  // barrier it sweeps up, completing each distance with the nearest rows of the other segments.
  __shared__ int seg_rows[SEGS][4][32];  // last obstacle, first obstacle, last free, first free
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane, k = blockIdx.y;
  const int L = (A.ny + SEGS - 1) / SEGS, i0 = min(A.ny, seg * L), i1 = min(A.ny, i0 + L);
  const bool col = j < A.nx;
  uint32_t* out = A.work + (int64_t)k * A.ny * A.nx + j;
  int last_o = -1, first_o = -1, last_f = -1, first_f = -1;
  if (col) {
    // kBatch loads in flight before the batch's stores (the stores could alias the loads)
    for (int ib = i0; ib < i1; ib += kBatch) {
      float v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) v[u] = ib + u < i1 ? __ldg(A.risk + phys(A, k, ib + u, j)) : 0.f;
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = ib + u;
        if (i >= i1) break;
        const bool ob = !(v[u] < A.thr);  // NaN: obstacle
        if (ob) {
          last_o = i;
          first_o = first_o < 0 ? i : first_o;
        } else {
          last_f = i;
          first_f = first_f < 0 ? i : first_f;
        }
        const uint32_t uo = last_o < 0 ? kNone : (uint32_t)(i - last_o);
        const uint32_t uf = last_f < 0 ? kNone : (uint32_t)(i - last_f);
        out[(int64_t)i * A.nx] = (uo << 16) | uf;
      }
    }
  }
  seg_rows[seg][0][lane] = last_o;
  seg_rows[seg][1][lane] = first_o;
  seg_rows[seg][2][lane] = last_f;
  seg_rows[seg][3][lane] = first_f;
  __syncthreads();
  if (!col) return;
  int above_o = -1, above_f = -1, next_o = INT_MAX, next_f = INT_MAX;
  for (int s2 = seg - 1; s2 >= 0; --s2) {
    if (above_o < 0) above_o = seg_rows[s2][0][lane];
    if (above_f < 0) above_f = seg_rows[s2][2][lane];
  }
  for (int s2 = seg + 1; s2 < SEGS; ++s2) {
    if (next_o == INT_MAX && seg_rows[s2][1][lane] >= 0) next_o = seg_rows[s2][1][lane];
    if (next_f == INT_MAX && seg_rows[s2][3][lane] >= 0) next_f = seg_rows[s2][3][lane];
  }
  const int W = A.W;
  auto fin = [&](uint32_t up_in_seg, int above, int next, int i) -> uint32_t {
    int d = up_in_seg != kNone ? (int)up_in_seg : (above >= 0 ? i - above : INT_MAX);
    if (next != INT_MAX) d = min(d, next - i);
    return d > W ? kNone : (uint32_t)d;
  };
  for (int ib = i1 - 1; ib >= i0; ib -= kBatch) {
    uint32_t w[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) w[u] = ib - u >= i0 ? out[(int64_t)(ib - u) * A.nx] : 0u;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = ib - u;
      if (i < i0) break;
      const uint32_t uo = w[u] >> 16, uf = w[u] & 0xFFFFu;
      if (uo == 0) next_o = i;
      if (uf == 0) next_f = i;
      out[(int64_t)i * A.nx] = (fin(uo, above_o, next_o, i) << 16) | fin(uf, above_f, next_f, i);
    }
  }
}

template <bool PAD>
__global__ void __launch_bounds__(kRowThreads) rows_kernel(const SdfArgs A, int P) {
  seb::pdl_entry();
  // squared column distances to obstacles and to free cells, [2][nx]; with PAD each row carries
  // P "no feature" sentinels on both sides ([2][P + nx + P]), so that the search reads no index
  // out of range without clamping it
  extern __shared__ int32_t gsq[];
  const int k = blockIdx.x / A.ny, i = blockIdx.x - k * A.ny;
  const int nx = A.nx, stride = PAD ? nx + 2 * P : nx, off = PAD ? P : 0;
  const uint32_t* row = A.work + ((int64_t)k * A.ny + i) * nx;
  for (int t = threadIdx.x; t < stride; t += blockDim.x) {
    const int j = t - off;
    int32_t o = kFar, f = kFar;
    if (j >= 0 && j < nx) {
      const uint32_t v = row[j];
      const int32_t uo = (int32_t)(v >> 16), uf = (int32_t)(v & 0xFFFFu);
      o = uo == (int32_t)kNone ? kFar : uo * uo;
      f = uf == (int32_t)kNone ? kFar : uf * uf;
    }
    gsq[t] = o;
    gsq[stride + t] = f;
  }
  __syncthreads();
  const int32_t* go2 = gsq + off;
  const int32_t* gf2 = gsq + stride + off;
  // squared distances stay below (nx + P)^2 + kFar < 2^31: 32-bit integers
  const int32_t W2 = A.W * A.W;
  const int last = nx - 1;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    const bool obst = go2[j] == 0;
    const int32_t* h = obst ? gf2 : go2;  // obstacle cells search the free cells, and the reverse
    int32_t best = h[j];
    const int lim = min(A.W, max(j, last - j));
    if (PAD) {
      // Four offsets per early-exit test; the last group may read up to 3 offsets past lim,
      // which lie inside the padding (P >= lim + 3) and, beyond W or past the row end, only
      // give values above W^2 that the clamp maps to the same result.
      int32_t s2 = 1;
      for (int s = 1; s <= lim; s += 4) {
        if (s2 >= best) break;  // every farther column is at least s^2 away
        const int32_t q1 = s2 + 2 * s + 1, q2 = q1 + 2 * s + 3, q3 = q2 + 2 * s + 5;
        best = min(best, s2 + min(h[j - s], h[j + s]));
        best = min(best, q1 + min(h[j - s - 1], h[j + s + 1]));
        best = min(best, q2 + min(h[j - s - 2], h[j + s + 2]));
        best = min(best, q3 + min(h[j - s - 3], h[j + s + 3]));
        s2 = q3 + 2 * s + 7;
      }
    } else {
      // Offsets past a row end re-read the end column at an overstated distance (its true
      // offset was already counted), which cannot lower the minimum: the indices are clamped.
      for (int s = 1; s <= lim; s += 2) {
        const int32_t s2 = s * s;
        if (s2 >= best) break;
        const int32_t t2 = s2 + 2 * s + 1;
        const int32_t a0 = h[max(j - s, 0)], b0 = h[min(j + s, last)];
        const int32_t a1 = h[max(j - s - 1, 0)], b1 = h[min(j + s + 1, last)];
        best = min(best, min(s2 + min(a0, b0), t2 + min(a1, b1)));
      }
    }
    float d = best > W2 ? INFINITY : A.res * sqrtf((float)best);
    d = fminf(d, A.clamp);
    A.sdf[phys(A, k, i, j)] = obst ? -d : d;
  }
}

// Packed form of the row pass for search bounds W <= kW16Max: every squared distance, capped
// at W^2 + 1 ("nothing within W"), fits in 16 bits, and so does every candidate, because
// W^2 + 1 + (W + 3)^2 < 2^16.  Two candidates then share a register: one packed add and one
// min.u16x2 (native from sm_90) handle two offsets, which halves the integer work and the
// shared loads of the search (the 32-bit pass is issue-bound; this one is bound by the
// shared-memory pipe).
//
// Shared memory per block, for each of the two rows (distances to obstacles, to free cells):
// four u16 copies of the row padded by P = W + 4 cap values on both sides, each Lc long (the
// slots past the padding are never read):
//   F_c[x + P + c] = h[x]            (c = 0, 1: forward, shifted by c)
//   R_c[(nx - 1 - x) + P + c] = h[x] (reversed, shifted by c)
// A cell j takes the copies whose parity makes its pairs 4-byte aligned: at offset s (odd),
// the u32 at F_cR[j + s + P + cR] is (h[j + s], h[j + s + 1]) and the u32 at
// R_cL[nx - 1 - j + s + P + cL] is (h[j - s], h[j - s - 1]), already paired offset by offset.
// qtab[g] (s = 1 + 4 g) holds the packed squared offsets ((s)^2, (s+1)^2), ((s+2)^2, (s+3)^2)
// and (s^2, s^2) for the termination test; its last entry ends every search.
constexpr int kW16Max = 179;

__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__global__ void __launch_bounds__(kRowThreads) rows16_kernel(const SdfArgs A, int P, int Lc, int G) {
  seb::pdl_entry();
  extern __shared__ uint4 smem16[];
  uint4* qtab = smem16;                                         // G + 1 entries
  uint16_t* rows = reinterpret_cast<uint16_t*>(smem16 + G + 1);  // [2 rows][4 copies][Lc]
  const int k = blockIdx.x / A.ny, i = blockIdx.x - k * A.ny;
  const int nx = A.nx;
  const uint32_t cap = (uint32_t)(A.W * A.W + 1);
  const uint32_t* row = A.work + ((int64_t)k * A.ny + i) * nx;
  for (int g = threadIdx.x; g <= G; g += blockDim.x) {
    const uint32_t s = 1 + 4 * (uint32_t)g;
    const uint32_t s1 = s + 1, s2 = s + 2, s3 = s + 3;
    qtab[g] = g < G ? make_uint4(s * s | (s1 * s1) << 16, s2 * s2 | (s3 * s3) << 16, s * s * 0x10001u, 0u)
                    : make_uint4(0u, 0u, 0xFFFFFFFFu, 0u);
  }
  for (int x = (int)threadIdx.x - P; x < nx + P; x += blockDim.x) {
    uint32_t o = cap, f = cap;
    if (x >= 0 && x < nx) {
      const uint32_t v = row[x];
      const uint32_t uo = v >> 16, uf = v & 0xFFFFu;
      if (uo != kNone) o = uo * uo;  // column distances are <= W when not kNone
      if (uf != kNone) f = uf * uf;
    }
    const int pf = x + P, pr = nx - 1 - x + P;
    uint16_t* ro = rows;
    uint16_t* rf = rows + (size_t)4 * Lc;
    ro[pf] = (uint16_t)o;
    ro[Lc + pf + 1] = (uint16_t)o;
    ro[2 * Lc + pr] = (uint16_t)o;
    ro[3 * Lc + pr + 1] = (uint16_t)o;
    rf[pf] = (uint16_t)f;
    rf[Lc + pf + 1] = (uint16_t)f;
    rf[2 * Lc + pr] = (uint16_t)f;
    rf[3 * Lc + pr + 1] = (uint16_t)f;
  }
  __syncthreads();
  const int32_t W2 = A.W * A.W;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    const bool obst = rows[j + P] == 0;
    const uint16_t* h = rows + (obst ? (size_t)4 * Lc : 0);  // obstacle cells search the free cells
    const int cR = (j + 1 + P) & 1, cL = (nx - j + P) & 1;
    const uint32_t* pr = reinterpret_cast<const uint32_t*>(h + (size_t)cR * Lc) + ((j + 1 + P + cR) >> 1);
    const uint32_t* pl = reinterpret_cast<const uint32_t*>(h + (size_t)(2 + cL) * Lc) + ((nx - j + P + cL) >> 1);
    uint32_t B = (uint32_t)h[j + P] * 0x10001u;
    for (const uint4* q = qtab;; ++q, pr += 2, pl += 2) {
      const uint4 Q = *q;
      if (vmin_u16x2(B, Q.z) != Q.z) break;  // a half below s^2: every farther offset costs more
      const uint32_t a = vmin_u16x2(pr[0], pl[0]) + Q.x;
      const uint32_t b = vmin_u16x2(pr[1], pl[1]) + Q.y;
      B = vmin_u16x2(B, vmin_u16x2(a, b));
    }
    const int32_t best = (int32_t)min(B & 0xFFFFu, B >> 16);
    float d = best > W2 ? INFINITY : A.res * sqrtf((float)best);
    d = fminf(d, A.clamp);
    A.sdf[phys(A, k, i, j)] = obst ? -d : d;
  }
}

}  // namespace

extern "C" size_t seb_sdf_workspace_bytes(int32_t nx, int32_t ny, int32_t n_yaw) {
  SEB_RANGE();
  if (nx < 1 || ny < 1 || n_yaw < 1 || nx > kMaxSide || ny > kMaxSide) return 0;
  return (size_t)nx * ny * n_yaw * sizeof(uint32_t);
}

extern "C" int seb_risk_sdf(const seb_grid* g, float risk_obstacle, float clamp, void* work, size_t work_bytes,
                            float* sdf, seb_stream_t stream) {
  SEB_RANGE();
  if (!g || !g->data || !sdf || !work) {
    seb::set_error("seb_risk_sdf: NULL grid, output or workspace");
    return SEB_ERR_INVALID_ARG;
  }
  if (g->nx < 1 || g->ny < 1 || g->n_yaw < 1 || g->nx > kMaxSide || g->ny > kMaxSide || g->ring_x < 0 ||
      g->ring_x >= g->nx || g->ring_y < 0 || g->ring_y >= g->ny || !(g->res > 0.f)) {
    seb::set_error("seb_risk_sdf: bad grid shape (1 <= nx, ny <= %d, n_yaw >= 1, 0 <= ring < n, res > 0)",
                   kMaxSide);
    return SEB_ERR_BAD_SHAPE;
  }
  if (!(clamp >= 0.f)) {
    seb::set_error("seb_risk_sdf: clamp must be >= 0 (inf for none)");
    return SEB_ERR_INVALID_ARG;
  }
  const size_t need = seb_sdf_workspace_bytes(g->nx, g->ny, g->n_yaw);
  if (work_bytes < need || ((uintptr_t)work & 3)) {
    seb::set_error("seb_risk_sdf: workspace too small or misaligned (%zu bytes needed)", need);
    return SEB_ERR_WORKSPACE;
  }
  if ((const void*)sdf == (const void*)g->data) {
    seb::set_error("seb_risk_sdf: the output may not alias the risk grid");
    return SEB_ERR_INVALID_ARG;
  }
  SdfArgs A;
  A.risk = g->data;
  A.sdf = sdf;
  A.work = static_cast<uint32_t*>(work);
  A.nx = g->nx;
  A.ny = g->ny;
  A.K = g->n_yaw;
  A.ring_x = g->ring_x;
  A.ring_y = g->ring_y;
  A.thr = risk_obstacle;
  A.res = g->res;
  A.clamp = clamp;
  // search bound: the diagonal always suffices; a finite clamp caps it at clamp / res + 1
  const double side = (double)(g->nx > g->ny ? g->nx : g->ny);
  double w = ceil((double)clamp / (double)g->res) + 1.0;
  if (!(w < side)) w = side;
  A.W = (int)w;
  const cudaStream_t st = (cudaStream_t)stream;
  // 16 row segments per stripe when the grid has few stripes (a small map), else 8
  const dim3 cgrid((unsigned)((A.nx + 31) / 32), (unsigned)A.K);
  cudaError_t e = (int64_t)cgrid.x * cgrid.y < 600 ? seb::launch_pdl(cols_kernel<16>, cgrid, dim3(32 * 16), 0, st, A)
                                                  : seb::launch_pdl(cols_kernel<8>, cgrid, dim3(32 * 8), 0, st, A);
  // packed row pass when every candidate fits in 16 bits and its rows fit in shared memory
  // Lc = 32 (mod 64) u16: a copy and its shifted twin start 16 banks apart, so the pair loads
  // of 32 consecutive cells (alternating between the two) hit 32 distinct banks
  const int P16 = A.W + 4, Lc = (A.nx + 2 * P16 + 2 + 63) / 64 * 64 + 32, G = (A.W - 1) / 4 + 1;
  const size_t smem16 = (size_t)(G + 1) * sizeof(uint4) + (size_t)8 * Lc * sizeof(uint16_t);
  if (e == cudaSuccess && A.W <= kW16Max && smem16 <= kPadSmemMax) {
    e = cudaFuncSetAttribute(rows16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16);
    if (e == cudaSuccess) {
      const int passes = (A.nx + kRowThreads - 1) / kRowThreads;
      const int rthreads = ((A.nx + passes - 1) / passes + 31) / 32 * 32;
      e = seb::launch_pdl(rows16_kernel, dim3((unsigned)((int64_t)A.K * A.ny)), dim3(rthreads), smem16, st, A,
                          P16, Lc, G);
    }
    if (e != cudaSuccess) {
      seb::set_error("seb_risk_sdf launch: %s", cudaGetErrorString(e));
      return SEB_ERR_CUDA;
    }
    return SEB_OK;
  }
  // padding of the row pass: the search reaches offset min(W, nx - 1) + 3
  const int P = min(A.W, A.nx - 1) + 4;
  const size_t psmem = (size_t)2 * (A.nx + 2 * (size_t)P) * sizeof(int32_t);
  const bool pad = psmem <= kPadSmemMax;
  const size_t rsmem = pad ? psmem : (size_t)2 * A.nx * sizeof(int32_t);
  auto rk = pad ? rows_kernel<true> : rows_kernel<false>;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
  if (e == cudaSuccess) {
    // as few passes over the row as kRowThreads allows, split evenly between the passes
    const int passes = (A.nx + kRowThreads - 1) / kRowThreads;
    const int rthreads = ((A.nx + passes - 1) / passes + 31) / 32 * 32;
    e = seb::launch_pdl(rk, dim3((unsigned)((int64_t)A.K * A.ny)), dim3(rthreads), rsmem, st, A, P);
  }
  if (e != cudaSuccess) {
    seb::set_error("seb_risk_sdf launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
