// Nearest-neighbour inpainting of the elevation map (Sec. V-A: the map is inpainted before the
// traversability pass; Sec. VII-B: nearest-neighbour filling).  Every unknown (NaN) cell takes
// the elevation of the nearest known cell centre (Euclidean); among equally near known cells the
// smallest column, then the smallest row wins; known cells keep their value.  With a radius
// (max_cells > 0) farther cells stay unknown.
//
// Exact and separable, in integers: the nearest known cell of (i, j) minimises
// (i - r(j'))^2 + (j - j')^2 over the columns j', with r(j') the nearest known row of column j'.
//   1. cols_kernel: segmented down / up sweeps per column (8, 16 or 32 row segments per 32-column
//      stripe, by map height, joined through their first and last known rows) store r(i, j),
//      the nearest known row of column j to row i (the upper one on a tie), or -1.
//   2. rows_kernel: a block per row stages (i - r(j'))^2 in shared memory; each unknown cell
//      searches outwards, s = 1, 2, ..., while s^2 does not exceed its best value.  A candidate
//      on the left wins ties (it has the smaller column), one on the right only strict
//      improvements, which realises the tie rule exactly.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "seb.h"
#include "seb_internal.h"

namespace {

constexpr int kRowThreads = 256;
constexpr int kMaxSide = 16384;
constexpr int32_t kFar = 1 << 30;  // no known cell: above any squared distance (< 2^29)

// SEGS row segments (warps) per 32-column stripe: a map has few stripes, so tall maps take more.
template <int SEGS>
__global__ void __launch_bounds__(32 * SEGS) nn_cols_kernel(const float* __restrict__ elev, int nx, int ny,
                                                              int32_t* __restrict__ near_row) {
  seb::pdl_entry();
  __shared__ int seg_rows[SEGS][2][32];  // last known row, first known row of each segment
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int L = (ny + SEGS - 1) / SEGS, i0 = min(ny, seg * L), i1 = min(ny, i0 + L);
  const bool col = j < nx;
  int last = -1, first = -1;
  if (col) {
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
      if (!isnan(__ldg(elev + (int64_t)i * nx + j))) {
        last = i;
        first = first < 0 ? i : first;
      }
      near_row[(int64_t)i * nx + j] = last;  // nearest known at or above, within the segment
    }
  }
  seg_rows[seg][0][lane] = last;
  seg_rows[seg][1][lane] = first;
  __syncthreads();
  if (!col) return;
  int above = -1, next = INT_MAX;
  for (int s = seg - 1; s >= 0 && above < 0; --s) above = seg_rows[s][0][lane];
  for (int s = seg + 1; s < SEGS && next == INT_MAX; ++s)
    if (seg_rows[s][1][lane] >= 0) next = seg_rows[s][1][lane];
#pragma unroll 4
  for (int i = i1 - 1; i >= i0; --i) {
    int up = near_row[(int64_t)i * nx + j];
    if (up == i) next = i;  // a known cell here
    if (up < 0) up = above;
    const int du = up >= 0 ? i - up : INT_MAX, dd = next != INT_MAX ? next - i : INT_MAX;
    near_row[(int64_t)i * nx + j] = du == INT_MAX && dd == INT_MAX ? -1 : (du <= dd ? up : next);
  }
}

__global__ void __launch_bounds__(kRowThreads) nn_rows_kernel(const float* __restrict__ elev,
                                                              const int32_t* __restrict__ near_row, int nx,
                                                              int ny, int W, float* __restrict__ out,
                                                              int32_t* __restrict__ src) {
  seb::pdl_entry();
  extern __shared__ int32_t h[];  // [nx]: squared row distance to column j's nearest known cell
  const int i = blockIdx.x;
  const int32_t* nr = near_row + (int64_t)i * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    const int r = nr[j];
    h[j] = r < 0 ? kFar : (i - r) * (i - r);
  }
  __syncthreads();
  // W > 0: radius in cells; W <= 0: unbounded (the row search then spans the whole row)
  const bool bounded = W > 0;
  const int32_t W2 = bounded ? W * W : 0;
  const int last = nx - 1;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    const int64_t o = (int64_t)i * nx + j;
    const float z = elev[o];
    int si = -1, sj = -1;
    float v = __int_as_float(0x7fc00000);
    if (!isnan(z)) {
      v = z;
      si = i;
      sj = j;
    } else {
      int32_t best = h[j];
      int bj = j;
      const int lim = bounded ? min(W, max(j, last - j)) : max(j, last - j);
      // offsets past a row end re-read the end column at an overstated distance, which can
      // neither beat nor tie the value that column had at its true offset
      for (int s = 1; s <= lim; ++s) {
        const int32_t s2 = s * s;
        if (s2 > best) break;  // every farther column is more than s^2 away (ties still count)
        const int cl = max(j - s, 0), cr = min(j + s, last);
        const int32_t vl = s2 + h[cl], vr = s2 + h[cr];
        if (vl <= best) {  // smaller column than the best so far: wins ties
          best = vl;
          bj = cl;
        }
        if (vr < best) {
          best = vr;
          bj = cr;
        }
      }
      if (best < kFar && (!bounded || best <= W2)) {
        si = near_row[(int64_t)i * nx + bj];
        sj = bj;
        v = elev[(int64_t)si * nx + sj];
      }
    }
    out[o] = v;
    if (src) {
      src[2 * o] = si;
      src[2 * o + 1] = sj;
    }
  }
}

}  // namespace

extern "C" size_t seb_inpaint_workspace_bytes(int32_t nx, int32_t ny) {
  SEB_RANGE();
  if (nx < 1 || ny < 1 || nx > kMaxSide || ny > kMaxSide) return 0;
  return (size_t)nx * ny * sizeof(int32_t);
}

extern "C" int seb_inpaint_nearest(const float* elev, int32_t nx, int32_t ny, int32_t max_cells, void* work,
                                   size_t work_bytes, float* out, int32_t* src, seb_stream_t stream) {
  SEB_RANGE();
  if (!elev || !out || !work) {
    seb::set_error("seb_inpaint_nearest: NULL elevation, output or workspace");
    return SEB_ERR_INVALID_ARG;
  }
  if (nx < 1 || ny < 1 || nx > kMaxSide || ny > kMaxSide) {
    seb::set_error("seb_inpaint_nearest: map sides must be in [1, %d]", kMaxSide);
    return SEB_ERR_BAD_SHAPE;
  }
  if ((const void*)out == (const void*)elev) {
    seb::set_error("seb_inpaint_nearest: the output may not alias the elevation");
    return SEB_ERR_INVALID_ARG;
  }
  const size_t need = seb_inpaint_workspace_bytes(nx, ny);
  if (work_bytes < need || ((uintptr_t)work & 3)) {
    seb::set_error("seb_inpaint_nearest: workspace too small or misaligned (%zu bytes needed)", need);
    return SEB_ERR_WORKSPACE;
  }
  const int W = max_cells > 0 && max_cells < kMaxSide ? max_cells : 0;  // 0: unbounded
  int32_t* near_row = static_cast<int32_t*>(work);
  const cudaStream_t st = (cudaStream_t)stream;
  // segments of at least 8 rows, up to 32 per stripe
  const dim3 cgrid((unsigned)((nx + 31) / 32));
  cudaError_t e = ny >= 256  ? seb::launch_pdl(nn_cols_kernel<32>, cgrid, dim3(32 * 32), 0, st, elev, nx, ny, near_row)
                  : ny >= 128 ? seb::launch_pdl(nn_cols_kernel<16>, cgrid, dim3(32 * 16), 0, st, elev, nx, ny, near_row)
                              : seb::launch_pdl(nn_cols_kernel<8>, cgrid, dim3(32 * 8), 0, st, elev, nx, ny, near_row);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(nn_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(nx * sizeof(int32_t)));
  if (e == cudaSuccess)
    e = seb::launch_pdl(nn_rows_kernel, dim3((unsigned)ny), dim3(kRowThreads), nx * sizeof(int32_t), st, elev,
                        near_row, nx, ny, W, out, src);
  if (e != cudaSuccess) {
    seb::set_error("seb_inpaint_nearest launch: %s", cudaGetErrorString(e));
    return SEB_ERR_CUDA;
  }
  return SEB_OK;
}
