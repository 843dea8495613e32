// Internal declarations shared by the libseb translation units (not part of the ABI).
#pragma once

#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "seb.h"

namespace seb {

// NVTX range around one entry point (header-only NVTX 3: a no-op unless a profiler such as
// ncu --nvtx attaches), named after the C function.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define SEB_RANGE() ::seb::NvtxRange seb_nvtx_range_(__func__)

// Thread layout of a CTA: 256 threads, each owning kG = 4 adjacent cells of one row, with
// 2^log_tpr threads per row.  log_tpr = 3: 32 x 32 cells (interior); 1: 8 x 128 (narrow
// column bands); 5: 128 x 8 (narrow row bands).  A warp always spans the full tile width.
constexpr int kThreads = 256;
constexpr int kG = 4;
constexpr int kMaxStageRows = 384;  // staged rows of any layout: 128 + 2 * 127 < 384

__host__ __device__ inline int stage_w(int log_tpr, int rx) { return ((kG << log_tpr) + 2 * rx) | 1; }
__host__ __device__ inline int stage_h(int log_tpr, int ry) { return (kThreads >> log_tpr) + 2 * ry; }

constexpr int kMaxPairs = 128;  // n_yaw <= 256; bins k and k + n_yaw/2 share a footprint
constexpr int kMaxRuns = 3072;  // total row runs over all yaw pairs
constexpr int kMaxRects = 12;   // rolling update: up to 4 bands, each split by layout

// Footprint tables of every yaw pair (Algorithm 1, FindEllipticalPoints, restated as row
// runs).  Passed to the kernels as a __grid_constant__ parameter, so it lives in the
// constant bank and its uniform reads are broadcast.
struct Tables {
  int32_t n_pairs;
  int32_t narrow;                    // (max N * max reach)^2 < 2^31: int32 covariance numerators
  int32_t rx, ry;                    // largest |di| / |dj| over every footprint
  int32_t run_start[kMaxPairs + 1];  // runs of pair p: [run_start[p], run_start[p+1])
  int32_t n_min[kMaxPairs];          // known cells needed to assess (per bin)
  float inv_n[kMaxPairs];            // 1 / N of the complete footprint, correctly rounded
  int32_t mom[kMaxPairs][6];         // N, sum di, sum dj, sum di^2, sum di dj, sum dj^2
  float cos_t[kMaxPairs], sin_t[kMaxPairs];  // heading of bin p (bin p + K/2 negates both)
  uint32_t runs[kMaxRuns];           // packed (dj + 128) | (lo + 128) << 8 | (hi + 128) << 16
};

struct Rect {
  int32_t x0, y0, w, h;  // cells stored: [x0, x0 + w) x [y0, y0 + h)
  int32_t tx, ty;        // origin of the tile grid (<= x0, y0)
  int32_t log_tpr;       // layout (see the kernels)
};

// Everything else a launch needs (by value, in the parameter bank).
struct Launch {
  const void* elev;  // logical [ny][nx]
  int32_t nx, ny;
  int32_t ring_x, ring_y;
  float* out;  // [5][K][ny][nx] physical (ring-indexed)
  uint8_t* flags;
  int64_t plane;  // nx * ny
  int32_t n_yaw;
  float res;
  float kappa_max, phi_x_max, phi_y_max;
  float inv_kappa_max, inv_phi_x_max, inv_phi_y_max;
  float w0, w1, w2;
  float gap_fp64;
  int32_t narrow_moments;  // N * sum di^2 etc. fit in int32
  int32_t n_req;          // rectangles of cells to recompute, before tiling
  Rect req[4];
  int32_t phase_x, phase_y;  // window origin mod 4 / mod 2 (global alignment of cell blocks)
  int32_t vec4;              // whole 4-cell blocks may be stored with 16-byte stores
  int32_t early;             // a later launch of a shift batch (seb_map_shift_batch): see the kernel
  int32_t tma;               // stage the tile with one TMA copy per CTA (set by the launcher)
  int32_t all_masked;        // every row run takes the masked moment path (rolling-shift bands)
  int32_t pairs_alloc;       // float2 slots of the staged vertical pairs (bounds checks of SEB_DEBUG builds)
  int32_t q_flush;           // row runs after which the packed missing-point moments are flushed (0: never)
  // SEB_BF16_TILED windows: the FP32 bases [TY][TX] and the window's phase in the 16-cell tiles
  const float* tile_base;
  int32_t base_tx, base_px, base_py;
  int32_t n_rects;
  Rect rects[kMaxRects];
  int32_t tile_start[kMaxRects + 1];
  int32_t tiles_x[kMaxRects];
  uint32_t* err;
  unsigned long long* counters;  // [0] FP64 eigen-solves, [1] degenerate cells
  // Optional (NULL = off): CTAs of tiles whose flag is 0 exit at once (one flag per tile of a
  // single-rectangle launch), and only cells whose mask byte is set ([ny][nx]) are stored.
  const uint8_t* tile_active;
  const uint8_t* store_mask;
};

// Control block at the start of every workspace.
struct Control {
  uint32_t err;
  uint32_t pad;
  unsigned long long n_fp64;
  unsigned long long n_degenerate;
};
constexpr size_t kControlBytes = 256;

enum DeviceError : uint32_t {
  kErrLaunchShape = 1u,    // blockDim / grid disagree with the launch record
  kErrStageTimeout = 2u,   // a CTA's bounded wait for its staged tile (TMA copy) ran out
  kErrBounds = 16u,        // SEB_DEBUG builds: an index check failed (the access was skipped)
};

// Index checks of SEB_DEBUG builds (-DSEB_DEBUG, paper_2503_02412_gb300.build(debug=True)):
// a failed check raises kErrBounds in the launch's error word and the guarded access is skipped;
// release builds compile the checks away and always take the access.
#ifdef SEB_DEBUG
#define SEB_IN_BOUNDS(err, cond) ((cond) ? true : (atomicOr((err), ::seb::kErrBounds), false))
#else
#define SEB_IN_BOUNDS(err, cond) true
#endif

// Continuous-pose query: the yaw-0 footprint lattice (a __grid_constant__ parameter).
constexpr int kMaxLattice = 256;
struct QTab {
  int32_t n, n_min;
  int8_t di[kMaxLattice], dj[kMaxLattice];
};

struct QLaunch {
  const void* elev;
  int32_t nx, ny;
  float res;
  double oi, oj;
  const float* poses;
  int64_t n;
  float* out;
  uint8_t* flags;
  float* saved;
  const float* gout;
  float* gpose;
  float kappa_max, phi_x_max, phi_y_max;
  float w0, w1, w2;
  float gap_fp64;
};

// SEB_BF16_TILED windows: 16 x 16 world-aligned tiles.
constexpr int kBaseTile = 16;
inline int tiled_tx(int nx) { return (nx + kBaseTile - 1) / kBaseTile + 1; }
inline size_t tiled_base_offset(int nx, int ny) { return ((size_t)nx * ny * 2 + 255) & ~(size_t)255; }

// Host helpers (seb_tables.cpp).  build_tables and build_lattice use no heap memory.
int build_tables(const seb_params& p, Tables* T, int32_t* total_runs);
// The yaw-0 lattice of the continuous-pose query: the offsets of yaw pair 0 in row-run order.
int build_lattice(const Tables& T, QTab* Q);
int validate_params(const seb_params& p);
size_t out_bytes(const seb_params& p);
size_t flags_bytes(const seb_params& p);

// Continuous-pose query (seb_query.cu): the lattice and the launch record of a parameter set
// (validated like seb_query_poses, heap-free), and the launcher.
int query_setup(const seb_params& p, const void* elev, int64_t origin_i, int64_t origin_j, const float* poses,
                int64_t n, QTab* Q, QLaunch* L);
cudaError_t launch_query(const QTab& Q, const QLaunch& L, int elev_dtype, bool backward, cudaStream_t st);

// Kernel launchers (seb_assess.cu).
// cuTensorMapEncodeTiled through the runtime's driver entry point (NULL when unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

cudaError_t launch_assess(const Tables& T, const Launch& L, int elev_dtype, int precision,
                          cudaStream_t stream);
cudaError_t launch_copy_out(const Launch& L, float* out_dev, uint8_t* flags_dev,
                            cudaStream_t stream);
void launch_defaults(const seb_params& p, const Tables& T, Launch* L);
void launch_request(Launch& L, int x0, int y0, int w, int h);
void launch_set_origin(Launch& L, int64_t origin_i, int64_t origin_j);

void set_error(const char* fmt, ...);

#ifdef __CUDACC__
// Programmatic dependent launch.  A kernel launched with launch_pdl may be scheduled while the
// stream's previous kernel drains; it calls pdl_entry() before any global memory access, which
// waits until that kernel has completed and its writes are visible (for an ordinary launch it
// returns at once), and lets the next such kernel be scheduled in turn.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  return e != cudaSuccess ? e : cudaGetLastError();
}
#endif

}  // namespace seb
