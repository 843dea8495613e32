// Internal declarations shared by the libseb translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "seb.h"

namespace seb {

// Tile of output cells per CTA and the thread layout inside it: 256 threads, each owning
// G = 4 adjacent cells of one row (8 threads per row, 32 rows).
constexpr int kTileW = 32;
constexpr int kTileH = 32;
constexpr int kThreads = 256;
constexpr int kG = 4;

constexpr int kMaxPairs = 128;  // n_yaw <= 256; bins k and k + n_yaw/2 share a footprint
constexpr int kMaxRuns = 3072;  // total row runs over all yaw pairs
constexpr int kMaxRects = 4;    // rolling update: two column bands + two row bands

// Footprint tables of every yaw pair (Algorithm 1, FindEllipticalPoints, restated as row
// runs).  Passed to the kernels as a __grid_constant__ parameter, so it lives in the
// constant bank and its uniform reads are broadcast.
struct Tables {
  int32_t n_pairs;
  int32_t rx, ry;                    // largest |di| / |dj| over every footprint
  int32_t run_start[kMaxPairs + 1];  // runs of pair p: [run_start[p], run_start[p+1])
  int32_t n_min[kMaxPairs];          // known cells needed to assess (per bin)
  int32_t mom[kMaxPairs][6];         // N, sum di, sum dj, sum di^2, sum di dj, sum dj^2
  float cos_t[kMaxPairs], sin_t[kMaxPairs];  // heading of bin p (bin p + K/2 negates both)
  uint32_t runs[kMaxRuns];           // packed (dj + 128) | (lo + 128) << 8 | (hi + 128) << 16
};

struct Rect {
  int32_t x0, y0, w, h;
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
  float w0, w1, w2;
  float gap_fp64;
  int32_t n_rects;
  Rect rects[kMaxRects];
  int32_t tile_start[kMaxRects + 1];
  int32_t tiles_x[kMaxRects];
  int32_t sw, sh;  // staged tile: sw columns (odd, for conflict-free banks) x sh rows
  uint32_t* err;
  unsigned long long* counters;  // [0] FP64 eigen-solves, [1] degenerate cells
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
  kErrLaunchShape = 1u,  // blockDim / grid disagree with the launch record
};

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

// Host helpers (seb_tables.cpp).
int build_tables(const seb_params& p, Tables* T, int32_t* total_runs);
int validate_params(const seb_params& p);
size_t out_bytes(const seb_params& p);
size_t flags_bytes(const seb_params& p);

// Kernel launchers (seb_assess.cu).
cudaError_t launch_assess(const Tables& T, const Launch& L, int elev_dtype, int precision,
                          cudaStream_t stream);
cudaError_t launch_copy_out(const Launch& L, float* out_dev, uint8_t* flags_dev,
                            cudaStream_t stream);
size_t assess_smem_bytes(const Tables& T);

void set_error(const char* fmt, ...);

}  // namespace seb
