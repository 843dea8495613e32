/*
 * libseb: SE(2)-grid traversability assessment on sm_103a (SEB-Naver, arXiv 2503.02412).
 *
 * For every cell (c, r) of a robot-centric elevation window and every yaw bin k of n_yaw
 * (theta_k = 2 pi k / n_yaw), the library gathers the elevation cells under the yaw-rotated
 * vehicle footprint, fits their 3x3 covariance, takes the eigenvector of the smallest
 * eigenvalue as the terrain normal z_b, builds the body frame of Eqs. 2-3 and scores risk
 * with the curvature and the separate fore-aft / lateral tilt limits of Algorithm 1
 * (Sec. V-B).  The window is a rolling map (Sec. V-A, Eq. (pm)): a move recomputes only
 * the cells whose footprint touches cells that entered or left the window.
 *
 * Conventions shared by every entry point:
 *   - elevation: row-major [ny][nx], x fastest, NaN = unknown; cell (c, r) has its centre
 *     at world ((o_i + c + 1/2) res, (o_j + r + 1/2) res), (o_i, o_j) the integer grid index
 *     of the window origin (Eq. (pm)).  Cells outside the window are unknown.
 *   - outputs: SoA float32 out[ch][k][r][c], ch = z, pitch, roll, roughness, risk, plus
 *     uint8 flags[k][r][c].  In the map's own buffers r and c are ring-indexed:
 *     physical = (logical + ring offset) mod n (see seb_view).
 *   - z = height of the fitted plane at the cell centre (m); pitch = asin(b3^T x_b),
 *     roll = asin(b3^T y_b) (rad, signed; Algorithm 1 uses their magnitudes);
 *     roughness = lambda_min / trace(Cov) (the curvature kappa_ter of Algorithm 1);
 *     risk in [0, 1], 1 = obstacle.
 *   - memory: every device buffer is owned by the caller.  The library never allocates
 *     device memory and never synchronises, except where an entry point says so.
 *   - streams: each call enqueues on the map's stream (seb_map_set_stream), or on the
 *     stream argument for the map-free calls; NULL is the legacy default stream.
 *   - errors: every call returns SEB_OK (0) or a negative SEB_ERR_* code and records a
 *     message retrievable with seb_last_error.  Kernels never trap: device-side problems
 *     set an error word that seb_map_check reads.
 */
#ifndef SEB_H_
#define SEB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SEB_OK 0
#define SEB_ERR_INVALID_ARG (-1)  /* NULL pointer, non-positive size, bad enum */
#define SEB_ERR_BAD_SHAPE (-2)    /* n_yaw odd, footprint too large for the tables */
#define SEB_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define SEB_ERR_TIMEOUT (-4)      /* a bounded host wait ran out */
#define SEB_ERR_DEVICE_FAULT (-5) /* a kernel raised the device error word */
#define SEB_ERR_WORKSPACE (-6)    /* workspace too small or misaligned */

/* Footprint shapes (Algorithm 1 uses an ellipse; the rectangle is the vehicle outline). */
#define SEB_RECT 0
#define SEB_ELLIPSE 1

/* Elevation storage types. */
#define SEB_F32 0
#define SEB_BF16 1
#define SEB_F16 2
/* BF16 height offsets from an FP32 base per 16 x 16 world-aligned tile: a window's buffer holds
 * the BF16 offsets [ny][nx] (logical order), then, at byte offset seb_tiled_base_offset(nx, ny),
 * the FP32 bases [TY][TX], TX = (nx + 15) / 16 + 1, TY = (ny + 15) / 16 + 1.  Cell (c, r) of a
 * window at origin (o_i, o_j) has the height base[(r + py) / 16][(c + px) / 16] + offset[r][c]
 * (FP32 sum), px = o_i mod 16, py = o_j mod 16 (0..15): the base belongs to the world tile of the
 * cell, so windows cut from one encoding of a world agree cell by cell.  Maps only (the
 * continuous query and the surrogate read FP32/BF16/FP16 heights). */
#define SEB_BF16_TILED 3

/* Moment accumulation. */
#define SEB_PLAIN_F32 0   /* FP32 sums about the footprint's reference height */
#define SEB_COMPENSATED 1 /* FP32 Neumaier-compensated sums about the same reference */

/* Output flags. */
#define SEB_FLAG_UNKNOWN 1    /* fewer than n_min known footprint cells */
#define SEB_FLAG_OBSTACLE 2   /* risk == 1 (an explicit obstacle, Algorithm 1) */
#define SEB_FLAG_DEGENERATE 4 /* normal undefined: eigen-gap ~ 0, n_z <= 1e-6 or yaw || normal */
#define SEB_FLAG_FP64 8       /* eigen-solve redone in FP64 (small relative eigen-gap) */
#define SEB_FLAG_SURROGATE 16 /* value predicted by the learned surrogate (seb_sur_infer) */

#define SEB_N_CH 5 /* z, pitch, roll, roughness, risk */

typedef struct CUstream_st* seb_stream_t; /* the same type as cudaStream_t */
typedef struct seb_map seb_map;

/*
 * Assessment parameters (Algorithm 1's inputs: footprint (e_x, e_y), w_r, kappa_max,
 * phi_x_max, phi_y_max).  Footprint membership of an integer cell offset (di, dj) at yaw
 * theta, with (u, v) = R(-theta)(di, dj) in cell units, a = length / (2 res),
 * b = width / (2 res): rectangle |u| <= a + 1e-6 and |v| <= b + 1e-6; ellipse
 * (u/a)^2 + (v/b)^2 <= 1 + 1e-6.  Bins k and k + n_yaw/2 share one footprint.
 */
typedef struct {
  int32_t nx, ny;     /* window size in cells (>= 1) */
  int32_t n_yaw;      /* yaw bins, even, 2..256 */
  float res;          /* cell size (m) */
  int32_t shape;      /* SEB_RECT | SEB_ELLIPSE */
  float length;       /* footprint extent along the heading (m) */
  float width;        /* footprint extent across the heading (m) */
  float kappa_max;    /* roughness limit (default 0.1) */
  float phi_x_max;    /* fore-aft tilt limit, rad (default 0.52, Sec. VII-B) */
  float phi_y_max;    /* lateral tilt limit, rad (default 0.52, Sec. VII-B) */
  float w[3];         /* risk weights for (kappa, |pitch|, |roll|) ratios (default 1/3 each) */
  int32_t n_min;      /* minimum known footprint cells; 0 = max(3, ceil(N_k / 2)) per bin */
  int32_t elev_dtype; /* SEB_F32 | SEB_BF16 | SEB_F16 | SEB_BF16_TILED */
  int32_t precision;  /* SEB_PLAIN_F32 | SEB_COMPENSATED */
  float gap_fp64;     /* relative eigen-gap (lambda_mid - lambda_min) / trace below which the
                         covariance and eigen-solve are redone in FP64 (default 1e-2) */
} seb_params;

/* Device pointers into a map's workspace, valid until the next update/shift/destroy. */
typedef struct {
  float* out;         /* [SEB_N_CH][n_yaw][ny][nx], ring-indexed */
  uint8_t* flags;     /* [n_yaw][ny][nx], ring-indexed */
  int32_t ring_x;     /* physical column = (logical + ring_x) mod nx */
  int32_t ring_y;     /* physical row = (logical + ring_y) mod ny */
  int64_t origin_i;   /* grid index of the window origin (Eq. (pm)) */
  int64_t origin_j;
  size_t out_offset;  /* byte offsets of out / flags from the workspace base */
  size_t flags_offset;
  int64_t last_cells; /* SE(2) cells (c, r, k) the last update/shift recomputed */
} seb_view;

/* Fills p with the defaults above (c1 geometry: 100 x 100 at 0.1 m, 36 bins, 0.6 x 0.4 m). */
void seb_params_default(seb_params* p);

/* Message for a status code (static storage). */
const char* seb_status_string(int status);

/* Last error message of the calling thread, or of a map when m is not NULL. */
const char* seb_last_error(const seb_map* m);

/*
 * Footprint table of yaw bin k (host only, no GPU needed): writes up to cap offsets
 * (di, dj) in row-run order (dj ascending, di ascending) and returns the count, or a
 * negative status.  Used to check the tables against an independent enumeration.
 */
int seb_footprint_table(const seb_params* p, int32_t k, int32_t* di, int32_t* dj, int32_t cap);

/* Bytes of device workspace a map needs: the SoA outputs, the flags and a small control
 * block (the device error word and counters). */
size_t seb_workspace_bytes(const seb_params* p);

/* Bytes of one elevation window of p->nx x p->ny cells in p->elev_dtype (0 for bad params), and
 * the byte offset of the bases in a SEB_BF16_TILED window (the BF16 offsets rounded up to 256). */
size_t seb_window_bytes(const seb_params* p);
size_t seb_tiled_base_offset(int32_t nx, int32_t ny);

/*
 * Encodes an FP32 elevation window (device [ny][nx], NaN = unknown, logical order, origin
 * (origin_i, origin_j)) as a SEB_BF16_TILED window in out_dev (device, 256-byte aligned,
 * seb_window_bytes bytes): per 16 x 16 world-aligned tile the base is the midpoint of the tile's
 * smallest and largest known height (0 without one), and each offset is the BF16 value nearest
 * to height - base (NaN stays NaN).  Encode a whole world once and cut windows from it when maps
 * roll: re-encoding each window gives tiles cut by the window edge other bases.
 */
int seb_encode_bf16_tiled(const float* elev_dev, int32_t nx, int32_t ny, int64_t origin_i, int64_t origin_j,
                          void* out_dev, seb_stream_t stream);

/*
 * Creates a map over caller-owned device workspace (>= seb_workspace_bytes, 256-byte
 * aligned).  Builds the footprint tables on the host; allocates host memory only.
 * Outputs are undefined until the first seb_map_update.
 */
int seb_map_create(const seb_params* p, void* workspace_dev, size_t bytes, seb_stream_t stream,
                   seb_map** out);

/* Frees the host handle.  The workspace stays the caller's. */
int seb_map_destroy(seb_map* m);

/* Sets the stream later calls enqueue on. */
int seb_map_set_stream(seb_map* m, seb_stream_t stream);

/*
 * Full rebuild (Algorithm 1 for every SE(2) cell).  elev_dev: device [ny][nx] in the map's
 * elev_dtype, logical order, at least 16-byte aligned; read only during the call's kernels.
 * (origin_i, origin_j): grid index of the window origin.  Sets the ring offsets to the origin
 * modulo the map size, so that a cell's physical row and column are its grid indices modulo
 * (ny, nx) for the whole life of the map (a rolling map over a torus, Sec. V-A).
 */
int seb_map_update(seb_map* m, const void* elev_dev, int64_t origin_i, int64_t origin_j);

/*
 * Rolling update (Sec. V-A): the window moves to (origin_i, origin_j); elev_dev holds the
 * whole new window in logical order.  The ring offsets advance by the move, and only the
 * cells whose footprint can see a cell that entered or left the window are recomputed:
 * a band of |move| + reach cells on the entering side and of reach cells on the leaving
 * side, per axis (reach = largest |offset| of any footprint along that axis), each widened to
 * whole 4 x 2 cell blocks in world alignment (the cells of a block share a reference height).
 * Every other cell keeps its stored value, which is bit-identical to a full rebuild.  A move of
 * at least the window size in either axis falls back to a full rebuild.
 */
int seb_map_shift(seb_map* m, const void* elev_dev, int64_t origin_i, int64_t origin_j);

/*
 * n rolling updates in order (Sec. V-A), with results bit-identical to n seb_map_shift calls:
 * elev_dev[i] (a host array of n device pointers) is the whole window of the i-th move, and
 * origins[2 i], origins[2 i + 1] (a host array) its origin.  All n windows must be written, in
 * the map's stream order, before this call; none may be overwritten until the call's work has
 * completed.  Each launch after the first may then stage and compute while the previous one is
 * still finishing, and it stores only after that one completes, which fills the GPU across the
 * moves.  view.last_cells afterwards counts the cells recomputed by the whole batch.  On an
 * error the moves before the failing one have been applied.
 */
int seb_map_shift_batch(seb_map* m, const void* const* elev_dev, const int64_t* origins, int32_t n);

/* Pointers and ring offsets of the current outputs. */
int seb_map_view(const seb_map* m, seb_view* v);

/* Copies the outputs to caller buffers in logical order (undoing the ring):
 * out_dev [SEB_N_CH][n_yaw][ny][nx] float32, flags_dev [n_yaw][ny][nx] (either may be NULL). */
int seb_map_copy_out(const seb_map* m, float* out_dev, uint8_t* flags_dev);

/*
 * Synchronises the map's stream (bounded wait of timeout_ms; <= 0 waits without bound),
 * reads the device error word and the counters, and clears them.  n_fp64 / n_degenerate
 * (may be NULL) receive the number of eigen-solves redone in FP64 and of degenerate cells
 * since the last check.  Returns SEB_ERR_DEVICE_FAULT if a kernel raised the error word.
 */
int seb_map_check(seb_map* m, int32_t timeout_ms, int64_t* n_fp64, int64_t* n_degenerate);

/*
 * Continuous-pose query (a differentiable form of the same assessment): for each pose
 * (x, y, yaw) in world metres/radians, the yaw-0 footprint lattice {(di res, dj res)} is
 * rotated by yaw and translated to (x, y); each lattice point takes the bilinear elevation
 * of the four surrounding cell centres (unknown if any of them is NaN or outside the
 * window); then covariance, normal, frame, outputs and risk follow Algorithm 1 as above,
 * with z the fitted-plane height at (x, y).
 *   poses_dev [n][3] float32; out_dev [n][SEB_N_CH] float32; flags_dev [n] uint8;
 *   saved_dev [n][SEB_QUERY_SAVED] float32 or NULL: per-pose state the backward reuses.
 */
#define SEB_QUERY_SAVED 16
int seb_query_poses(const seb_params* p, const void* elev_dev, int64_t origin_i, int64_t origin_j,
                    const float* poses_dev, int64_t n, float* out_dev, uint8_t* flags_dev,
                    float* saved_dev, seb_stream_t stream);

/*
 * Hand-written adjoint of seb_query_poses: grad_pose[i] = sum_ch grad_out[i][ch] *
 * d out[i][ch] / d pose[i] over the five output channels (grad_out [n][SEB_N_CH]).  The set of
 * known lattice points is held fixed; the risk gradient is 0 on the clamped (risk = 1)
 * branches and sign(0) = 0 at |.| kinks.  saved_dev may be NULL (recomputed).
 */
int seb_query_poses_backward(const seb_params* p, const void* elev_dev, int64_t origin_i,
                             int64_t origin_j, const float* poses_dev, const float* saved_dev,
                             const float* grad_out_dev, float* grad_pose_dev, int64_t n,
                             seb_stream_t stream);

/*
 * SE(2) grid lookup (Sec. VI: the planner reads Risk and the signed distance field at
 * continuous states by trilinear interpolation of the grid, with the yaw handled on SO(2)).
 * A seb_grid names one float32 channel [n_yaw][ny][nx] on the device, ring-indexed like the
 * map's outputs: the value of cell (c, r) and yaw bin k sits at world
 * ((origin_i + c + 1/2) res, (origin_j + r + 1/2) res, 2 pi k / n_yaw) and is stored at
 * data[k][(r + ring_y) mod ny][(c + ring_x) mod nx].  The grid is read, never written.
 */
typedef struct {
  const float* data;
  int32_t nx, ny, n_yaw;
  int32_t ring_x, ring_y;
  int64_t origin_i, origin_j;
  float res;
} seb_grid;

/* Fills g with output channel `channel` (0..SEB_N_CH-1: z, pitch, roll, roughness, risk) of
 * the map; valid until the map's next update or shift.  SEB_ERR_INVALID_ARG before the first
 * update or for a bad channel. */
int seb_map_grid(const seb_map* m, int32_t channel, seb_grid* g);

/*
 * Trilinear lookup at poses_dev [n][3] (x, y, yaw in world metres / radians):
 *   u = x / res - origin_i - 1/2,  v = y / res - origin_j - 1/2,  w = yaw n_yaw / (2 pi)
 *   reduced to [0, n_yaw).  A pose is inside when 0 <= u <= nx - 1 and 0 <= v <= ny - 1.
 *   Its cell is (c0, r0) = (min(floor u, nx - 2), min(floor v, ny - 2)) and its yaw bins are
 *   k0 = floor w, k1 = (k0 + 1) mod n_yaw (the SO(2) wrap).  The value blends the 8 corners
 *   with weights (1 - a or a)(1 - b or b)(1 - t or t), a = u - c0, b = v - r0, t = w - k0;
 *   the gradient is the derivative of the same blend in world units (d/dx, d/dy, d/dyaw).
 * val_dev [n] is required; grad_dev [n][3] and flags_dev [n] may be NULL.  Outside the window:
 * value `fill`, gradient 0 and SEB_FLAG_UNKNOWN; a NaN value (an unknown corner) also sets
 * SEB_FLAG_UNKNOWN.  A pose with a non-finite coordinate or |yaw| > 1e4 rad counts as outside.
 * Needs nx, ny >= 2 and 1 <= n_yaw <= 4096 (else SEB_ERR_BAD_SHAPE); poses are read once, no
 * state is kept.
 */
int seb_se2_lookup(const seb_grid* g, const float* poses_dev, int64_t n, float fill, float* val_dev,
                   float* grad_dev, uint8_t* flags_dev, seb_stream_t stream);

/* Adjoint of seb_se2_lookup: grad_pose_dev [n][3] = grad_val_dev[i] * d value_i / d pose_i
 * (0 outside the window). */
int seb_se2_lookup_vjp(const seb_grid* g, const float* poses_dev, int64_t n, const float* grad_val_dev,
                       float* grad_pose_dev, seb_stream_t stream);

/*
 * Signed distance field of the obstacle set (Sec. VI: the planner's collision term reads an
 * SDF over SE(2) whose value at a state is the distance to the edge of the nearest region,
 * negative inside obstacles; the paper builds it from the risk map).  Per yaw bin, obstacles
 * are the cells of `risk` with risk >= risk_obstacle (NaN counts as an obstacle; 1 selects
 * Algorithm 1's explicit obstacles, unknown cells included); distances are Euclidean between
 * cell centres of that bin's (x, y) plane, in metres, in the window's logical order:
 *   sdf = res * (distance to the nearest obstacle - distance to the nearest free cell),
 * clamped to [-clamp, clamp] (clamp >= 0; INFINITY for none; an empty set contributes +inf).
 * sdf_dev [n_yaw][ny][nx] float32 is written ring-indexed like risk, so a seb_grid with risk's
 * fields and data = sdf_dev describes it; it may not alias risk.  work_dev: caller-owned,
 * 4-byte aligned, at least seb_sdf_workspace_bytes(nx, ny, n_yaw) bytes.  Exact (integer)
 * squared distances; sides up to 16384 cells.
 */
size_t seb_sdf_workspace_bytes(int32_t nx, int32_t ny, int32_t n_yaw);
int seb_risk_sdf(const seb_grid* risk, float risk_obstacle, float clamp, void* work_dev, size_t work_bytes,
                 float* sdf_dev, seb_stream_t stream);

/*
 * Nearest-neighbour inpainting of an elevation map (Sec. V-A: the map is inpainted before the
 * traversability pass; Sec. VII-B: nearest-neighbour filling).  elev_dev [ny][nx] float32 in
 * logical order, NaN = unknown.  Every unknown cell of out_dev [ny][nx] takes the value of the
 * known cell whose centre is nearest (Euclidean); among equally near known cells the smallest
 * column, then the smallest row wins; known cells are copied.  max_cells > 0 leaves unknown
 * the cells whose nearest known cell is farther than max_cells cells; a map without known
 * cells stays unknown.  source_dev [ny][nx][2] int32 (may be NULL) receives the (row, column)
 * each value came from, (-1, -1) where none.  out_dev may not alias elev_dev.  work_dev:
 * caller-owned, 4-byte aligned, seb_inpaint_workspace_bytes(nx, ny) bytes.  Sides up to 16384.
 */
size_t seb_inpaint_workspace_bytes(int32_t nx, int32_t ny);
int seb_inpaint_nearest(const float* elev_dev, int32_t nx, int32_t ny, int32_t max_cells, void* work_dev,
                        size_t work_bytes, float* out_dev, int32_t* source_dev, seb_stream_t stream);

/*
 * Elevation-map update from LiDAR scans (Sec. V-A).  The map is a robot-centred window of
 * nx x ny cells at res metres, each holding a height and its variance (NaN = unknown), stored
 * at [world row mod ny][world column mod nx].  seb_elev_integrate takes one scan and, in the
 * order of Sec. V-A:
 *  1. sets the window origin to the robot's cell minus (nx / 2, ny / 2) (Eq. pm) and clears
 *     the cells that were not in the previous window;
 *  2. ray casting: for every point whose (x, y) lies in the window, clears each cell that the
 *     segment sensor -> point crosses in (x, y), the point's own cell excepted, when the cell's
 *     height exceeds the ray's highest height over it plus clear_margin;
 *  3. ignores points outside the window and keeps those whose body-frame height lies in
 *     [z_min, z_max]; a kept point has world height z = b3^T (R_B (R_BS p + p_BS) + p_B) and
 *     variance J_S^T Sigma_S J_S + J_R^T Sigma_R J_R + J_B^T Sigma_B J_B, J_S = (R_B R_BS)^T b3,
 *     J_R = (R_BS p + p_BS)^ R_B^T b3 (right perturbation of R_B), J_B = -b3;
 *  4. fuses the kept points per cell (one-dimensional Kalman filter, information form) against
 *     the estimate (h, s2) from before this fusion: a point with (z - h) / sqrt(s2) > gate is
 *     above the gate, one within [-gate, gate] inside, one below is dropped; a cell with points
 *     above the gate is reset to their fusion, otherwise its estimate is fused with the points
 *     inside; an unknown cell takes the fusion of all its points.
 * The result does not depend on the order of the points.  Matrices are row-major float32;
 * points_dev [n][3] float32 in the sensor frame, n <= max_points.  The workspace is
 * caller-owned, 256-byte aligned device memory of seb_elev_workspace_bytes() bytes.
 */
typedef struct {
  int32_t nx, ny;
  float res;
  float z_min, z_max;   /* body-frame height filter (m) */
  float gate;           /* Mahalanobis gate (standard deviations), default 2.5 */
  float clear_margin;   /* ray casting clears cells higher than the ray by more than this (m) */
} seb_elev_params;

typedef struct {
  float R_B[9], p_B[3];     /* body -> world rotation and body position */
  float R_BS[9], p_BS[3];   /* sensor -> body rotation and sensor position in the body frame */
  float Sigma_S[9];         /* point covariance (sensor model) */
  float Sigma_R[9];         /* attitude covariance */
  float Sigma_B[9];         /* position covariance */
} seb_scan_pose;

typedef struct {
  float* height;            /* [ny][nx], storage order (see above) */
  float* variance;
  int32_t ring_x, ring_y;   /* storage column = (logical column + ring_x) mod nx, same for rows */
  int64_t origin_i, origin_j;
} seb_elev_view;

typedef struct seb_elev seb_elev;

void seb_elev_params_default(seb_elev_params* p);
size_t seb_elev_workspace_bytes(const seb_elev_params* p, int64_t max_points);
int seb_elev_create(const seb_elev_params* p, int64_t max_points, void* workspace_dev, size_t bytes,
                    seb_stream_t stream, seb_elev** out);
int seb_elev_destroy(seb_elev* e);
int seb_elev_set_stream(seb_elev* e, seb_stream_t stream);
int seb_elev_integrate(seb_elev* e, const seb_scan_pose* pose, const float* points_dev, int64_t n);
int seb_elev_view_get(const seb_elev* e, seb_elev_view* v);
/* Heights / variances in logical (window) order [ny][nx]; either pointer may be NULL. */
int seb_elev_copy_out(const seb_elev* e, float* height_dev, float* variance_dev);

/*
 * Learned surrogate (not in the paper, which names learned traversability as less reliable
 * than geometry, Sec. II-A): a BF16 convolutional network predicting, per cell and yaw pair,
 * (z - z_cell, pitch, roll, risk) of the assessment above from an elevation patch.  Slope
 * features (central differences) -> 4 x [3x3 conv, 32 channels, dilations 1, 2, 4, 8, ReLU]
 * -> 1x1 head to 4 x n_yaw/2 outputs; receptive field 31 cells (a 48 x 48 crop, the centre
 * of a 64 x 64 patch, gives the 16 x 16 centre cells).  Weights and stored activations BF16,
 * accumulation and gradients FP32, FP32 master weights with Adam.  Trained on the GPU on
 * patches the exact kernel labels; run fully convolutionally over a map with the exact kernel
 * as fallback near unknown cells, step edges and the map border.
 *
 * The handle lives on caller workspace (>= seb_sur_workspace_bytes, 256-byte aligned) sized
 * for training batches of up to max_batch patches and for inference on a p->nx x p->ny map;
 * p gives the exact assessment the network imitates (p->elev_dtype must be SEB_F32).
 * seb_sur_view reports byte offsets of the parts of the workspace (weights for save / load,
 * batch buffers, activations) so a caller can inspect or checkpoint them.
 */
typedef struct seb_sur seb_sur;
typedef struct {
  int64_t n_params;           /* FP32 master parameters */
  int32_t n_out;              /* 2 * n_yaw head outputs */
  int32_t max_batch;
  size_t master, adam_m, adam_v, grad, weights_bf16;  /* [n_params] each */
  size_t features;            /* [max_batch][46][46][2] BF16 */
  size_t labels;              /* [max_batch][16][16][n_out] FP32 (NaN = no label) */
  size_t act[4];              /* [max_batch][side][side][32] BF16, sides 44, 40, 32, 16 */
  size_t dact[4];             /* FP32 gradients of the same */
  size_t pred, dpred;         /* [max_batch][16][16][n_out] FP32 */
  size_t map_features, map_act[4], mask, tiles, partials, loss_partials, totals;
  int64_t off_w[4], off_b[4], off_wh, off_bh;  /* parameter offsets (elements) */
} seb_sur_view;

size_t seb_sur_workspace_bytes(const seb_params* p, int32_t max_batch);
int seb_sur_create(const seb_params* p, int32_t max_batch, void* workspace_dev, size_t bytes,
                   seb_stream_t stream, seb_sur** out);
int seb_sur_destroy(seb_sur* h);
int seb_sur_set_stream(seb_sur* h, seb_stream_t stream);
int seb_sur_view_get(const seb_sur* h, seb_sur_view* v);
/* Engine of the 32 -> 32 convolutions, forward and backward: SEB_SUR_TCGEN05 (default; tensor
 * cores: tcgen05.mma implicit GEMMs with BF16 operands and FP32 accumulation in tensor memory;
 * forward M = 128 output pixels, N = 32, K = 288; input gradient M = 128 input pixels, N = 32,
 * K = 288; weight gradient M = 3 x 128 (tap, channel) rows, N = 32, K = the pixels; the FP32
 * upstream gradient enters as a BF16 high part plus a BF16 low part) or SEB_SUR_SIMT (FP32 CUDA
 * cores).  The first layer (2 input channels) and the 1x1 head run on the CUDA cores. */
#define SEB_SUR_SIMT 0
#define SEB_SUR_TCGEN05 1
int seb_sur_set_engine(seb_sur* h, int32_t engine);
/* He-normal weights from a counter-based generator (SplitMix64 + Box-Muller), zero Adam state. */
int seb_sur_init(seb_sur* h, uint64_t seed);
/*
 * Writes training patches [offset, offset + n) of the batch: centres_dev [n][2] (cx, cy) name
 * 48 x 48 crops [cx-24, cx+24) x [cy-24, cy+24) of elev_dev [ny][nx]; labels come from
 * exact_dev, the exact assessment of that elevation in logical order [5][n_yaw][ny][nx]
 * (seb_map_copy_out).  Crops outside the map raise the device error word.
 */
int seb_sur_gather(seb_sur* h, const float* elev_dev, const float* exact_dev, int32_t nx, int32_t ny,
                   const int32_t* centres_dev, int32_t n, int32_t offset);
/* Forward, mean squared error over the finite labels, backward and one Adam step (step >= 1)
 * on the first `batch` patches; loss_dev (may be NULL) receives the loss. */
int seb_sur_train_step(seb_sur* h, int32_t batch, float lr, int32_t step, float* loss_dev);
/* Forward only (evaluation) into the pred buffer. */
int seb_sur_forward(seb_sur* h, int32_t batch);
/*
 * Inference on a p->nx x p->ny map: writes out_dev [5][n_yaw][ny][nx] and flags_dev like a
 * map (roughness is not predicted: NaN, flag SEB_FLAG_SURROGATE) for the cells at least 16
 * from the border; mask_dev [ny][nx] (may be NULL) receives the fallback mask (a NaN or a
 * 4-neighbour step above `step` metres within Chebyshev distance `radius`, or the border);
 * with exact_fallback != 0 the exact kernel then overwrites every masked cell (border cells
 * included); with exact_fallback == 0 the border cells of out_dev and flags_dev are not written.
 */
int seb_sur_infer(seb_sur* h, const float* elev_dev, float step, int32_t radius, int32_t exact_fallback,
                  float* out_dev, uint8_t* flags_dev, uint8_t* mask_dev);
/*
 * Checkpoint / resume of training (the paper has no learned model; this serves the surrogate
 * above).  The image holds everything the training step carries from one call to the next: the
 * FP32 master weights, the Adam first and second moments, the BF16 weights the kernels read and
 * the Adam step of the last seb_sur_train_step, behind a 64-byte header that names the network's
 * size.  Training itself draws no random numbers (the caller seeds seb_terrain_bumpy and picks
 * the patch centres), and its reductions run in a fixed order, so a run resumed from an image
 * with the caller's own generator state restored repeats the original run bit for bit.
 *   seb_sur_state_bytes: size of the image (0 for NULL).
 *   seb_sur_save: writes the image to caller-owned HOST memory host_dst (>= that many bytes);
 *     enqueues the copies on the handle's stream and synchronises it (a blocking call).
 *   seb_sur_load: restores an image into a handle of the same network (same n_yaw); rejects
 *     images of another size or without the header with SEB_ERR_INVALID_ARG; blocking.
 *   seb_sur_step: the Adam step of the last train step (0 after init, the saved step after a
 *     load), -1 for NULL.
 */
size_t seb_sur_state_bytes(const seb_sur* h);
int seb_sur_save(seb_sur* h, void* host_dst, size_t bytes);
int seb_sur_load(seb_sur* h, const void* host_src, size_t bytes);
int64_t seb_sur_step(const seb_sur* h);
/* Terrain of the small-map recipe on the GPU (training data): per world 36 parameters
 * (tan slope, azimuth, noise sigma, unused, then (amplitude, sigma, cx, cy) x 8 bumps); the
 * noise is N(0, sigma) from a counter-based generator seeded by seed.  out_dev [n][ny][nx]. */
int seb_terrain_bumpy(const float* params_dev, int32_t n, int32_t nx, int32_t ny, float res, uint64_t seed,
                      float* out_dev, seb_stream_t stream);

/*
 * Allocation-free pose query: the forward and the backward of seb_query_poses /
 * seb_query_poses_backward in one call, for callers that cannot allocate device memory
 * (a real-time loop held to a fixed memory budget, or an embedding host whose allocator the
 * library may not touch).  The paper has no counterpart: this is a packaging of the query
 * above.  The per-pose state passed from the forward to the backward lives in a file-scope
 * device array of SEB_NOALLOC_MAX_POSES records (4 MiB) instead of a caller buffer; every GPU
 * that loads the library keeps that array until the process exits.
 *   poses_dev [n][3], grad_out_dev [n][SEB_N_CH] (inputs); out_dev [n][SEB_N_CH],
 *   flags_dev [n], grad_pose_dev [n][3] (outputs, caller-owned).
 * n > SEB_NOALLOC_MAX_POSES returns SEB_ERR_INVALID_ARG with a message naming the limit.
 * Parameters are validated exactly as seb_query_poses validates them (same lattice, same
 * limits).  Calls no cudaMalloc, cudaFree or other allocating routine, and no host heap
 * allocation either.  All calls share the array: calls whose kernels overlap on the GPU
 * (unordered streams) race on it; calls on one stream are safe.  Nothing in it needs clearing:
 * the forward writes every record the backward reads.  The first call on a device looks the
 * array's address up (cudaGetSymbolAddress, with that device current); under lazy module
 * loading that lookup is what loads the library's device code and the 4 MiB array onto the
 * device, so it can fail for lack of device memory.  Make one warm-up call per device at
 * start-up (n = 0 is not enough: it returns before the lookup; any n >= 1 does it), before any
 * stream capture and before the fixed memory budget is taken.
 */
#define SEB_NOALLOC_MAX_POSES 65536
int seb_query_poses_grad_noalloc(const seb_params* p, const void* elev_dev, int64_t origin_i,
                                 int64_t origin_j, const float* poses_dev, int64_t n,
                                 const float* grad_out_dev, float* out_dev, uint8_t* flags_dev,
                                 float* grad_pose_dev, seb_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SEB_H_ */
