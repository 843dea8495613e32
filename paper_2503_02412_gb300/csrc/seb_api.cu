// C ABI of libseb (declared in include/seb.h): map lifetime, full rebuild, rolling shift
// (Sec. V-A: the window follows the robot, Eq. (pm); cells that leave become unknown),
// views, copies and error reporting.  Host-side logic only; kernels live in the other
// translation units.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <new>
#include <thread>

#include "seb_internal.h"

struct seb_map {
  seb_params p;
  seb::Tables T;
  int32_t total_runs;
  uint8_t* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  float* out;
  uint8_t* flags;
  seb::Control* ctl;
  int32_t ring_x, ring_y;
  int64_t oi, oj;
  int64_t last_cells;
  bool valid;
  char err[256];
};

namespace seb {

static thread_local char g_err[256] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

static int cuda_fail(seb_map* m, cudaError_t e, const char* where) {
  set_error("%s: %s", where, cudaGetErrorString(e));
  if (m) snprintf(m->err, sizeof(m->err), "%s", g_err);
  return SEB_ERR_CUDA;
}

static int fail(seb_map* m, int code, const char* msg) {
  set_error("%s", msg);
  if (m) snprintf(m->err, sizeof(m->err), "%s", msg);
  return code;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void launch_defaults(const seb_params& p, const Tables& T, Launch* L) {
  memset(L, 0, sizeof(*L));
  L->nx = p.nx;
  L->ny = p.ny;
  L->plane = (int64_t)p.nx * p.ny;
  L->n_yaw = p.n_yaw;
  L->res = p.res;
  L->kappa_max = p.kappa_max;
  L->phi_x_max = p.phi_x_max;
  L->phi_y_max = p.phi_y_max;
  L->inv_kappa_max = 1.f / p.kappa_max;
  L->inv_phi_x_max = 1.f / p.phi_x_max;
  L->inv_phi_y_max = 1.f / p.phi_y_max;
  L->w0 = p.w[0];
  L->w1 = p.w[1];
  L->w2 = p.w[2];
  L->gap_fp64 = p.gap_fp64;
  L->narrow_moments = T.narrow;
}

static Launch base_launch(const seb_map* m, const void* elev) {
  Launch L;
  launch_defaults(m->p, m->T, &L);
  L.elev = elev;
  if (m->p.elev_dtype == SEB_BF16_TILED && elev) {
    L.tile_base = reinterpret_cast<const float*>(static_cast<const uint8_t*>(elev) +
                                                 tiled_base_offset(m->p.nx, m->p.ny));
    L.base_tx = tiled_tx(m->p.nx);
  }
  L.ring_x = m->ring_x;
  L.ring_y = m->ring_y;
  L.out = m->out;
  L.flags = m->flags;
  L.err = &m->ctl->err;
  L.counters = &m->ctl->n_fp64;
  return L;
}

void launch_request(Launch& L, int x0, int y0, int w, int h) {
  if (w <= 0 || h <= 0 || L.n_req >= 4) return;
  L.req[L.n_req++] = Rect{x0, y0, w, h, x0, y0, 0};
}

void launch_set_origin(Launch& L, int64_t oi, int64_t oj) {
  L.phase_x = (int32_t)(((oi % 4) + 4) % 4);
  L.phase_y = (int32_t)(((oj % 2) + 2) % 2);
  L.base_px = (int32_t)(((oi % kBaseTile) + kBaseTile) % kBaseTile);
  L.base_py = (int32_t)(((oj % kBaseTile) + kBaseTile) % kBaseTile);
}

static int64_t rect_cells(const Launch& L, int n_yaw) {
  int64_t c = 0;
  for (int i = 0; i < L.n_req; ++i) c += (int64_t)L.req[i].w * L.req[i].h;
  return c * n_yaw;
}

static int check_elev(seb_map* m, const void* elev) {
  if (!elev) return fail(m, SEB_ERR_INVALID_ARG, "elevation pointer is NULL");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, elev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(m, e, "cudaPointerGetAttributes(elevation)");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(m, SEB_ERR_INVALID_ARG, "elevation must be device memory");
  return SEB_OK;
}

}  // namespace seb

using namespace seb;

extern "C" {

void seb_params_default(seb_params* p) {
  SEB_RANGE();
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = 100;
  p->ny = 100;
  p->n_yaw = 36;
  p->res = 0.1f;
  p->shape = SEB_RECT;
  p->length = 0.6f;
  p->width = 0.4f;
  p->kappa_max = 0.1f;
  p->phi_x_max = 0.52f;
  p->phi_y_max = 0.52f;
  p->w[0] = p->w[1] = p->w[2] = 1.0f / 3.0f;
  p->n_min = 0;
  p->elev_dtype = SEB_F32;
  p->precision = SEB_PLAIN_F32;
  p->gap_fp64 = 1e-2f;
}

const char* seb_status_string(int s) {
  SEB_RANGE();
  switch (s) {
    case SEB_OK: return "ok";
    case SEB_ERR_INVALID_ARG: return "invalid argument";
    case SEB_ERR_BAD_SHAPE: return "unsupported shape";
    case SEB_ERR_CUDA: return "CUDA error";
    case SEB_ERR_TIMEOUT: return "timeout";
    case SEB_ERR_DEVICE_FAULT: return "device error word set";
    case SEB_ERR_WORKSPACE: return "workspace too small or misaligned";
    default: return "unknown status";
  }
}

const char* seb_last_error(const seb_map* m) { return m ? m->err : g_err; }

size_t seb_workspace_bytes(const seb_params* p) {
  SEB_RANGE();
  if (!p || validate_params(*p) != SEB_OK) return 0;
  return kControlBytes + align256(out_bytes(*p)) + align256(flags_bytes(*p));
}

size_t seb_tiled_base_offset(int32_t nx, int32_t ny) {
  if (nx < 1 || ny < 1) return 0;
  return tiled_base_offset(nx, ny);
}

size_t seb_window_bytes(const seb_params* p) {
  if (!p || validate_params(*p) != SEB_OK) return 0;
  const size_t n = (size_t)p->nx * p->ny;
  switch (p->elev_dtype) {
    case SEB_F32: return n * 4;
    case SEB_BF16:
    case SEB_F16: return n * 2;
    default: return tiled_base_offset(p->nx, p->ny) + (size_t)tiled_tx(p->nx) * tiled_tx(p->ny) * 4;
  }
}

int seb_map_create(const seb_params* p, void* ws, size_t bytes, seb_stream_t stream, seb_map** out) {
  SEB_RANGE();
  if (!p || !out) return fail(nullptr, SEB_ERR_INVALID_ARG, "params or out pointer is NULL");
  *out = nullptr;
  int rc = validate_params(*p);
  if (rc) return fail(nullptr, rc, "invalid parameters");
  if (!ws || ((uintptr_t)ws & 255)) return fail(nullptr, SEB_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
  if (bytes < seb_workspace_bytes(p)) return fail(nullptr, SEB_ERR_WORKSPACE, "workspace too small");
  seb_map* m = new (std::nothrow) seb_map;
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "out of host memory");
  memset(m, 0, sizeof(*m));
  m->p = *p;
  rc = build_tables(*p, &m->T, &m->total_runs);
  if (rc) {
    delete m;
    return rc;
  }
  m->ws = (uint8_t*)ws;
  m->ws_bytes = bytes;
  m->stream = (cudaStream_t)stream;
  m->ctl = (Control*)ws;
  m->out = (float*)(m->ws + kControlBytes);
  m->flags = m->ws + kControlBytes + align256(out_bytes(*p));
  cudaError_t e = cudaMemsetAsync(m->ctl, 0, sizeof(Control), m->stream);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(nullptr, e, "cudaMemsetAsync(control)");
  }
  *out = m;
  return SEB_OK;
}

int seb_map_destroy(seb_map* m) {
  SEB_RANGE();
  if (!m) return SEB_ERR_INVALID_ARG;
  delete m;
  return SEB_OK;
}

int seb_map_set_stream(seb_map* m, seb_stream_t s) {
  SEB_RANGE();
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  m->stream = (cudaStream_t)s;
  return SEB_OK;
}

static int update_impl(seb_map* m, const void* elev, int64_t oi, int64_t oj, int early) {
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  int rc = check_elev(m, elev);
  if (rc) return rc;
  // physical index = grid index mod n (the window's torus), so that a rebuild and any later
  // shift see the same physical alignment of the globally aligned cell blocks
  m->ring_x = (int32_t)(((oi % m->p.nx) + m->p.nx) % m->p.nx);
  m->ring_y = (int32_t)(((oj % m->p.ny) + m->p.ny) % m->p.ny);
  Launch L = base_launch(m, elev);
  L.early = early;
  launch_set_origin(L, oi, oj);
  launch_request(L, 0, 0, m->p.nx, m->p.ny);
  cudaError_t e = launch_assess(m->T, L, m->p.elev_dtype, m->p.precision, m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "assess launch");
  m->last_cells = rect_cells(L, m->p.n_yaw);
  m->oi = oi;
  m->oj = oj;
  m->valid = true;
  return SEB_OK;
}

int seb_map_update(seb_map* m, const void* elev, int64_t oi, int64_t oj) {
  SEB_RANGE();
  return update_impl(m, elev, oi, oj, 0);
}

static int shift_impl(seb_map* m, const void* elev, int64_t oi, int64_t oj, int early) {
  SEB_RANGE();
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  if (!m->valid) return update_impl(m, elev, oi, oj, early);
  int rc = check_elev(m, elev);
  if (rc) return rc;
  const int64_t dx = oi - m->oi, dy = oj - m->oj;
  const int nx = m->p.nx, ny = m->p.ny;
  if (dx >= nx || -dx >= nx || dy >= ny || -dy >= ny) return update_impl(m, elev, oi, oj, early);
  if (dx == 0 && dy == 0) {
    m->last_cells = 0;
    return SEB_OK;
  }
  // Logical cell c of the new window is logical c + dx of the old one; the ring offset
  // keeps every surviving cell at its physical address.
  m->ring_x = (int32_t)(((m->ring_x + dx) % nx + nx) % nx);
  m->ring_y = (int32_t)(((m->ring_y + dy) % ny + ny) % ny);
  // Column bands: cells that now see entering columns, and cells that used to see columns that
  // left the window (the footprint's reach inwards from either edge).  Row bands likewise.
  const int rx = m->T.rx, ry = m->T.ry;
  int left = 0, right = 0, top = 0, bottom = 0;
  if (dx > 0) {
    right = (int)dx + rx;
    left = rx;
  } else if (dx < 0) {
    left = (int)(-dx) + rx;
    right = rx;
  }
  if (dy > 0) {
    bottom = (int)dy + ry;
    top = ry;
  } else if (dy < 0) {
    top = (int)(-dy) + ry;
    bottom = ry;
  }
  // Cells of a 4 x 2 block (world column = 0 mod 4, world row = 0 mod 2) share a reference
  // height, so each band is widened to whole blocks: a block with a cell in a band is
  // recomputed whole, and every other block keeps its inputs and its reference.
  const int px = (int)(((oi % 4) + 4) % 4), py = (int)(((oj % 2) + 2) % 2);
  if (left > 0) left += (4 - (left + px) % 4) % 4;
  if (right > 0) right += (nx - right + px) % 4;
  if (top > 0) top += (2 - (top + py) % 2) % 2;
  if (bottom > 0) bottom += (ny - bottom + py) % 2;
  Launch L = base_launch(m, elev);
  L.early = early;
  launch_set_origin(L, oi, oj);
  if (left + right >= nx || top + bottom >= ny) {
    launch_request(L, 0, 0, nx, ny);
  } else {
    L.all_masked = 1;  // bands along the window edge (the results do not depend on this choice)
    launch_request(L, 0, 0, left, ny);
    launch_request(L, nx - right, 0, right, ny);
    launch_request(L, left, 0, nx - left - right, top);
    launch_request(L, left, ny - bottom, nx - left - right, bottom);
  }
  cudaError_t e = launch_assess(m->T, L, m->p.elev_dtype, m->p.precision, m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "assess launch (shift)");
  m->last_cells = rect_cells(L, m->p.n_yaw);
  m->oi = oi;
  m->oj = oj;
  return SEB_OK;
}

int seb_map_shift(seb_map* m, const void* elev, int64_t oi, int64_t oj) {
  SEB_RANGE();
  return shift_impl(m, elev, oi, oj, 0);
}

int seb_map_shift_batch(seb_map* m, const void* const* elev, const int64_t* origins, int32_t n) {
  SEB_RANGE();
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || (n > 0 && (!elev || !origins)))
    return fail(m, SEB_ERR_INVALID_ARG, "shift batch: NULL window or origin array, or negative count");
  int64_t cells = 0;
  for (int32_t i = 0; i < n; ++i) {
    // The first launch of the batch waits for everything before it; the later ones may start
    // early.  A zero move launches nothing, so "first" is counted in launches, not in moves.
    const int rc = shift_impl(m, elev[i], origins[2 * i], origins[2 * i + 1], cells > 0 ? 1 : 0);
    if (rc) return rc;
    cells += m->last_cells;
  }
  m->last_cells = cells;
  return SEB_OK;
}

int seb_map_grid(const seb_map* m, int32_t channel, seb_grid* g) {
  SEB_RANGE();
  if (!m || !g) return fail(nullptr, SEB_ERR_INVALID_ARG, "map or grid is NULL");
  if (channel < 0 || channel >= SEB_N_CH) return fail(nullptr, SEB_ERR_INVALID_ARG, "channel out of range");
  if (!m->valid) return fail(nullptr, SEB_ERR_INVALID_ARG, "map has no outputs before its first update");
  const int64_t plane = (int64_t)m->p.nx * m->p.ny;
  g->data = m->out + (int64_t)channel * m->p.n_yaw * plane;
  g->nx = m->p.nx;
  g->ny = m->p.ny;
  g->n_yaw = m->p.n_yaw;
  g->ring_x = m->ring_x;
  g->ring_y = m->ring_y;
  g->origin_i = m->oi;
  g->origin_j = m->oj;
  g->res = m->p.res;
  return SEB_OK;
}

int seb_map_view(const seb_map* m, seb_view* v) {
  SEB_RANGE();
  if (!m || !v) return fail(nullptr, SEB_ERR_INVALID_ARG, "map or view is NULL");
  v->out = m->out;
  v->flags = m->flags;
  v->ring_x = m->ring_x;
  v->ring_y = m->ring_y;
  v->origin_i = m->oi;
  v->origin_j = m->oj;
  v->out_offset = (size_t)((uint8_t*)m->out - m->ws);
  v->flags_offset = (size_t)(m->flags - m->ws);
  v->last_cells = m->last_cells;
  return SEB_OK;
}

int seb_map_copy_out(const seb_map* m, float* out_dev, uint8_t* flags_dev) {
  SEB_RANGE();
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  if (!out_dev && !flags_dev) return SEB_OK;
  Launch L = base_launch(m, nullptr);
  cudaError_t e = launch_copy_out(L, out_dev, flags_dev, m->stream);
  if (e != cudaSuccess) return cuda_fail(const_cast<seb_map*>(m), e, "copy_out launch");
  return SEB_OK;
}

int seb_map_check(seb_map* m, int32_t timeout_ms, int64_t* n_fp64, int64_t* n_degenerate) {
  SEB_RANGE();
  if (!m) return fail(nullptr, SEB_ERR_INVALID_ARG, "map is NULL");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaStreamQuery(m->stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_fail(m, q, "cudaStreamQuery");
    if (timeout_ms > 0 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return fail(m, SEB_ERR_TIMEOUT, "stream did not finish within the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  Control c;
  cudaError_t e = cudaMemcpyAsync(&c, m->ctl, sizeof(c), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->ctl, 0, sizeof(Control), m->stream);
  if (e != cudaSuccess) return cuda_fail(m, e, "reading the control block");
  if (n_fp64) *n_fp64 = (int64_t)c.n_fp64;
  if (n_degenerate) *n_degenerate = (int64_t)c.n_degenerate;
  if (c.err) {
    char msg[96];
    snprintf(msg, sizeof(msg), "device error word 0x%x", c.err);
    return fail(m, SEB_ERR_DEVICE_FAULT, msg);
  }
  return SEB_OK;
}

}  // extern "C"
