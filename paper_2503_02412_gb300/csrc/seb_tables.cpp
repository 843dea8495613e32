// Footprint tables on the host (Algorithm 1, FindEllipticalPoints), built once per map.
//
// For yaw pair p (bins p and p + K/2, theta_p = 2 pi p / K) an integer cell offset
// (di, dj) belongs to the footprint when its body-frame coordinates in cell units,
// u = cos(theta) di + sin(theta) dj and v = -sin(theta) di + cos(theta) dj, satisfy
//   rectangle: |u| <= a + 1e-6 and |v| <= b + 1e-6,   a = length / (2 res), b = width / (2 res)
//   ellipse:   (u/a)^2 + (v/b)^2 <= 1 + 1e-6.
// The set is centrally symmetric, so the bin at theta + pi uses the same set.  Each row
// dj of the set is stored as maximal runs of consecutive di, in dj-ascending order; the
// kernels accumulate the moments in exactly this order, whatever tile a cell falls in.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "seb_internal.h"

namespace seb {

int validate_params(const seb_params& p) {
  if (p.nx < 1 || p.ny < 1) return SEB_ERR_INVALID_ARG;
  if (p.n_yaw < 2 || p.n_yaw > 2 * kMaxPairs || (p.n_yaw & 1)) return SEB_ERR_BAD_SHAPE;
  if (!(p.res > 0.f) || !(p.length > 0.f) || !(p.width > 0.f)) return SEB_ERR_INVALID_ARG;
  if (p.shape != SEB_RECT && p.shape != SEB_ELLIPSE) return SEB_ERR_INVALID_ARG;
  if (!(p.kappa_max > 0.f) || !(p.phi_x_max > 0.f) || !(p.phi_y_max > 0.f))
    return SEB_ERR_INVALID_ARG;
  if (p.elev_dtype != SEB_F32 && p.elev_dtype != SEB_BF16 && p.elev_dtype != SEB_F16 &&
      p.elev_dtype != SEB_BF16_TILED)
    return SEB_ERR_INVALID_ARG;
  if (p.precision != SEB_PLAIN_F32 && p.precision != SEB_COMPENSATED) return SEB_ERR_INVALID_ARG;
  if (p.n_min < 0) return SEB_ERR_INVALID_ARG;
  if ((int64_t)p.nx * p.ny > (int64_t)1 << 31) return SEB_ERR_BAD_SHAPE;
  return SEB_OK;
}

size_t out_bytes(const seb_params& p) {
  return (size_t)SEB_N_CH * p.n_yaw * (size_t)p.nx * p.ny * sizeof(float);
}
size_t flags_bytes(const seb_params& p) { return (size_t)p.n_yaw * (size_t)p.nx * p.ny; }

static bool member(const seb_params& p, double c, double s, int di, int dj) {
  const double a = (double)p.length / (2.0 * (double)p.res);
  const double b = (double)p.width / (2.0 * (double)p.res);
  const double u = c * di + s * dj;
  const double v = -s * di + c * dj;
  if (p.shape == SEB_RECT) return fabs(u) <= a + 1e-6 && fabs(v) <= b + 1e-6;
  return (u / a) * (u / a) + (v / b) * (v / b) <= 1.0 + 1e-6;
}

// Offsets of yaw pair q in row-run order (dj ascending, then di ascending), handed to visit(di, dj)
// one at a time: no heap memory, so every caller (the allocation-free query included) enumerates
// the same sets with the same rule.
template <typename Visit>
static void enumerate(const seb_params& p, int q, Visit visit) {
  const double a = (double)p.length / (2.0 * (double)p.res);
  const double b = (double)p.width / (2.0 * (double)p.res);
  const int B = (int)ceil(sqrt(a * a + b * b)) + 1;
  const double th = 2.0 * M_PI * (double)q / (double)p.n_yaw;
  const double c = cos(th), s = sin(th);
  for (int y = -B; y <= B; ++y)
    for (int x = -B; x <= B; ++x)
      if (member(p, c, s, x, y)) visit(x, y);
}

int build_tables(const seb_params& p, Tables* T, int32_t* total_runs) {
  memset(T, 0, sizeof(*T));
  const int half = p.n_yaw / 2;
  T->n_pairs = half;
  int nr = 0, rx = 0, ry = 0;
  for (int q = 0; q < half; ++q) {
    T->run_start[q] = nr;
    int64_t m[6] = {0, 0, 0, 0, 0, 0};
    // maximal runs of consecutive di in one row, closed when the next offset does not extend them
    int run_dj = 0, run_lo = 0, run_hi = 0;
    bool open = false, bad = false;
    auto close = [&]() {
      if (!open || bad) return;
      if (nr >= kMaxRuns) {
        set_error("footprint needs more than %d row runs", kMaxRuns);
        bad = true;
        return;
      }
      if (run_dj < -127 || run_dj > 127 || run_lo < -127 || run_hi > 127) {
        set_error("footprint reach exceeds 127 cells");
        bad = true;
        return;
      }
      T->runs[nr++] = (uint32_t)(run_dj + 128) | ((uint32_t)(run_lo + 128) << 8) | ((uint32_t)(run_hi + 128) << 16);
    };
    enumerate(p, q, [&](int di, int dj) {
      m[0] += 1;
      m[1] += di;
      m[2] += dj;
      m[3] += (int64_t)di * di;
      m[4] += (int64_t)di * dj;
      m[5] += (int64_t)dj * dj;
      rx = abs(di) > rx ? abs(di) : rx;
      ry = abs(dj) > ry ? abs(dj) : ry;
      if (open && dj == run_dj && di == run_hi + 1) {
        run_hi = di;
        return;
      }
      close();
      open = true;
      run_dj = dj;
      run_lo = run_hi = di;
    });
    close();
    if (bad) return SEB_ERR_BAD_SHAPE;
    const int n = (int)m[0];
    for (int t = 0; t < 6; ++t) {
      if (m[t] > (1 << 24) || m[t] < -(1 << 24)) {
        set_error("footprint moments exceed 2^24");
        return SEB_ERR_BAD_SHAPE;
      }
      T->mom[q][t] = (int32_t)m[t];
    }
    T->n_min[q] = p.n_min > 0 ? p.n_min : ((n + 1) / 2 > 3 ? (n + 1) / 2 : 3);
    T->inv_n[q] = n > 0 ? 1.0f / (float)n : 0.f;  // IEEE division: the value 1.f / N gives on the GPU
    const double th = 2.0 * M_PI * (double)q / (double)p.n_yaw;
    T->cos_t[q] = (float)cos(th);
    T->sin_t[q] = (float)sin(th);
  }
  T->run_start[half] = nr;
  // Masked partial moments are summed exactly in FP32: keep every partial sum below 2^24.
  int nmax = 0;
  for (int q = 0; q < half; ++q) nmax = T->mom[q][0] > nmax ? T->mom[q][0] : nmax;
  const int64_t big = (int64_t)nmax * (rx > ry ? rx : ry) * (rx > ry ? rx : ry);
  if (big > (1 << 24)) {
    set_error("footprint too large for exact FP32 moments");
    return SEB_ERR_BAD_SHAPE;
  }
  T->rx = rx;
  T->ry = ry;
  const int64_t nr2 = (int64_t)nmax * (rx > ry ? rx : ry);
  T->narrow = nr2 * nr2 < ((int64_t)1 << 31) ? 1 : 0;
  // The staged tile of every layout (plus the row flags) must fit in 227 KB of shared memory.
  for (int lg = 1; lg <= 5; lg += 2)
    if (stage_h(lg, ry) > kMaxStageRows ||
        ((size_t)stage_w(lg, rx) * stage_h(lg, ry) + kMaxStageRows) * sizeof(float) > 227 * 1024) {
      set_error("footprint reach too large for the staged tile");
      return SEB_ERR_BAD_SHAPE;
    }
  if (total_runs) *total_runs = nr;
  return SEB_OK;
}

int build_lattice(const Tables& T, QTab* Q) {
  int n = 0;
  for (int r = T.run_start[0]; r < T.run_start[1]; ++r) {
    const uint32_t pk = T.runs[r];
    const int y = (int)(pk & 0xff) - 128, lo = (int)((pk >> 8) & 0xff) - 128, hi = (int)((pk >> 16) & 0xff) - 128;
    for (int x = lo; x <= hi; ++x) {
      if (n >= kMaxLattice) {
        set_error("footprint lattice exceeds %d points", kMaxLattice);
        return SEB_ERR_BAD_SHAPE;
      }
      Q->di[n] = (int8_t)x;
      Q->dj[n] = (int8_t)y;
      ++n;
    }
  }
  Q->n = n;
  Q->n_min = T.n_min[0];
  return SEB_OK;
}

}  // namespace seb

extern "C" int seb_footprint_table(const seb_params* p, int32_t k, int32_t* di, int32_t* dj,
                                   int32_t cap) {
  SEB_RANGE();
  if (!p) return SEB_ERR_INVALID_ARG;
  int rc = seb::validate_params(*p);
  if (rc) return rc;
  if (k < 0 || k >= p->n_yaw) return SEB_ERR_INVALID_ARG;
  seb::Tables* T = new seb::Tables;
  rc = seb::build_tables(*p, T, nullptr);
  if (rc) {
    delete T;
    return rc;
  }
  const int q = k % (p->n_yaw / 2);
  int n = 0;
  for (int r = T->run_start[q]; r < T->run_start[q + 1]; ++r) {
    const uint32_t pk = T->runs[r];
    const int y = (int)(pk & 0xff) - 128, lo = (int)((pk >> 8) & 0xff) - 128,
              hi = (int)((pk >> 16) & 0xff) - 128;
    for (int x = lo; x <= hi; ++x, ++n)
      if (n < cap && di && dj) {
        di[n] = x;
        dj[n] = y;
      }
  }
  delete T;
  return n;
}
