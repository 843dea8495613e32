/*
 * FP64 CPU oracle for SE(2)-grid traversability assessment (SEB-Naver, Sec. III and
 * Sec. V-B, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path
 * is checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant with the CUDA library:
 * every rule below is restated here from the paper in its own code.
 *
 * What it computes, for every cell (c, r) of a [ny][nx] elevation window and every yaw
 * bin k of n_yaw bins (theta_k = 2*pi*k/n_yaw):
 *   1. the footprint: every integer cell offset (di, dj) whose coordinates in the body
 *      frame, (u, v) = R(-theta)(di, dj) in cell units, lie in the vehicle footprint
 *      (Algorithm 1, FindEllipticalPoints).  Rectangle: |u| <= a + 1e-6 and |v| <= b + 1e-6
 *      with a = length / (2 res), b = width / (2 res).  Ellipse: (u/a)^2 + (v/b)^2 <= 1 + 1e-6.
 *      Bins k >= n_yaw/2 use theta_{k - n_yaw/2}: the footprint is centrally symmetric, so
 *      the set at theta + pi is by definition the set at theta.
 *   2. the known points among them (inside the window and not NaN), as world points
 *      ((o_i + c + di + 1/2) res, (o_j + r + dj + 1/2) res, z);
 *   3. fewer than n_min known points -> UNKNOWN (risk 1, other outputs NaN);
 *   4. mean and population covariance Cov = sum (p - mean)(p - mean)^T / N (Algorithm 1);
 *   5. eigen-decomposition by cyclic Jacobi (Golub & Van Loan, Matrix Computations,
 *      Sec. 8.5), to a relative off-diagonal norm of 1e-15;
 *   6. z_b = the unit eigenvector of the smallest eigenvalue, sign chosen so that
 *      b3^T z_b > 0 (the S^2_+ half-sphere of Sec. III); curvature kappa = lambda_min / trace;
 *   7. y_b = (z_b x x_yaw) / |z_b x x_yaw|, x_b = y_b x z_b (Eqs. 2-3, Sec. III);
 *      pitch = asin(b3^T x_b), roll = asin(b3^T y_b) (signed; Algorithm 1 takes |.|);
 *   8. z = height of the fitted plane at the pose centre (x_c, y_c):
 *      z = mean_z - (n_x (x_c - mean_x) + n_y (y_c - mean_y)) / n_z;
 *   9. risk (Algorithm 1): 1 if kappa > kappa_max, else 1 if |pitch| > phi_x_max or
 *      |roll| > phi_y_max, else w . [kappa/kappa_max, |pitch|/phi_x_max, |roll|/phi_y_max].
 *      A normal that is nearly horizontal (n_z <= 1e-6), a yaw parallel to the normal
 *      (|z_b x x_yaw| < 1e-6) or a relative eigen-gap (lambda_mid - lambda_min)/trace below
 *      1e-12 makes the cell DEGENERATE: risk 1, z/pitch/roll NaN.
 *
 * The continuous-pose query (a differentiable form of the same assessment) samples the
 * elevation by bilinear interpolation at the footprint lattice of yaw 0, rotated by the
 * pose yaw and translated to the pose position; its FP64 reverse-mode gradient is written
 * out by hand in orc_pose_vjp and checked against central differences by the tests.
 *
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared -pthread -o liborc.so seb_oracle.c -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_UNKNOWN 1
#define ORC_OBSTACLE 2
#define ORC_DEGENERATE 4

#define ORC_PI 3.14159265358979323846

typedef struct {
  int nx, ny, n_yaw;
  double res;
  int shape; /* 0 = rectangle, 1 = ellipse */
  double length, width;
  double kappa_max, phi_x_max, phi_y_max;
  double w[3];
  int n_min; /* 0 -> max(3, ceil(N_k / 2)) with N_k the footprint size of bin k */
} orc_params;

/* ------------------------------------------------------------------------------------ */
/* Footprint membership (Algorithm 1, FindEllipticalPoints)                               */
/* ------------------------------------------------------------------------------------ */

static int inside_footprint(const orc_params* P, double theta, int di, int dj) {
  double a = P->length / (2.0 * P->res);
  double b = P->width / (2.0 * P->res);
  double c = cos(theta), s = sin(theta);
  double u = c * di + s * dj;
  double v = -s * di + c * dj;
  if (P->shape == 0) return fabs(u) <= a + 1e-6 && fabs(v) <= b + 1e-6;
  return (u / a) * (u / a) + (v / b) * (v / b) <= 1.0 + 1e-6;
}

static double table_theta(const orc_params* P, int k) {
  int half = P->n_yaw / 2;
  return 2.0 * ORC_PI * (double)(k % half) / (double)P->n_yaw;
}

/* Enumerate the footprint of yaw bin k, rows (dj) outer, columns (di) inner, ascending.
 * Returns the count; writes at most cap offsets. */
int orc_footprint(const orc_params* P, int k, int* di_out, int* dj_out, int cap) {
  double a = P->length / (2.0 * P->res);
  double b = P->width / (2.0 * P->res);
  int B = (int)ceil(sqrt(a * a + b * b)) + 1;
  double th = table_theta(P, k);
  int n = 0;
  for (int dj = -B; dj <= B; ++dj)
    for (int di = -B; di <= B; ++di)
      if (inside_footprint(P, th, di, dj)) {
        if (n < cap) {
          di_out[n] = di;
          dj_out[n] = dj;
        }
        ++n;
      }
  return n;
}

static int min_points(const orc_params* P, int n_foot) {
  if (P->n_min > 0) return P->n_min;
  int h = (n_foot + 1) / 2;
  return h > 3 ? h : 3;
}

/* ------------------------------------------------------------------------------------ */
/* Cyclic Jacobi for a symmetric 3x3 matrix (Golub & Van Loan, Sec. 8.5)                  */
/* ------------------------------------------------------------------------------------ */

/* A is given as the 6 unique entries (xx, xy, xz, yy, yz, zz).  On return evals holds the
 * eigenvalues in ascending order and evecs the matching unit eigenvectors as columns
 * (evecs[3*i + j] = component i of eigenvector j).  Returns the sweep count. */
int orc_jacobi3(const double A6[6], double evals[3], double evecs[9]) {
  double A[3][3] = {{A6[0], A6[1], A6[2]}, {A6[1], A6[3], A6[4]}, {A6[2], A6[4], A6[5]}};
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double fro = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
  fro = sqrt(fro);
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    double off = 2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]);
    if (sqrt(off) <= 1e-15 * fro || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        /* symmetric 2x2 Schur decomposition: choose (c, s) that zeroes A[p][q] */
        double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = tau >= 0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        J[p][p] = c;
        J[p][q] = s;
        J[q][p] = -s;
        J[q][q] = c;
        double T[3][3], N[3][3];
        /* A <- J^T A J */
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int l = 0; l < 3; ++l) acc += A[i][l] * J[l][j];
            T[i][j] = acc;
          }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int l = 0; l < 3; ++l) acc += J[l][i] * T[l][j];
            N[i][j] = acc;
          }
        N[p][q] = N[q][p] = 0.0;
        memcpy(A, N, sizeof(A));
        /* V <- V J */
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int l = 0; l < 3; ++l) acc += V[i][l] * J[l][j];
            T[i][j] = acc;
          }
        memcpy(V, T, sizeof(V));
      }
  }
  int idx[3] = {0, 1, 2};
  double d[3] = {A[0][0], A[1][1], A[2][2]};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (d[idx[j]] < d[idx[i]]) {
        int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  for (int j = 0; j < 3; ++j) {
    evals[j] = d[idx[j]];
    for (int i = 0; i < 3; ++i) evecs[3 * i + j] = V[i][idx[j]];
  }
  return sweep;
}

/* ------------------------------------------------------------------------------------ */
/* Shared tail: covariance of a point set -> outputs (Algorithm 1 from the mean on)       */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int n;
  double mean[3];
  double cov[6]; /* xx xy xz yy yz zz */
  double evals[3];
  double evecs[9];
  double nrm[3]; /* z_b */
  double xb[3], yb[3];
  double u_norm;
  double gap; /* (lambda_mid - lambda_min) / trace */
} orc_detail;

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

static double clamp1(double x) { return x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x); }

/* pts: n points (x, y, z).  (xc, yc) the pose centre, theta the yaw.  out[5] =
 * z, pitch, roll, roughness (kappa), risk.  Returns flags. */
static int assess_points(const orc_params* P, const double* pts, int n, int n_min, double xc,
                         double yc, double theta, double out[5], orc_detail* D) {
  for (int i = 0; i < 5; ++i) out[i] = NAN;
  if (D) memset(D, 0, sizeof(*D));
  if (D) D->n = n;
  if (n < n_min) {
    out[4] = 1.0;
    return ORC_UNKNOWN | ORC_OBSTACLE;
  }
  double m[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 3; ++j) m[j] += pts[3 * i + j];
  for (int j = 0; j < 3; ++j) m[j] /= n;
  double C[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    double e0 = pts[3 * i] - m[0], e1 = pts[3 * i + 1] - m[1], e2 = pts[3 * i + 2] - m[2];
    C[0] += e0 * e0;
    C[1] += e0 * e1;
    C[2] += e0 * e2;
    C[3] += e1 * e1;
    C[4] += e1 * e2;
    C[5] += e2 * e2;
  }
  for (int j = 0; j < 6; ++j) C[j] /= n;
  double ev[3], V[9];
  orc_jacobi3(C, ev, V);
  double nv[3] = {V[0], V[3], V[6]};
  if (nv[2] < 0) {
    nv[0] = -nv[0];
    nv[1] = -nv[1];
    nv[2] = -nv[2];
  }
  double tr = C[0] + C[3] + C[5];
  double kappa = ev[0] / tr;
  double gap = (ev[1] - ev[0]) / tr;
  double xyaw[3] = {cos(theta), sin(theta), 0.0};
  double u[3];
  cross3(nv, xyaw, u);
  double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (D) {
    memcpy(D->mean, m, sizeof(m));
    memcpy(D->cov, C, sizeof(C));
    memcpy(D->evals, ev, sizeof(ev));
    memcpy(D->evecs, V, sizeof(V));
    memcpy(D->nrm, nv, sizeof(nv));
    D->u_norm = un;
    D->gap = gap;
  }
  out[3] = kappa;
  if (gap < 1e-12 || nv[2] <= 1e-6 || un < 1e-6) {
    out[4] = 1.0;
    return ORC_DEGENERATE | ORC_OBSTACLE;
  }
  double yb[3] = {u[0] / un, u[1] / un, u[2] / un};
  double xb[3];
  cross3(yb, nv, xb);
  if (D) {
    memcpy(D->xb, xb, sizeof(xb));
    memcpy(D->yb, yb, sizeof(yb));
  }
  double pitch = asin(clamp1(xb[2]));
  double roll = asin(clamp1(yb[2]));
  out[0] = m[2] - (nv[0] * (xc - m[0]) + nv[1] * (yc - m[1])) / nv[2];
  out[1] = pitch;
  out[2] = roll;
  int flags = 0;
  if (kappa > P->kappa_max) {
    out[4] = 1.0;
    flags |= ORC_OBSTACLE;
  } else if (fabs(pitch) > P->phi_x_max || fabs(roll) > P->phi_y_max) {
    out[4] = 1.0;
    flags |= ORC_OBSTACLE;
  } else {
    out[4] = P->w[0] * kappa / P->kappa_max + P->w[1] * fabs(pitch) / P->phi_x_max +
             P->w[2] * fabs(roll) / P->phi_y_max;
  }
  return flags;
}

/* ------------------------------------------------------------------------------------ */
/* Grid assessment                                                                        */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int n;
  int* di;
  int* dj;
} orc_table;

static int build_tables(const orc_params* P, orc_table* T) {
  for (int k = 0; k < P->n_yaw; ++k) {
    int n = orc_footprint(P, k, NULL, NULL, 0);
    T[k].n = n;
    T[k].di = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    T[k].dj = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    if (!T[k].di || !T[k].dj) return -1;
    orc_footprint(P, k, T[k].di, T[k].dj, n);
  }
  return 0;
}

static void free_tables(const orc_params* P, orc_table* T) {
  for (int k = 0; k < P->n_yaw; ++k) {
    free(T[k].di);
    free(T[k].dj);
  }
}

static int assess_cell(const orc_params* P, const orc_table* T, const double* elev, int64_t oi,
                       int64_t oj, int c, int r, int k, double* pts, double out[5], orc_detail* D) {
  const orc_table* t = &T[k];
  int n = 0;
  for (int q = 0; q < t->n; ++q) {
    int cc = c + t->di[q], rr = r + t->dj[q];
    if (cc < 0 || cc >= P->nx || rr < 0 || rr >= P->ny) continue;
    double z = elev[(int64_t)rr * P->nx + cc];
    if (isnan(z)) continue;
    pts[3 * n] = ((double)oi + cc + 0.5) * P->res;
    pts[3 * n + 1] = ((double)oj + rr + 0.5) * P->res;
    pts[3 * n + 2] = z;
    ++n;
  }
  double xc = ((double)oi + c + 0.5) * P->res;
  double yc = ((double)oj + r + 0.5) * P->res;
  double theta = 2.0 * ORC_PI * (double)k / (double)P->n_yaw;
  return assess_points(P, pts, n, min_points(P, t->n), xc, yc, theta, out, D);
}

typedef struct {
  const orc_params* P;
  const orc_table* T;
  const double* elev;
  int64_t oi, oj;
  /* grid mode */
  double* out;
  uint8_t* flags;
  double* gapg;
  int row0, row1;
  /* list mode */
  const int32_t* cells;
  int64_t i0, i1;
  double* gap;
  int max_n;
} orc_job;

static void* grid_worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  const orc_params* P = J->P;
  double* pts = (double*)malloc(sizeof(double) * 3 * (J->max_n > 0 ? J->max_n : 1));
  int64_t plane = (int64_t)P->nx * P->ny;
  int64_t chs = plane * P->n_yaw;
  for (int r = J->row0; r < J->row1; ++r)
    for (int k = 0; k < P->n_yaw; ++k)
      for (int c = 0; c < P->nx; ++c) {
        double o[5];
        orc_detail D;
        int f = assess_cell(P, J->T, J->elev, J->oi, J->oj, c, r, k, pts, o, &D);
        int64_t idx = (int64_t)k * plane + (int64_t)r * P->nx + c;
        for (int ch = 0; ch < 5; ++ch) J->out[ch * chs + idx] = o[ch];
        J->flags[idx] = (uint8_t)f;
        if (J->gapg) J->gapg[idx] = D.n >= 3 ? D.gap : NAN;
      }
  free(pts);
  return NULL;
}

static int max_table(const orc_params* P, const orc_table* T) {
  int m = 0;
  for (int k = 0; k < P->n_yaw; ++k) m = T[k].n > m ? T[k].n : m;
  return m;
}

/* Full window: out is [5][n_yaw][ny][nx] (z, pitch, roll, roughness, risk), flags
 * [n_yaw][ny][nx], gap [n_yaw][ny][nx] (may be NULL) the relative eigen-gap
 * (lambda_mid - lambda_min) / trace.  Returns 0, or -1 on bad parameters. */
int orc_grid(const orc_params* P, const double* elev, int64_t oi, int64_t oj, double* out,
             uint8_t* flags, double* gap, int n_threads) {
  if (P->n_yaw < 2 || (P->n_yaw & 1) || P->nx <= 0 || P->ny <= 0) return -1;
  orc_table* T = (orc_table*)calloc(P->n_yaw, sizeof(orc_table));
  if (build_tables(P, T)) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > P->ny) n_threads = P->ny;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  orc_job* jobs = (orc_job*)calloc(n_threads, sizeof(orc_job));
  for (int t = 0; t < n_threads; ++t) {
    orc_job* J = &jobs[t];
    J->P = P;
    J->T = T;
    J->elev = elev;
    J->oi = oi;
    J->oj = oj;
    J->out = out;
    J->flags = flags;
    J->gapg = gap;
    J->row0 = (int)((int64_t)P->ny * t / n_threads);
    J->row1 = (int)((int64_t)P->ny * (t + 1) / n_threads);
    J->max_n = max_table(P, T);
    pthread_create(&th[t], NULL, grid_worker, J);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  free_tables(P, T);
  free(T);
  return 0;
}

static void* list_worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  double* pts = (double*)malloc(sizeof(double) * 3 * (J->max_n > 0 ? J->max_n : 1));
  for (int64_t i = J->i0; i < J->i1; ++i) {
    int c = J->cells[3 * i], r = J->cells[3 * i + 1], k = J->cells[3 * i + 2];
    orc_detail D;
    double o[5];
    int f = assess_cell(J->P, J->T, J->elev, J->oi, J->oj, c, r, k, pts, o, &D);
    for (int ch = 0; ch < 5; ++ch) J->out[5 * i + ch] = o[ch];
    J->flags[i] = (uint8_t)f;
    if (J->gap) J->gap[i] = D.n >= 3 ? D.gap : NAN;
  }
  free(pts);
  return NULL;
}

/* Listed cells only: cells is [n][3] (c, r, k); out [n][5]; flags [n]; gap [n] (may be
 * NULL) receives the relative eigen-gap (lambda_mid - lambda_min) / trace. */
int orc_cells(const orc_params* P, const double* elev, int64_t oi, int64_t oj,
              const int32_t* cells, int64_t n, double* out, uint8_t* flags, double* gap,
              int n_threads) {
  if (P->n_yaw < 2 || (P->n_yaw & 1)) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int c = cells[3 * i], r = cells[3 * i + 1], k = cells[3 * i + 2];
    if (c < 0 || c >= P->nx || r < 0 || r >= P->ny || k < 0 || k >= P->n_yaw) return -1;
  }
  orc_table* T = (orc_table*)calloc(P->n_yaw, sizeof(orc_table));
  if (build_tables(P, T)) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n) n_threads = n > 0 ? (int)n : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  orc_job* jobs = (orc_job*)calloc(n_threads, sizeof(orc_job));
  for (int t = 0; t < n_threads; ++t) {
    orc_job* J = &jobs[t];
    J->P = P;
    J->T = T;
    J->elev = elev;
    J->oi = oi;
    J->oj = oj;
    J->out = out;
    J->flags = flags;
    J->cells = cells;
    J->gap = gap;
    J->i0 = n * t / n_threads;
    J->i1 = n * (t + 1) / n_threads;
    J->max_n = max_table(P, T);
    pthread_create(&th[t], NULL, list_worker, J);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  free_tables(P, T);
  free(T);
  return 0;
}

/* One cell with its intermediate quantities, for hand-computed checks.  detail receives
 * n, mean[3], cov[6], evals[3], evecs[9], z_b[3], x_b[3], y_b[3], |z_b x x_yaw|, gap
 * (33 doubles). */
int orc_cell_detail(const orc_params* P, const double* elev, int64_t oi, int64_t oj, int c,
                    int r, int k, double out[5], double* detail) {
  if (P->n_yaw < 2 || (P->n_yaw & 1)) return -1;
  orc_table* T = (orc_table*)calloc(P->n_yaw, sizeof(orc_table));
  if (build_tables(P, T)) return -1;
  double* pts = (double*)malloc(sizeof(double) * 3 * (max_table(P, T) + 1));
  orc_detail D;
  int f = assess_cell(P, T, elev, oi, oj, c, r, k, pts, out, &D);
  detail[0] = D.n;
  memcpy(detail + 1, D.mean, 3 * sizeof(double));
  memcpy(detail + 4, D.cov, 6 * sizeof(double));
  memcpy(detail + 10, D.evals, 3 * sizeof(double));
  memcpy(detail + 13, D.evecs, 9 * sizeof(double));
  memcpy(detail + 22, D.nrm, 3 * sizeof(double));
  memcpy(detail + 25, D.xb, 3 * sizeof(double));
  memcpy(detail + 28, D.yb, 3 * sizeof(double));
  detail[31] = D.u_norm;
  detail[32] = D.gap;
  free(pts);
  free_tables(P, T);
  free(T);
  return f;
}

/* ------------------------------------------------------------------------------------ */
/* Continuous-pose query: bilinear elevation on the rotated yaw-0 footprint lattice       */
/* ------------------------------------------------------------------------------------ */

/* Bilinear elevation at world (X, Y).  Cell (c, r) has its centre at grid coordinate
 * (c, r) = (X / res - o_i - 1/2, Y / res - o_j - 1/2).  Returns 0 and NaN if a corner is
 * outside the window or unknown.  dzdx, dzdy receive the partial derivatives (1/m). */
static int bilinear(const orc_params* P, const double* elev, int64_t oi, int64_t oj, double X,
                    double Y, double* z, double* dzdx, double* dzdy, double* gx_out) {
  double gx = X / P->res - (double)oi - 0.5;
  double gy = Y / P->res - (double)oj - 0.5;
  double fx0 = floor(gx), fy0 = floor(gy);
  *z = NAN;
  if (fx0 < 0 || fy0 < 0 || fx0 + 1 > P->nx - 1 || fy0 + 1 > P->ny - 1) return 0;
  int64_t c0 = (int64_t)fx0, r0 = (int64_t)fy0;
  double fx = gx - fx0, fy = gy - fy0;
  double z00 = elev[r0 * P->nx + c0], z10 = elev[r0 * P->nx + c0 + 1];
  double z01 = elev[(r0 + 1) * P->nx + c0], z11 = elev[(r0 + 1) * P->nx + c0 + 1];
  if (isnan(z00) || isnan(z10) || isnan(z01) || isnan(z11)) return 0;
  *z = (1 - fx) * (1 - fy) * z00 + fx * (1 - fy) * z10 + (1 - fx) * fy * z01 + fx * fy * z11;
  if (dzdx) *dzdx = ((1 - fy) * (z10 - z00) + fy * (z11 - z01)) / P->res;
  if (dzdy) *dzdy = ((1 - fx) * (z01 - z00) + fx * (z11 - z10)) / P->res;
  if (gx_out) {
    gx_out[0] = fx;
    gx_out[1] = fy;
  }
  return 1;
}

typedef struct {
  int n;        /* footprint lattice size */
  int* di;      /* lattice offsets (cells) */
  int* dj;
} orc_lattice;

static int lattice(const orc_params* P, orc_lattice* L) {
  orc_params Q = *P;
  int n = orc_footprint(&Q, 0, NULL, NULL, 0);
  L->n = n;
  L->di = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  L->dj = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  orc_footprint(&Q, 0, L->di, L->dj, n);
  return n;
}

/* Forward at one pose.  pts receives the valid points, dz the bilinear gradients,
 * lat the (i, j) lattice indices of the valid points. */
static int pose_forward(const orc_params* P, const orc_lattice* L, const double* elev, int64_t oi,
                        int64_t oj, const double pose[3], double* pts, double* dz, int* lat,
                        double out[5], orc_detail* D, int* n_valid) {
  double x = pose[0], y = pose[1], th = pose[2];
  double c = cos(th), s = sin(th);
  int n = 0;
  for (int q = 0; q < L->n; ++q) {
    double ii = L->di[q] * P->res, jj = L->dj[q] * P->res;
    double X = x + c * ii - s * jj;
    double Y = y + s * ii + c * jj;
    double z, gx, gy;
    if (!bilinear(P, elev, oi, oj, X, Y, &z, &gx, &gy, NULL)) continue;
    pts[3 * n] = X;
    pts[3 * n + 1] = Y;
    pts[3 * n + 2] = z;
    if (dz) {
      dz[2 * n] = gx;
      dz[2 * n + 1] = gy;
    }
    if (lat) {
      lat[2 * n] = L->di[q];
      lat[2 * n + 1] = L->dj[q];
    }
    ++n;
  }
  *n_valid = n;
  return assess_points(P, pts, n, min_points(P, L->n), x, y, th, out, D);
}

typedef struct {
  const orc_params* P;
  const orc_lattice* L;
  const double* elev;
  int64_t oi, oj;
  const double* poses;
  const double* gout;
  double* out;
  uint8_t* flags;
  double* gpose;
  int64_t i0, i1;
} orc_pjob;

static void pose_vjp_one(const orc_params* P, const orc_lattice* L, const double* elev, int64_t oi,
                         int64_t oj, const double pose[3], const double g[4], double gp[3],
                         double* pts, double* dz, int* lat);

static void* pose_worker(void* arg) {
  orc_pjob* J = (orc_pjob*)arg;
  int m = J->L->n > 0 ? J->L->n : 1;
  double* pts = (double*)malloc(sizeof(double) * 3 * m);
  double* dz = (double*)malloc(sizeof(double) * 2 * m);
  int* lat = (int*)malloc(sizeof(int) * 2 * m);
  for (int64_t i = J->i0; i < J->i1; ++i) {
    if (J->gpose) {
      pose_vjp_one(J->P, J->L, J->elev, J->oi, J->oj, J->poses + 3 * i, J->gout + 5 * i,
                   J->gpose + 3 * i, pts, dz, lat);
    } else {
      double o[5];
      int nv;
      int f = pose_forward(J->P, J->L, J->elev, J->oi, J->oj, J->poses + 3 * i, pts, NULL, NULL, o,
                           NULL, &nv);
      for (int ch = 0; ch < 5; ++ch) J->out[5 * i + ch] = o[ch];
      J->flags[i] = (uint8_t)f;
    }
  }
  free(pts);
  free(dz);
  free(lat);
  return NULL;
}

static int run_poses(const orc_params* P, const double* elev, int64_t oi, int64_t oj,
                     const double* poses, int64_t n, const double* gout, double* out,
                     uint8_t* flags, double* gpose, int n_threads) {
  orc_lattice L;
  lattice(P, &L);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n) n_threads = n > 0 ? (int)n : 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  orc_pjob* jobs = (orc_pjob*)calloc(n_threads, sizeof(orc_pjob));
  for (int t = 0; t < n_threads; ++t) {
    orc_pjob* J = &jobs[t];
    J->P = P;
    J->L = &L;
    J->elev = elev;
    J->oi = oi;
    J->oj = oj;
    J->poses = poses;
    J->gout = gout;
    J->out = out;
    J->flags = flags;
    J->gpose = gpose;
    J->i0 = n * t / n_threads;
    J->i1 = n * (t + 1) / n_threads;
    pthread_create(&th[t], NULL, pose_worker, J);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  free(L.di);
  free(L.dj);
  return 0;
}

/* Forward for n poses [n][3] (x, y, yaw in world metres / radians): out [n][5], flags [n]. */
int orc_poses(const orc_params* P, const double* elev, int64_t oi, int64_t oj,
              const double* poses, int64_t n, double* out, uint8_t* flags, int n_threads) {
  if (P->n_yaw < 2 || (P->n_yaw & 1)) return -1;
  return run_poses(P, elev, oi, oj, poses, n, NULL, out, flags, NULL, n_threads);
}

/*
 * Reverse-mode gradient of (z, pitch, roll, roughness, risk) with respect to the pose
 * (x, y, yaw), contracted with gout [n][5].  The valid point set is held fixed (points whose bilinear
 * corners are all known); derivatives are one-sided at |.| kinks (sign(0) = 0) and zero
 * on the clamped risk = 1 branches.  Written directly from the forward definitions:
 *   C = (1/N) sum (P_i - m)(P_i - m)^T, z_b = +-v_min, d lambda_min = n^T dC n,
 *   d n = sum_{j != min} v_j v_j^T dC n / (lambda_min - lambda_j).
 */
static void pose_vjp_one(const orc_params* P, const orc_lattice* L, const double* elev, int64_t oi,
                         int64_t oj, const double pose[3], const double g[4], double gp[3],
                         double* pts, double* dz, int* lat) {
  gp[0] = gp[1] = gp[2] = 0.0;
  double out[5];
  orc_detail D;
  int n;
  int flags = pose_forward(P, L, elev, oi, oj, pose, pts, dz, lat, out, &D, &n);
  if (flags & (ORC_UNKNOWN | ORC_DEGENERATE)) return;
  const double x = pose[0], y = pose[1], th = pose[2];
  const double cth = cos(th), sth = sin(th);
  const double* nv = D.nrm;
  const double* xb = D.xb;
  const double* yb = D.yb;
  const double* m = D.mean;
  double tr = D.cov[0] + D.cov[3] + D.cov[5];
  double lam0 = D.evals[0];
  double pitch = out[1], roll = out[2];

  double kb = g[3], pb = g[1], rb = g[2];
  if (!(flags & ORC_OBSTACLE)) {
    double sp = pitch > 0 ? 1.0 : (pitch < 0 ? -1.0 : 0.0);
    double sr = roll > 0 ? 1.0 : (roll < 0 ? -1.0 : 0.0);
    kb += g[4] * P->w[0] / P->kappa_max;
    pb += g[4] * P->w[1] * sp / P->phi_x_max;
    rb += g[4] * P->w[2] * sr / P->phi_y_max;
  }
  double xbb[3] = {0, 0, pb / sqrt(1.0 - xb[2] * xb[2])};
  double ybb[3] = {0, 0, rb / sqrt(1.0 - yb[2] * yb[2])};
  double nb[3] = {0, 0, 0};
  double t3[3];
  /* x_b = y_b x n */
  cross3(nv, xbb, t3);
  for (int i = 0; i < 3; ++i) ybb[i] += t3[i];
  cross3(xbb, yb, t3);
  for (int i = 0; i < 3; ++i) nb[i] += t3[i];
  /* y_b = u / |u|, u = n x x_yaw */
  double ydot = yb[0] * ybb[0] + yb[1] * ybb[1] + yb[2] * ybb[2];
  double ub[3];
  for (int i = 0; i < 3; ++i) ub[i] = (ybb[i] - yb[i] * ydot) / D.u_norm;
  double xyaw[3] = {cth, sth, 0.0};
  cross3(xyaw, ub, t3);
  for (int i = 0; i < 3; ++i) nb[i] += t3[i];
  double xyb[3];
  cross3(ub, nv, xyb);
  double thb = -sth * xyb[0] + cth * xyb[1];
  /* z = m_z - (n_x (x - m_x) + n_y (y - m_y)) / n_z */
  double dx = x - m[0], dy = y - m[1];
  double h = nv[0] * dx + nv[1] * dy;
  double mb[3] = {0, 0, g[0]};
  nb[0] += -g[0] * dx / nv[2];
  nb[1] += -g[0] * dy / nv[2];
  nb[2] += g[0] * h / (nv[2] * nv[2]);
  double xpb = -g[0] * nv[0] / nv[2];
  double ypb = -g[0] * nv[1] / nv[2];
  mb[0] += g[0] * nv[0] / nv[2];
  mb[1] += g[0] * nv[1] / nv[2];
  /* kappa = lambda_min / trace */
  double lamb = kb / tr;
  double trb = -kb * lam0 / (tr * tr);
  /* Cov adjoint (general 3x3, row-major) */
  double Cb[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Cb[3 * i + j] = lamb * nv[i] * nv[j] + (i == j ? trb : 0.0);
  for (int jv = 1; jv < 3; ++jv) {
    double v[3] = {D.evecs[jv], D.evecs[3 + jv], D.evecs[6 + jv]};
    double coef = (v[0] * nb[0] + v[1] * nb[1] + v[2] * nb[2]) / (lam0 - D.evals[jv]);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Cb[3 * i + j] += coef * v[i] * nv[j];
  }
  double S[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[3 * i + j] = Cb[3 * i + j] + Cb[3 * j + i];
  /* points -> pose */
  double gx = xpb, gy = ypb, gth = thb;
  for (int q = 0; q < n; ++q) {
    double e[3] = {pts[3 * q] - m[0], pts[3 * q + 1] - m[1], pts[3 * q + 2] - m[2]};
    double pb3[3];
    for (int i = 0; i < 3; ++i)
      pb3[i] = (S[3 * i] * e[0] + S[3 * i + 1] * e[1] + S[3 * i + 2] * e[2] + mb[i]) / n;
    double Xb = pb3[0] + pb3[2] * dz[2 * q];
    double Yb = pb3[1] + pb3[2] * dz[2 * q + 1];
    double ii = lat[2 * q] * P->res, jj = lat[2 * q + 1] * P->res;
    gx += Xb;
    gy += Yb;
    gth += Xb * (-sth * ii - cth * jj) + Yb * (cth * ii - sth * jj);
  }
  gp[0] = gx;
  gp[1] = gy;
  gp[2] = gth;
}

/* Gradient for n poses: gout [n][5] (z, pitch, roll, roughness, risk) -> gpose [n][3]. */
int orc_poses_vjp(const orc_params* P, const double* elev, int64_t oi, int64_t oj,
                  const double* poses, int64_t n, const double* gout, double* gpose,
                  int n_threads) {
  if (P->n_yaw < 2 || (P->n_yaw & 1)) return -1;
  return run_poses(P, elev, oi, oj, poses, n, gout, NULL, NULL, gpose, n_threads);
}
