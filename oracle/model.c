/*
 * model.c -- dynamics, validity check and region binning (oracle side).
 *
 * TEST INFRASTRUCTURE ONLY (see kpo.h).  Everything is double precision and
 * written for clarity, not speed.
 *
 * Dynamics (Sec. II, Eq. 1-2; the paper names the three systems in Sec. VI
 * without giving their equations, so the equations below are the textbook
 * forms the paper cites):
 *   double integrator (6D):  p' = v, v' = u                   (explicit Euler)
 *   Dubins airplane (6D, Chitsaz & LaValle 2007):
 *        x' = v cos(psi) cos(theta), y' = v sin(psi) cos(theta),
 *        z' = v sin(theta), psi' = u1, theta' = u2, v' = u3  (classic RK4)
 *   quadrotor (12D, Newton-Euler, plus configuration):
 *        p' = v,  eta' = W(phi, theta) omega,
 *        m v' = R(phi, theta, psi) [0 0 sum T]^T - m g e3,
 *        I omega' = tau - omega x (I omega),
 *        tau = [l (T2 - T4), l (T3 - T1), c (T1 - T2 + T3 - T4)]   (RK4)
 *
 * Validity (Sec. II valid set; Algorithm 2, validity of the segment): after
 * every integrator step the state must lie in the state box, and the
 * axis-aligned box spanned by the positions before and after the step must
 * not meet any obstacle.  Obstacles are closed sets (Sec. II), so touching
 * counts as a collision.
 *
 * Binning (Sec. III, decomposition R and sub-regions R_i^k): a uniform grid
 * over the workspace position, optionally with speed bins and with cells
 * over further state dimensions in the region index (a grid over the whole
 * state space, as in the paper's experiments, Sec. VI); each region holds a
 * uniform sub-grid over position.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kpo_internal.h"

/* ------------------------------------------------------------------ */
/* vector fields                                                        */
/* ------------------------------------------------------------------ */

static void f_dubins(const double *x, const double *u, double *dx) {
  double psi = x[3], theta = x[4], v = x[5];
  dx[0] = v * cos(psi) * cos(theta);
  dx[1] = v * sin(psi) * cos(theta);
  dx[2] = v * sin(theta);
  dx[3] = u[0];
  dx[4] = u[1];
  dx[5] = u[2];
}

static void f_quad(const double *phys, const double *x, const double *u,
                   double *dx) {
  double m = phys[0], g = phys[1], l = phys[2], c = phys[3];
  double Ix = phys[4], Iy = phys[5], Iz = phys[6];
  double phi = x[3], theta = x[4], psi = x[5];
  double vx = x[6], vy = x[7], vz = x[8];
  double p = x[9], q = x[10], r = x[11];
  double T1 = u[0], T2 = u[1], T3 = u[2], T4 = u[3];

  /* position */
  dx[0] = vx;
  dx[1] = vy;
  dx[2] = vz;
  /* Euler-angle rates from body rates (ZYX angles) */
  double sphi = sin(phi), cphi = cos(phi);
  double ttheta = tan(theta), ctheta = cos(theta);
  dx[3] = p + sphi * ttheta * q + cphi * ttheta * r;
  dx[4] = cphi * q - sphi * r;
  dx[5] = (sphi * q + cphi * r) / ctheta;
  /* translational: thrust along the body z axis, rotated to the world */
  double stheta = sin(theta), spsi = sin(psi), cpsi = cos(psi);
  double thrust = T1 + T2 + T3 + T4;
  double bz_x = cphi * stheta * cpsi + sphi * spsi;
  double bz_y = cphi * stheta * spsi - sphi * cpsi;
  double bz_z = cphi * ctheta;
  dx[6] = thrust / m * bz_x;
  dx[7] = thrust / m * bz_y;
  dx[8] = thrust / m * bz_z - g;
  /* rotational: Euler's equations with a diagonal inertia */
  double tau_x = l * (T2 - T4);
  double tau_y = l * (T3 - T1);
  double tau_z = c * (T1 - T2 + T3 - T4);
  double Lx = Ix * p, Ly = Iy * q, Lz = Iz * r; /* I omega */
  double gx = q * Lz - r * Ly;                 /* omega x (I omega) */
  double gy = r * Lx - p * Lz;
  double gz = p * Ly - q * Lx;
  dx[9] = (tau_x - gx) / Ix;
  dx[10] = (tau_y - gy) / Iy;
  dx[11] = (tau_z - gz) / Iz;
}

static void vector_field(const kpo_config *cfg, const double *x,
                         const double *u, double *dx) {
  switch (cfg->system) {
  case KPO_DUBINS:
    f_dubins(x, u, dx);
    break;
  case KPO_QUAD:
    f_quad(cfg->phys, x, u, dx);
    break;
  default: /* double integrator */
    for (int i = 0; i < 3; ++i) {
      dx[i] = x[3 + i];
      dx[3 + i] = u[i];
    }
  }
}

static int state_dim(int system) { return system == KPO_QUAD ? 12 : 6; }

void kpo_step(const kpo_config *cfg, const double *x, const double *u,
              double h, double *x_out) {
  int d = state_dim(cfg->system);
  if (cfg->system == KPO_DI) {
    /* explicit Euler: x_{i+1} = x_i + h f(x_i, u) */
    double dx[12];
    vector_field(cfg, x, u, dx);
    for (int i = 0; i < d; ++i) x_out[i] = x[i] + h * dx[i];
    return;
  }
  /* classic fourth-order Runge-Kutta */
  double k1[12], k2[12], k3[12], k4[12], tmp[12];
  vector_field(cfg, x, u, k1);
  for (int i = 0; i < d; ++i) tmp[i] = x[i] + 0.5 * h * k1[i];
  vector_field(cfg, tmp, u, k2);
  for (int i = 0; i < d; ++i) tmp[i] = x[i] + 0.5 * h * k2[i];
  vector_field(cfg, tmp, u, k3);
  for (int i = 0; i < d; ++i) tmp[i] = x[i] + h * k3[i];
  vector_field(cfg, tmp, u, k4);
  for (int i = 0; i < d; ++i)
    x_out[i] = x[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

void kpo_propagate(const kpo_config *cfg, const double *x0, const double *u,
                   int32_t k, double *traj) {
  int d = state_dim(cfg->system);
  memcpy(traj, x0, sizeof(double) * d);
  for (int i = 0; i < k; ++i)
    kpo_step(cfg, traj + (size_t)i * d, u, cfg->dt, traj + (size_t)(i + 1) * d);
}

/* ------------------------------------------------------------------ */
/* validity                                                            */
/* ------------------------------------------------------------------ */

/* Returns 1 when the state lies in the closed state box.  *margin is the
 * smallest normalised distance to a bound (negative when violated: the
 * largest normalised violation). */
static int bounds_ok(const kpo *o, const double *x, double *margin) {
  double worst_in = INFINITY, worst_out = 0.0;
  int ok = 1;
  for (int i = 0; i < o->d; ++i) {
    double lo = o->cfg.x_lo[i], hi = o->cfg.x_hi[i];
    double scale = (isfinite(lo) && isfinite(hi)) ? (hi - lo) : 1.0;
    if (!(lo <= x[i] && x[i] <= hi)) { /* NaN is invalid too */
      ok = 0;
      double depth = isnan(x[i]) ? INFINITY
                                 : (x[i] < lo ? lo - x[i] : x[i] - hi) / scale;
      if (depth > worst_out) worst_out = depth;
    } else {
      double m = fmin(x[i] - lo, hi - x[i]) / scale;
      if (m < worst_in) worst_in = m;
    }
  }
  *margin = ok ? worst_in : -worst_out;
  return ok;
}

int32_t kpo_step_valid(const kpo *o, const double *x0, const double *x1,
                       double *margin) {
  double bmargin;
  int ok = bounds_ok(o, x1, &bmargin);
  /* axis-aligned box of the two positions */
  double slo[3], shi[3];
  for (int a = 0; a < 3; ++a) {
    slo[a] = fmin(x0[a], x1[a]);
    shi[a] = fmax(x0[a], x1[a]);
  }
  double min_sep = INFINITY; /* over boxes that are separated */
  double max_pen = 0.0;      /* over boxes that are hit       */
  int hit = 0;
  for (int b = 0; b < o->nb; ++b) {
    const double *bx = o->boxes + 6 * (size_t)b;
    /* per-axis gap between the two closed intervals; the boxes meet
     * exactly when no axis has a positive gap */
    double sep = -INFINITY;
    for (int a = 0; a < 3; ++a) {
      double scale = o->cfg.ws_hi[a] - o->cfg.ws_lo[a];
      double gap = fmax(bx[a] - shi[a], slo[a] - bx[3 + a]) / scale;
      if (gap > sep) sep = gap;
    }
    if (sep <= 0.0) {
      hit = 1;
      if (-sep > max_pen) max_pen = -sep;
    } else if (sep < min_sep) {
      min_sep = sep;
    }
  }
  if (ok && !hit) {
    *margin = fmin(bmargin, min_sep);
    return 1;
  }
  /* invalid: how far inside the invalid side the strongest violation is */
  double v = 0.0;
  if (!ok) v = fmax(v, -bmargin);
  if (hit) v = fmax(v, max_pen);
  *margin = v;
  return 0;
}

/* ------------------------------------------------------------------ */
/* binning                                                              */
/* ------------------------------------------------------------------ */

/* Cell of coordinate t (already scaled to cell units) among n cells,
 * clamped to [0, n-1]; *margin = distance (in cell units) to the nearest
 * interior face, i.e. a face whose crossing changes the cell. */
static int cell_of(double t, int n, double *margin) {
  int i;
  if (!(t >= 0.0)) /* also NaN */
    i = 0;
  else if (t >= (double)n)
    i = n - 1;
  else
    i = (int)floor(t);
  double m = INFINITY;
  if (isnan(t)) {
    m = 0.0;
  } else {
    for (int f = 1; f < n; ++f) {
      double dist = fabs(t - (double)f);
      if (dist < m) m = dist;
    }
  }
  *margin = m;
  return i;
}

static double speed_of(const kpo *o, const double *x) {
  switch (o->cfg.system) {
  case KPO_DUBINS:
    return fabs(x[5]);
  case KPO_QUAD:
    return sqrt(x[6] * x[6] + x[7] * x[7] + x[8] * x[8]);
  default:
    return sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
  }
}

/* ------------------------------------------------------------------ */
/* free-space-obeying decomposition (Sec. IV-B)                         */
/* ------------------------------------------------------------------ */

/* The regions are the leaves of a kd-tree over the workspace whose
 * splitting planes are obstacle faces.  A cell is split while some face of
 * a box that meets the cell's interior lies strictly inside it: on the axis
 * with the most distinct such face coordinates (the lowest axis on a tie),
 * at the lower median of them.  A leaf therefore has no obstacle face
 * crossing it, so it is either inside an obstacle or free of every one.
 * Nodes are numbered in depth-first pre-order, the left child (the side
 * below the plane) right after its parent; leaves are numbered in the same
 * order. */

static int cmp_double(const void *a, const void *b) {
  const double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

static int kd_push(kpo *o) {
  if (o->kd_n == o->kd_cap) {
    const int cap = o->kd_cap ? 2 * o->kd_cap : 64;
    o->kd_axis = (int *)realloc(o->kd_axis, sizeof(int) * (size_t)cap);
    o->kd_right = (int *)realloc(o->kd_right, sizeof(int) * (size_t)cap);
    o->kd_leaf = (int *)realloc(o->kd_leaf, sizeof(int) * (size_t)cap);
    o->kd_split = (double *)realloc(o->kd_split, sizeof(double) * (size_t)cap);
    o->kd_cap = cap;
  }
  return o->kd_n++;
}

static int kd_build(kpo *o, const double lo[3], const double hi[3], double *cand) {
  const int node = kd_push(o);
  int best_axis = -1, best_m = 0;
  double split = 0.0;
  for (int a = 0; a < 3; ++a) {
    int m = 0;
    for (int b = 0; b < o->nb; ++b) {
      const double *bx = o->boxes + 6 * (size_t)b;
      int meets = 1;
      for (int c = 0; c < 3; ++c)
        if (!(bx[c] < hi[c] && bx[3 + c] > lo[c])) meets = 0;
      if (!meets) continue;
      for (int s = 0; s < 2; ++s) {
        const double f = bx[3 * s + a];
        if (f > lo[a] && f < hi[a]) cand[m++] = f;
      }
    }
    qsort(cand, (size_t)m, sizeof(double), cmp_double);
    int u = 0;
    for (int i = 0; i < m; ++i)
      if (u == 0 || cand[i] != cand[u - 1]) cand[u++] = cand[i];
    if (u > best_m) {
      best_m = u;
      best_axis = a;
      split = cand[(u - 1) / 2];
    }
  }
  if (best_axis < 0) {
    if (o->n_leaves == KPO_FSO_MAX_LEAVES) return -1;
    const int leaf = o->n_leaves++;
    o->kd_axis[node] = 3;
    o->kd_leaf[node] = leaf;
    o->kd_right[node] = -1;
    o->kd_split[node] = 0.0;
    for (int a = 0; a < 3; ++a) {
      o->leaf_lo[3 * leaf + a] = lo[a];
      o->leaf_hi[3 * leaf + a] = hi[a];
    }
    return 0;
  }
  o->kd_axis[node] = best_axis;
  o->kd_leaf[node] = -1;
  o->kd_split[node] = split;
  double clo[3], chi[3];
  memcpy(clo, lo, sizeof clo);
  memcpy(chi, hi, sizeof chi);
  chi[best_axis] = split;
  if (kd_build(o, clo, chi, cand) != 0) return -1;
  o->kd_right[node] = o->kd_n;
  memcpy(chi, hi, sizeof chi);
  clo[best_axis] = split;
  return kd_build(o, clo, chi, cand);
}

int kpo_build_fso(kpo *o) {
  o->leaf_lo = (double *)calloc(3 * (size_t)KPO_FSO_MAX_LEAVES, sizeof(double));
  o->leaf_hi = (double *)calloc(3 * (size_t)KPO_FSO_MAX_LEAVES, sizeof(double));
  double *cand = (double *)malloc(sizeof(double) * (size_t)(2 * o->nb + 1));
  o->n_leaves = 0;
  o->kd_n = 0;
  const int rc = kd_build(o, o->cfg.ws_lo, o->cfg.ws_hi, cand);
  free(cand);
  if (rc != 0) return -1;
  /* Eq. 3's vol: each leaf's own workspace volume */
  o->region_vol = (double *)calloc((size_t)o->n_leaves, sizeof(double));
  for (int r = 0; r < o->n_leaves; ++r)
    o->region_vol[r] = (o->leaf_hi[3 * r] - o->leaf_lo[3 * r]) *
                       (o->leaf_hi[3 * r + 1] - o->leaf_lo[3 * r + 1]) *
                       (o->leaf_hi[3 * r + 2] - o->leaf_lo[3 * r + 2]);
  return 0;
}

int32_t kpo_fso_leaves(const kpo *o, double *lo, double *hi, int32_t cap) {
  if (!o->cfg.fso) return 0;
  for (int r = 0; r < o->n_leaves && r < cap; ++r)
    for (int a = 0; a < 3; ++a) {
      lo[3 * r + a] = o->leaf_lo[3 * r + a];
      hi[3 * r + a] = o->leaf_hi[3 * r + a];
    }
  return o->n_leaves;
}

/* Leaf of position p (descend: below the plane goes left) and the sub-grid
 * cell inside it; *margin = the nearest face crossed on the way or of the
 * sub-grid, in units of the workspace extent along its axis. */
static void bin_fso(const kpo *o, const double *x, int32_t *region, int32_t *sub,
                    double *margin) {
  double worst = INFINITY;
  int node = 0;
  while (o->kd_axis[node] != 3) {
    const int a = o->kd_axis[node];
    const double s = o->kd_split[node];
    const double m = fabs(x[a] - s) / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]);
    if (m < worst || isnan(m)) worst = isnan(m) ? 0.0 : m;
    node = x[a] < s ? node + 1 : o->kd_right[node];
  }
  const int r = o->kd_leaf[node];
  int fine[3];
  for (int a = 0; a < 3; ++a) {
    const int n = o->cfg.sub[a];
    const double lo = o->leaf_lo[3 * r + a], hi = o->leaf_hi[3 * r + a];
    double m;
    fine[a] = cell_of((x[a] - lo) * ((double)n / (hi - lo)), n, &m);
    m *= (hi - lo) / (double)n / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]);
    if (m < worst) worst = m;
  }
  const int k = fine[0] + o->cfg.sub[0] * (fine[1] + o->cfg.sub[1] * fine[2]);
  *region = r;
  *sub = r * o->n_sub_per + k;
  if (margin) *margin = worst;
}

void kpo_bin(const kpo *o, const double *x, int32_t *region, int32_t *sub,
             double *margin) {
  if (o->cfg.fso) {
    bin_fso(o, x, region, sub, margin);
    return;
  }
  int cell[3], fine[3];
  double worst = INFINITY;
  for (int a = 0; a < 3; ++a) {
    int n = o->cfg.grid[a] * o->cfg.sub[a]; /* fine cells along the axis */
    double t = (x[a] - o->cfg.ws_lo[a]) *
               ((double)n / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]));
    double m;
    fine[a] = cell_of(t, n, &m);
    m /= (double)n; /* to normalised workspace units */
    if (m < worst) worst = m;
    cell[a] = fine[a] / o->cfg.sub[a];
    fine[a] = fine[a] % o->cfg.sub[a];
  }
  int sb = 0;
  if (o->cfg.speed_bins > 1) {
    double m;
    double t = speed_of(o, x) * ((double)o->cfg.speed_bins / o->cfg.speed_hi);
    sb = cell_of(t, o->cfg.speed_bins, &m);
    m /= (double)o->cfg.speed_bins;
    if (m < worst) worst = m;
  }
  /* further state dimensions of a state-space grid, slowest in the index:
   * e = c_3 + n_3 (c_4 + n_4 (...)) over the decomposed dimensions */
  int e = 0, stride = 1;
  for (int dd = 3; dd < o->d; ++dd) {
    const int n = o->cfg.state_grid[dd];
    if (n <= 1) continue;
    double t;
    if (isfinite(o->cfg.x_lo[dd]) && isfinite(o->cfg.x_hi[dd])) {
      t = (x[dd] - o->cfg.x_lo[dd]) * ((double)n / (o->cfg.x_hi[dd] - o->cfg.x_lo[dd]));
    } else {
      const double pi = 3.14159265358979323846;
      const double y = x[dd] - 2.0 * pi * floor((x[dd] + pi) / (2.0 * pi));
      t = (y + pi) * ((double)n / (2.0 * pi));
    }
    double m;
    const int c = cell_of(t, n, &m);
    if (!(isfinite(o->cfg.x_lo[dd]) && isfinite(o->cfg.x_hi[dd]))) {
      /* -pi and pi are the same face of a wrapped dimension */
      if (t < m) m = t;
      if ((double)n - t < m) m = (double)n - t;
    }
    m /= (double)n;
    if (m < worst) worst = m;
    e += stride * c;
    stride *= n;
  }
  int gx = o->cfg.grid[0], gy = o->cfg.grid[1], gz = o->cfg.grid[2];
  const int nsb = o->cfg.speed_bins > 1 ? o->cfg.speed_bins : 1;
  int r = cell[0] + gx * (cell[1] + gy * (cell[2] + gz * (sb + nsb * e)));
  int k = fine[0] + o->cfg.sub[0] * (fine[1] + o->cfg.sub[1] * fine[2]);
  *region = r;
  *sub = r * o->n_sub_per + k;
  if (margin) *margin = worst;
}

/* ------------------------------------------------------------------ */
/* dense re-validation of an edge                                       */
/* ------------------------------------------------------------------ */

/* Violation depth of a single state: bounds and point-in-closed-box. */
static double point_violation(const kpo *o, const double *x) {
  double bm;
  double v = 0.0;
  if (!bounds_ok(o, x, &bm)) v = -bm;
  for (int b = 0; b < o->nb; ++b) {
    const double *bx = o->boxes + 6 * (size_t)b;
    double pen = INFINITY;
    for (int a = 0; a < 3; ++a) {
      double scale = o->cfg.ws_hi[a] - o->cfg.ws_lo[a];
      double in = fmin(x[a] - bx[a], bx[3 + a] - x[a]) / scale;
      if (in < pen) pen = in;
    }
    /* pen >= 0 means inside the closed box; report a touch as a tiny
     * positive depth so that it is never mistaken for 'valid' */
    if (pen >= 0.0) v = fmax(v, fmax(pen, 1e-300));
  }
  return v;
}

double kpo_dense_check(const kpo *o, const double *x0, const double *u,
                       int32_t k, int32_t sub, double *x_end) {
  double x[12], nx[12], y[12];
  int d = o->d;
  memcpy(x, x0, sizeof(double) * d);
  double worst = 0.0;
  for (int i = 0; i < k; ++i) {
    kpo_step(&o->cfg, x, u, o->cfg.dt, nx); /* the integrator's own step */
    if (o->cfg.system == KPO_DI) {
      /* the Euler step is a straight segment in position: sample it */
      for (int s = 1; s <= sub; ++s) {
        double w = (double)s / (double)sub;
        for (int j = 0; j < d; ++j) y[j] = x[j] + w * (nx[j] - x[j]);
        worst = fmax(worst, point_violation(o, y));
      }
    } else {
      /* re-integrate the step with 'sub' RK4 sub-steps */
      memcpy(y, x, sizeof(double) * d);
      for (int s = 1; s <= sub; ++s) {
        double z[12];
        kpo_step(&o->cfg, y, u, o->cfg.dt / (double)sub, z);
        memcpy(y, z, sizeof(double) * d);
        worst = fmax(worst, point_violation(o, y));
      }
    }
    memcpy(x, nx, sizeof(double) * d);
  }
  if (x_end) memcpy(x_end, x, sizeof(double) * d);
  return worst;
}
