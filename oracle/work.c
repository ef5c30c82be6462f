/*
 * work.c -- algorithmic work of the expansion, counted during replay
 * (oracle side).
 *
 * TEST INFRASTRUCTURE ONLY (see kpo.h).
 *
 * The measurement of the hot path reports achieved useful lane operations
 * per second.  Useful work is what Propagate (Algorithm 2) must compute for
 * the samples it draws, under this counting rule:
 *   - one lane operation per arithmetic or logic operation a lane needs;
 *     no addressing, loop control, padding, divergence or data movement;
 *   - a Philox4x32-10 block: 10 rounds of 6 integer operations (two
 *     32x32 -> 64-bit products counted as 2 each, two xors), 60 per block,
 *     two blocks per sample (controls; duration, accept draw, selector);
 *   - sine and cosine of one angle: 6 (a 2 pi argument reduction of 4:
 *     scale, round, two fused multiply-adds; then 1 each for the two
 *     hardware approximations); a correctly rounded division or
 *     reciprocal: 4;
 *   - per integrator step: the integrator's own multiplies and adds, then
 *     the state-box test (2 compares per state entry); terms that depend
 *     on the control alone (the quadrotor's thrust and torques) once per
 *     sample;
 *   - per step whose end state is in the state box: the step's hull (6
 *     min/max over the two positions) and 8 operations per box tested;
 *   - per sample: the control map (4 per control: 24-bit word to [0, 1)
 *     by shift, convert and scale, then the affine map), the duration (2),
 *     the accept-draw compare (1), binning (20) and the counter and claim
 *     updates (2).
 * Box tests (counted once a work grid is set: they are slow to count) are
 * counted two ways: a linear scan of the obstacles in index
 * order that stops at the first box the hull meets (the method's plain
 * checker), and the same over the boxes listed in the uniform-grid cells
 * the hull overlaps, visited cell by cell (z slowest, then y, then x) with
 * each cell's boxes in index order, stopping at the first box met (the
 * broad phase; the grid shape is an input).  The broad phase first looks up
 * the clearance of the cell holding the hull's low corner: the smallest, over
 * boxes, of the largest per-axis gap between the cell and the box in that
 * axis's cell units, at most 4 cells, less 1e-3, counted in whole sixteenths
 * of a cell; a hull inside the cell grown by that much on every side is
 * tested against no box.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kpo_internal.h"

#define W_PHILOX_BLOCK 60
#define W_SINCOS 6
#define W_DIV 4
#define W_CONTROL 4
#define W_DURATION 2
#define W_ACCEPT 1
#define W_BIN 20
#define W_COUNT 2
#define W_BOUND 2
#define W_HULL 6
#define W_BOX 8

/* Integrator operations of one step (Eq. 1-2 of each system). */
static uint64_t integrator_ops(int system) {
  switch (system) {
    case KPO_DI:
      /* explicit Euler: p += h v and v += h u on 3 axes, one FMA each */
      return 3 * 2;
    case KPO_DUBINS:
      /* RK4: 4 field evaluations (sin/cos of yaw and pitch, then 5
       * products), 3 stage points (6 FMA each), the combination (4 per
       * entry), and the step constants h/2 (1) and h/6 (a division) */
      return 4 * (2 * W_SINCOS + 5) + 3 * 6 + 6 * 4 + 1 + W_DIV;
    default:
      /* RK4: 4 field evaluations (sin/cos of roll, pitch and yaw, the
       * reciprocal of cos(pitch), and 34 multiplies and adds: Euler-angle
       * rates 10, the thrust rotated to the world frame 9, the rigid-body
       * rotation I w' = tau - w x (I w) 15), 3 stage points (12 FMA each),
       * the combination (4 per entry) and the step constants (1 + a
       * division) */
      return 4 * (3 * W_SINCOS + W_DIV + 34) + 3 * 12 + 12 * 4 + 1 + W_DIV;
  }
}

/* Operations that depend on the sample's control alone (once per sample). */
static uint64_t control_only_ops(int system) {
  /* quadrotor: total thrust (3 adds) and its scaling (1), the three body
   * torques (2 + 2 + 4) */
  return system == KPO_QUAD ? 3 + 1 + 2 + 2 + 4 : 0;
}

uint64_t kpo_work_ops_sample(const kpo *o) {
  return 2 * W_PHILOX_BLOCK + (uint64_t)o->N * W_CONTROL + W_DURATION + W_ACCEPT + W_BIN +
         W_COUNT + control_only_ops(o->cfg.system);
}

uint64_t kpo_work_ops_step(const kpo *o) {
  return integrator_ops(o->cfg.system) + (uint64_t)o->d * W_BOUND;
}

uint64_t kpo_work_ops_hull(void) { return W_HULL; }
uint64_t kpo_work_ops_box(void) { return W_BOX; }

/* Cell of coordinate v along axis a of the work grid (clamped). */
static int wcell(const kpo *o, int a, double v) {
  const int g = o->wgrid[a];
  const double t = (v - o->cfg.ws_lo[a]) * ((double)g / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]));
  if (!(t >= 0.0)) return 0;
  if (t >= (double)g) return g - 1;
  return (int)floor(t);
}

static int box_meets(const double *bx, const double *lo, const double *hi) {
  for (int a = 0; a < 3; ++a)
    if (!(lo[a] <= bx[3 + a] && bx[a] <= hi[a])) return 0;
  return 1;
}

void kpo_step_work(kpo *o, const double *x0, const double *x1) {
  o->work.steps += 1;
  o->work.ops += kpo_work_ops_step(o);
  for (int i = 0; i < o->d; ++i) {
    const double lo = o->cfg.x_lo[i], hi = o->cfg.x_hi[i];
    if (!(lo <= x1[i] && x1[i] <= hi)) return; /* no hull test */
  }
  o->work.hulls += 1;
  o->work.ops += W_HULL;
  if (!o->wbox) return; /* box tests are counted once a work grid is set */
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = fmin(x0[a], x1[a]);
    hi[a] = fmax(x0[a], x1[a]);
  }
  /* linear scan in box order */
  for (int b = 0; b < o->nb; ++b) {
    o->work.box_scan += 1;
    if (box_meets(o->boxes + 6 * (size_t)b, lo, hi)) break;
  }
  /* the boxes of the grid cells the hull overlaps, unless the hull lies in
   * its low corner's cell grown by the cell's clearance */
  int c0[3], c1[3];
  for (int a = 0; a < 3; ++a) {
    c0[a] = wcell(o, a, lo[a]);
    c1[a] = wcell(o, a, hi[a]);
  }
  {
    const double r =
        o->wclear[c0[0] + o->wgrid[0] * (c0[1] + o->wgrid[1] * c0[2])] / 16.0;
    int inside = r > 0.0;
    for (int a = 0; a < 3 && inside; ++a) {
      const double s = (double)o->wgrid[a] / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]);
      const double tl = (lo[a] - o->cfg.ws_lo[a]) * s, th = (hi[a] - o->cfg.ws_lo[a]) * s;
      if (!(tl >= c0[a] - r && th <= c0[a] + 1 + r)) inside = 0;
    }
    if (inside) return;
  }
  uint64_t n = 0;
  int hit = 0;
  for (int cz = c0[2]; cz <= c1[2] && !hit; ++cz)
    for (int cy = c0[1]; cy <= c1[1] && !hit; ++cy)
      for (int cx = c0[0]; cx <= c1[0] && !hit; ++cx) {
        const int c[3] = {cx, cy, cz};
        for (int b = 0; b < o->nb && !hit; ++b) {
          const int32_t *cr = o->wbox + 6 * (size_t)b; /* the box's cell range */
          int listed = 1;
          for (int a = 0; a < 3; ++a)
            if (c[a] < cr[a] || c[a] > cr[3 + a]) listed = 0;
          if (!listed) continue;
          ++n;
          if (box_meets(o->boxes + 6 * (size_t)b, lo, hi)) hit = 1;
        }
      }
  o->work.box_grid += n;
  o->work.ops += W_BOX * n;
}

void kpo_sample_work(kpo *o) {
  o->work.samples += 1;
  o->work.ops += kpo_work_ops_sample(o);
}

void kpo_set_work_grid(kpo *o, const int32_t g[3]) {
  for (int a = 0; a < 3; ++a) o->wgrid[a] = g[a] > 0 ? g[a] : 1;
  free(o->wbox);
  o->wbox = (int32_t *)malloc(sizeof(int32_t) * 6 * (size_t)(o->nb > 0 ? o->nb : 1));
  for (int b = 0; b < o->nb; ++b)
    for (int a = 0; a < 3; ++a) {
      o->wbox[6 * (size_t)b + a] = wcell(o, a, o->boxes[6 * (size_t)b + a]);
      o->wbox[6 * (size_t)b + 3 + a] = wcell(o, a, o->boxes[6 * (size_t)b + 3 + a]);
    }
  /* each cell's clearance: the L-infinity gap (per axis in cell units) to
   * the nearest box, at most 4 cells, less 1e-3, in whole sixteenths */
  const int C = o->wgrid[0] * o->wgrid[1] * o->wgrid[2];
  free(o->wclear);
  o->wclear = (int32_t *)malloc(sizeof(int32_t) * (size_t)C);
  for (int c = 0; c < C; ++c) {
    const int cc[3] = {c % o->wgrid[0], (c / o->wgrid[0]) % o->wgrid[1],
                       c / (o->wgrid[0] * o->wgrid[1])};
    double r = 4.0;
    for (int b = 0; b < o->nb; ++b) {
      double gap = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double s = (double)o->wgrid[a] / (o->cfg.ws_hi[a] - o->cfg.ws_lo[a]);
        const double bl = (o->boxes[6 * (size_t)b + a] - o->cfg.ws_lo[a]) * s;
        const double bh = (o->boxes[6 * (size_t)b + 3 + a] - o->cfg.ws_lo[a]) * s;
        gap = fmax(gap, fmax(bl - (cc[a] + 1), cc[a] - bh));
      }
      r = fmin(r, gap);
    }
    const double v = (r - 1e-3) * 16.0;
    o->wclear[c] = v >= 1.0 ? (int32_t)fmin(255.0, floor(v)) : 0;
  }
}

void kpo_get_work(const kpo *o, kpo_work *out) { *out = o->work; }

void kpo_clear_work(kpo *o) { memset(&o->work, 0, sizeof o->work); }

int32_t kpo_work_clearance(const kpo *o, int32_t *out) {
  const int C = o->wgrid[0] * o->wgrid[1] * o->wgrid[2];
  if (!o->wclear) return 0;
  memcpy(out, o->wclear, sizeof(int32_t) * (size_t)C);
  return C;
}
