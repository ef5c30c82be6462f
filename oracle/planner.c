/*
 * planner.c -- Kino-PAX main loop in double precision (oracle side).
 *
 * TEST INFRASTRUCTURE ONLY (see kpo.h).
 *
 * One call of kpo_iterate is one pass of the Algorithm 1 loop body:
 *   Propagate (Algorithm 2) -> UpdateEstimates (Algorithm 3, Eq. 3-5)
 *   -> UpdateNodeSets (Algorithm 4), with lambda from Eq. 6.
 *
 * Where the paper leaves a choice open this file takes the following
 * readings (each is also listed with its reason in the design notes):
 *  R1 duration: dt in (0, T_prop] is drawn as an integer number k of
 *     integrator steps, k uniform in [k_min, k_max].
 *  R2 validity: checked after every integrator step (state box, and the
 *     axis-aligned box of the step's two positions against every closed
 *     obstacle); the sample stops at its first invalid step.
 *  R3 region of an invalid sample: the state at its first invalid step.
 *  R5 "unvisited" under parallel expansion: visited flags are those at the
 *     start of the pass; among the valid samples that reach an unvisited
 *     sub-region the one with the smallest sample key is its
 *     representative; all other valid samples take the P_accept draw.
 *  R6 node sets: every node already in the tree makes one draw against the
 *     P_accept of its region computed in this pass; it is in V_E next iff
 *     the draw succeeds, otherwise in V_O.  New nodes enter V_E.
 *  R7 R_avail (regions holding a tree node) includes this pass's new
 *     nodes; regions outside R_avail keep P_accept = 1; n_valid/n_invalid
 *     are cumulative.  New nodes are appended before UpdateEstimates.
 *  R9 goal: the final state of each new node is tested; the smallest node
 *     id among new goal nodes is returned.
 *  R11 Eq. 3-5 are evaluated in the fixed order written in kpo_eq345 and
 *     the sum in Eq. 5 is a pairwise sum over the region array in index
 *     order, padded with zeros to a power of two.  A draw w (a 32-bit
 *     Philox word) succeeds iff w < thr, thr = floor(P * 2^32) (2^32 when
 *     P >= 1).
 * Random stream: Philox4x32-10 keyed by the 64-bit seed; counter
 * (iteration, node id, sample j, purpose) with purpose 0 = control words,
 * 1 = (duration, accept draw, selector, spare), 2 = node-set draw (j = 0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kpo_internal.h"

#define TWO32 4294967296.0

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

int32_t kpo_state_dim(const kpo *o) { return o->d; }
int32_t kpo_control_dim(const kpo *o) { return o->N; }
int32_t kpo_num_regions(const kpo *o) { return o->R; }
int32_t kpo_num_subregions(const kpo *o) { return o->n_sub; }
int32_t kpo_status(const kpo *o) { return o->status; }
int32_t kpo_goal_node(const kpo *o) { return o->goal_node; }
int32_t kpo_num_nodes(const kpo *o) { return o->n; }
int32_t kpo_iteration(const kpo *o) { return o->iteration; }

kpo *kpo_create(const kpo_config *cfg, const float *boxes, int32_t n_boxes) {
  if (cfg->t_e < 1 || cfg->lambda_max < 1 || cfg->k_min < 1 ||
      cfg->k_max < cfg->k_min || n_boxes < 0)
    return NULL;
  kpo *o = (kpo *)xcalloc(1, sizeof(kpo));
  o->cfg = *cfg;
  o->d = cfg->system == KPO_QUAD ? 12 : 6;
  o->N = cfg->system == KPO_QUAD ? 4 : 3;
  int sb = cfg->speed_bins > 1 ? cfg->speed_bins : 1;
  o->cfg.speed_bins = sb;
  o->R = cfg->grid[0] * cfg->grid[1] * cfg->grid[2] * sb;
  for (int dd = 0; dd < 12; ++dd) {
    if (dd < 3 || dd >= o->d || o->cfg.state_grid[dd] < 1) o->cfg.state_grid[dd] = 1;
    o->R *= o->cfg.state_grid[dd];
  }
  o->n_sub_per = cfg->sub[0] * cfg->sub[1] * cfg->sub[2];
  o->vol = 1.0;
  for (int a = 0; a < 3; ++a)
    o->vol *= (cfg->ws_hi[a] - cfg->ws_lo[a]) / (double)cfg->grid[a];
  o->nb = n_boxes;
  o->boxes = (double *)xcalloc((size_t)n_boxes * 6, sizeof(double));
  for (int i = 0; i < 6 * n_boxes; ++i) o->boxes[i] = (double)boxes[i];
  if (cfg->fso) {
    /* the regions are the kd-tree's leaves, each with its own volume */
    if (kpo_build_fso(o) != 0) {
      kpo_destroy(o);
      return NULL;
    }
    o->R = o->n_leaves;
  }
  o->n_sub = o->R * o->n_sub_per;
  size_t te = (size_t)cfg->t_e;
  o->x = (double *)xcalloc(te * o->d, sizeof(double));
  o->parent = (int *)xcalloc(te, sizeof(int));
  o->u = (double *)xcalloc(te * o->N, sizeof(double));
  o->steps = (int *)xcalloc(te, sizeof(int));
  o->region = (int *)xcalloc(te, sizeof(int));
  o->sub = (int *)xcalloc(te, sizeof(int));
  o->in_ve = (unsigned char *)xcalloc(te, 1);
  o->n_valid = (uint64_t *)xcalloc(o->R, sizeof(uint64_t));
  o->n_invalid = (uint64_t *)xcalloc(o->R, sizeof(uint64_t));
  o->cov = (uint32_t *)xcalloc(o->R, sizeof(uint32_t));
  o->avail = (unsigned char *)xcalloc(o->R, 1);
  o->visited = (unsigned char *)xcalloc(o->n_sub, 1);
  o->score = (double *)xcalloc(o->R, sizeof(double));
  o->p_accept = (double *)xcalloc(o->R, sizeof(double));
  o->thr = (uint64_t *)xcalloc(o->R, sizeof(uint64_t));
  o->status = KPO_ERR;
  o->goal_node = -1;
  o->wgrid[0] = o->wgrid[1] = o->wgrid[2] = 1;
  return o;
}

void kpo_destroy(kpo *o) {
  if (!o) return;
  free(o->boxes); free(o->x); free(o->parent); free(o->u); free(o->steps);
  free(o->region); free(o->sub); free(o->in_ve); free(o->n_valid);
  free(o->n_invalid); free(o->cov); free(o->avail); free(o->visited);
  free(o->score); free(o->p_accept); free(o->thr); free(o->mlp);
  free(o->kd_axis); free(o->kd_right); free(o->kd_leaf); free(o->kd_split);
  free(o->leaf_lo); free(o->leaf_hi); free(o->region_vol); free(o->wbox); free(o->wclear);
  free(o);
}

/* ------------------------------------------------------------------ */
/* Eq. 3-5 and Eq. 6                                                    */
/* ------------------------------------------------------------------ */

/* Pairwise sum of a[lo .. lo+n), n a power of two; entries at or past
 * 'len' are the zero padding. */
static double pairwise(const double *a, int len, int lo, int n) {
  if (n == 1) return lo < len ? a[lo] : 0.0;
  return pairwise(a, len, lo, n / 2) + pairwise(a, len, lo + n / 2, n / 2);
}

void kpo_eq345(int32_t n, const uint32_t *n_valid, const uint32_t *n_invalid,
               const uint32_t *cov, const uint8_t *avail, double vol,
               double delta, double eps, double *score, double *p_accept,
               uint64_t *thr, double *score_sum) {
  double *v = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) v[i] = vol;
  kpo_eq345_vol(n, n_valid, n_invalid, cov, avail, v, delta, eps, score, p_accept, thr,
                score_sum);
  free(v);
}

void kpo_eq345_vol(int32_t n, const uint32_t *n_valid, const uint32_t *n_invalid,
                   const uint32_t *cov, const uint8_t *avail, const double *vol_r,
                   double delta, double eps, double *score, double *p_accept,
                   uint64_t *thr, double *score_sum) {
  for (int i = 0; i < n; ++i) {
    score[i] = 0.0;
    if (!avail[i]) continue;
    const double vol = vol_r[i];
    double nv = (double)n_valid[i], ni = (double)n_invalid[i];
    /* Eq. 3: FreeVol = (delta + n_valid) vol / (delta + n_valid + n_invalid) */
    double freevol = ((delta + nv) * vol) / ((delta + nv) + ni);
    /* Eq. 4: Score = FreeVol^4 / ((1 + Cov) (1 + (n_valid + n_invalid)^2)) */
    double f4 = (freevol * freevol) * (freevol * freevol);
    double n_all = nv + ni;
    double den = (1.0 + (double)cov[i]) * (1.0 + n_all * n_all);
    score[i] = f4 / den;
  }
  int p2 = 1;
  while (p2 < n) p2 *= 2;
  double sum = n > 0 ? pairwise(score, n, 0, p2) : 0.0;
  for (int i = 0; i < n; ++i) {
    double p;
    if (!avail[i]) {
      p = 1.0; /* Algorithm 1 starts every region at 1; regions without a node keep it */
    } else if (sum > 0.0) {
      /* Eq. 5: P_accept = min{1, Score / sum over R_avail + eps} */
      p = score[i] / sum + eps;
      if (p > 1.0) p = 1.0;
    } else {
      p = eps < 1.0 ? eps : 1.0; /* every score underflowed */
    }
    p_accept[i] = p;
    thr[i] = p >= 1.0 ? (uint64_t)1 << 32 : (uint64_t)floor(p * TWO32);
  }
  if (score_sum) *score_sum = sum;
}

void kpo_region_volumes(const kpo *o, double *vol) {
  for (int r = 0; r < o->R; ++r) vol[r] = o->region_vol ? o->region_vol[r] : o->vol;
}

int32_t kpo_lambda(int32_t t_e, int32_t n_tree, int32_t n_ve,
                   int32_t lambda_max) {
  if (n_ve <= 0) return lambda_max;
  int32_t room = t_e - n_tree;
  if (room < 0) room = 0;
  int32_t lam = room / n_ve; /* floor: both non-negative */
  return lam < lambda_max ? lam : lambda_max;
}

/* ------------------------------------------------------------------ */
/* helpers                                                              */
/* ------------------------------------------------------------------ */

static double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

static int in_goal(const kpo *o, const double *x, double *margin) {
  double dx = x[0] - o->cfg.goal_c[0], dy = x[1] - o->cfg.goal_c[1],
         dz = x[2] - o->cfg.goal_c[2];
  double dist = sqrt(dx * dx + dy * dy + dz * dz);
  if (margin) *margin = fabs(dist - o->cfg.goal_r);
  return dist <= o->cfg.goal_r;
}

/* Plain definitions of the region metrics that follow from the tree:
 * R_avail = regions holding a tree node, Cov = visited sub-regions. */
static void refresh_region_sets(kpo *o) {
  memset(o->avail, 0, (size_t)o->R);
  for (int v = 0; v < o->n; ++v) o->avail[o->region[v]] = 1;
  for (int r = 0; r < o->R; ++r) {
    uint32_t c = 0;
    for (int k = 0; k < o->n_sub_per; ++k) c += o->visited[r * o->n_sub_per + k];
    o->cov[r] = c;
  }
}

static void update_estimates(kpo *o) {
  /* Algorithm 3 on the uint32 views of the cumulative counters */
  uint32_t *nv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)o->R);
  uint32_t *ni = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)o->R);
  for (int r = 0; r < o->R; ++r) {
    nv[r] = (uint32_t)o->n_valid[r];
    ni[r] = (uint32_t)o->n_invalid[r];
  }
  if (o->region_vol)
    kpo_eq345_vol(o->R, nv, ni, o->cov, o->avail, o->region_vol, o->cfg.delta, o->cfg.eps,
                  o->score, o->p_accept, o->thr, &o->score_sum);
  else
    kpo_eq345(o->R, nv, ni, o->cov, o->avail, o->vol, o->cfg.delta, o->cfg.eps,
              o->score, o->p_accept, o->thr, &o->score_sum);
  free(nv);
  free(ni);
}

static void draw(const kpo *o, uint32_t it, uint32_t node, uint32_t j,
                 uint32_t purpose, uint32_t out[4]) {
  uint32_t ctr[4] = {it, node, j, purpose};
  uint32_t key[2] = {(uint32_t)(o->cfg.seed & 0xffffffffu),
                     (uint32_t)(o->cfg.seed >> 32)};
  kpo_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* learned proposal                                                     */
/* ------------------------------------------------------------------ */

#define PI_ 3.14159265358979323846

void kpo_features(const kpo *o, int32_t v, double *f) {
  const double *x = o->x + (size_t)v * o->d;
  for (int i = 0; i < 32; ++i) f[i] = 0.0;
  for (int i = 0; i < 6 && i < o->d; ++i) {
    const double lo = o->cfg.x_lo[i], hi = o->cfg.x_hi[i];
    if (isfinite(lo) && isfinite(hi) && hi > lo)
      f[i] = 2.0 * (x[i] - lo) / (hi - lo) - 1.0;
    else
      f[i] = (x[i] - 2.0 * PI_ * floor((x[i] + PI_) / (2.0 * PI_))) / PI_;
  }
  for (int a = 0; a < 3; ++a) f[6 + a] = o->cfg.goal_c[a] - x[a];
  const int r = o->region[v];
  const double nv = (double)o->n_valid[r], ni = (double)o->n_invalid[r];
  f[9] = (double)o->cov[r] / (double)o->n_sub_per;
  f[10] = (o->cfg.delta + nv) / (o->cfg.delta + nv + ni);
  f[11] = log1p(nv);
  f[12] = log1p(ni);
  f[13] = (double)o->thr[r] / TWO32;
  /* face neighbours in the position grid, same speed bin (none when the
   * regions are kd-tree leaves) */
  if (o->cfg.fso) return;
  const int gx = o->cfg.grid[0], gy = o->cfg.grid[1], gz = o->cfg.grid[2];
  const int cx = r % gx, cy = (r / gx) % gy, cz = (r / (gx * gy)) % gz;
  const int sb = r / (gx * gy * gz);
  const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dz[6] = {0, 0, 0, 0, -1, 1};
  for (int k = 0; k < 6; ++k) {
    const int nx = cx + dx[k], ny = cy + dy[k], nz = cz + dz[k];
    if (nx < 0 || nx >= gx || ny < 0 || ny >= gy || nz < 0 || nz >= gz) continue;
    const int rn = nx + gx * (ny + gy * (nz + gz * sb));
    f[14 + k] = (double)o->thr[rn] / TWO32;
  }
}

void kpo_box_muller(const uint32_t w[4], double z[4]) {
  for (int pr = 0; pr < 2; ++pr) {
    const double r1 = ((double)(w[2 * pr] >> 8) + 1.0) * (1.0 / 16777216.0); /* (0, 1] */
    const double r2 = (double)(w[2 * pr + 1] >> 8) * (1.0 / 16777216.0);   /* [0, 1) */
    const double rad = sqrt(-2.0 * log(r1));
    z[2 * pr] = rad * cos(2.0 * PI_ * r2);
    z[2 * pr + 1] = rad * sin(2.0 * PI_ * r2);
  }
}

int32_t kpo_set_mlp(kpo *o, const float *params, double mix) {
  free(o->mlp);
  o->mlp = NULL;
  if (!params) return 0;
  if (o->d != 6) return KPO_ERR;
  const int n = kpo_mlp_num_params();
  o->mlp = (double *)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; ++i) o->mlp[i] = (double)params[i];
  o->mix = mix;
  return 0;
}

int32_t kpo_set_harvest(kpo *o, double *feat, double *target, int32_t capacity) {
  o->hv_feat = feat;
  o->hv_target = target;
  o->hv_cap = capacity;
  o->hv_count = 0;
  return 0;
}

int32_t kpo_harvest_count(const kpo *o) { return o->hv_count; }

/* ------------------------------------------------------------------ */
/* Algorithm 1, initialisation                                         */
/* ------------------------------------------------------------------ */

int32_t kpo_reset(kpo *o, const float *x_init) {
  double x[12];
  for (int i = 0; i < o->d; ++i) x[i] = (double)x_init[i];
  double m;
  /* x_init must be valid: a zero-length step checks the point itself */
  if (!kpo_step_valid(o, x, x, &m)) {
    o->status = KPO_ERR;
    return KPO_ERR;
  }
  o->n = 1;
  memcpy(o->x, x, sizeof(double) * o->d);
  o->parent[0] = -1;
  memset(o->u, 0, sizeof(double) * o->N);
  o->steps[0] = 0;
  kpo_bin(o, x, &o->region[0], &o->sub[0], NULL);
  o->in_ve[0] = 1; /* V_E = {x_init} */
  memset(o->n_valid, 0, sizeof(uint64_t) * o->R);
  memset(o->n_invalid, 0, sizeof(uint64_t) * o->R);
  memset(o->visited, 0, (size_t)o->n_sub);
  o->visited[o->sub[0]] = 1;
  refresh_region_sets(o);
  for (int r = 0; r < o->R; ++r) { /* P_accept = 1 for every region */
    o->p_accept[r] = 1.0;
    o->thr[r] = (uint64_t)1 << 32;
    o->score[r] = 0.0;
  }
  o->score_sum = 0.0;
  o->iteration = 0;
  o->goal_node = -1;
  o->status = KPO_RUNNING;
  kpo_clear_work(o);
  if (in_goal(o, x, NULL)) {
    o->goal_node = 0;
    o->status = KPO_SOLVED;
  }
  return o->status;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 loop body                                                */
/* ------------------------------------------------------------------ */

int32_t kpo_iterate(kpo *o, kpo_records *rec, kpo_iter_stats *st) {
  if (o->status != KPO_RUNNING) return o->status;
  const int d = o->d, N = o->N;
  const uint32_t it = (uint32_t)o->iteration;

  /* V_E in ascending node id */
  int *ve = (int *)malloc(sizeof(int) * (size_t)(o->n > 0 ? o->n : 1));
  int nve = 0;
  for (int v = 0; v < o->n; ++v)
    if (o->in_ve[v]) ve[nve++] = v;

  /* Eq. 6 */
  int lambda = kpo_lambda(o->cfg.t_e, o->n, nve, o->cfg.lambda_max);
  if (nve > 0 && lambda == 0) {
    free(ve);
    o->status = KPO_FULL;
    return o->status;
  }
  int S = nve * lambda;

  /* per-sample working arrays */
  double *xs = (double *)xcalloc((size_t)S * d, sizeof(double));
  double *us = (double *)xcalloc((size_t)S * N, sizeof(double));
  int *ks = (int *)xcalloc((size_t)S, sizeof(int));
  int *rs = (int *)xcalloc((size_t)S, sizeof(int));
  int *ss = (int *)xcalloc((size_t)S, sizeof(int));
  unsigned char *fl = (unsigned char *)xcalloc((size_t)S, 1);
  unsigned char *visited0 = (unsigned char *)malloc((size_t)o->n_sub);
  memcpy(visited0, o->visited, (size_t)o->n_sub);
  double *traj = (double *)malloc(sizeof(double) * (size_t)(o->cfg.k_max + 1) * d);

  /* learned proposal: features and network outputs per expanded node */
  double *feat = NULL, *net = NULL;
  if (o->mlp || o->hv_feat) {
    feat = (double *)malloc(sizeof(double) * 32 * (size_t)(nve > 0 ? nve : 1));
    for (int p = 0; p < nve; ++p) kpo_features(o, ve[p], feat + 32 * (size_t)p);
  }
  if (o->mlp) {
    net = (double *)malloc(sizeof(double) * 8 * (size_t)(nve > 0 ? nve : 1));
    kpo_mlp_forward(o->mlp, feat, nve, net);
  }
  const uint64_t mix_thr = o->mlp ? (uint64_t)floor(o->mix * TWO32) : 0;

  /* ---------------- Algorithm 2: Propagate ---------------- */
  int n_valid_total = 0;
  for (int p = 0; p < nve; ++p) {
    int v = ve[p];
    for (int j = 0; j < lambda; ++j) {
      int key = p * lambda + j;
      uint32_t w0[4], w1[4];
      draw(o, it, (uint32_t)v, (uint32_t)j, 0, w0);
      draw(o, it, (uint32_t)v, (uint32_t)j, 1, w1);
      /* random control u in U and duration k * dt */
      double u[4];
      for (int i = 0; i < N; ++i)
        u[i] = o->cfg.u_lo[i] + (o->cfg.u_hi[i] - o->cfg.u_lo[i]) * unit24(w0[i]);
      uint64_t span = (uint64_t)(o->cfg.k_max - o->cfg.k_min + 1);
      int k = o->cfg.k_min + (int)(((uint64_t)w1[0] * span) >> 32);
      if (net && (uint64_t)w1[2] < mix_thr) {
        /* learned draw from the network's Gaussian */
        uint32_t w3[4];
        double z[4], q[4];
        draw(o, it, (uint32_t)v, (uint32_t)j, 3, w3);
        kpo_box_muller(w3, z);
        const double *nn = net + 8 * (size_t)p;
        for (int i = 0; i < 4; ++i) {
          q[i] = nn[i] + exp(nn[4 + i]) * z[i];
          q[i] = q[i] < -1.0 ? -1.0 : (q[i] > 1.0 ? 1.0 : q[i]);
        }
        for (int i = 0; i < N; ++i)
          u[i] = o->cfg.u_lo[i] + (o->cfg.u_hi[i] - o->cfg.u_lo[i]) * (q[i] + 1.0) * 0.5;
        /* the duration keeps the uniform draw (the network's duration
         * output is trained but not drawn from) */
      }
      /* PropagateODE with the validity check after every step */
      memcpy(traj, o->x + (size_t)v * d, sizeof(double) * d);
      int valid = 1, fail = 0, last = 0;
      double m_valid = INFINITY;
      kpo_sample_work(o);
      for (int i = 1; i <= k; ++i) {
        kpo_step(&o->cfg, traj + (size_t)(i - 1) * d, u, o->cfg.dt,
                 traj + (size_t)i * d);
        kpo_step_work(o, traj + (size_t)(i - 1) * d, traj + (size_t)i * d);
        double m;
        int ok = kpo_step_valid(o, traj + (size_t)(i - 1) * d,
                                traj + (size_t)i * d, &m);
        if (m < m_valid) m_valid = m;
        last = i;
        if (!ok) {
          valid = 0;
          fail = i;
          break;
        }
      }
      const double *xe = traj + (size_t)last * d;
      /* map x' to R_i^k */
      int r, s;
      double m_bin;
      kpo_bin(o, xe, &r, &s, &m_bin);
      unsigned char f = 0;
      if (valid) {
        o->n_valid[r] += 1;
        ++n_valid_total;
        f |= 1;
        if (!visited0[s]) f |= 2;              /* may represent R_i^k */
        if ((uint64_t)w1[1] < o->thr[r]) f |= 4; /* P_accept(R_i) draw */
      } else {
        o->n_invalid[r] += 1;
      }
      memcpy(xs + (size_t)key * d, xe, sizeof(double) * d);
      memcpy(us + (size_t)key * N, u, sizeof(double) * N);
      ks[key] = k;
      rs[key] = r;
      ss[key] = s;
      fl[key] = f;
      if (rec && key < rec->capacity) {
        if (rec->node) rec->node[key] = v;
        if (rec->k) rec->k[key] = k;
        if (rec->uraw)
          for (int i = 0; i < 4; ++i) rec->uraw[4 * (size_t)key + i] = w0[i];
        if (rec->fail_step) rec->fail_step[key] = fail;
        if (rec->region) rec->region[key] = r;
        if (rec->sub) rec->sub[key] = s;
        if (rec->state) memcpy(rec->state + (size_t)key * d, xe, sizeof(double) * d);
        if (rec->m_valid) rec->m_valid[key] = m_valid;
        if (rec->m_bin) rec->m_bin[key] = m_bin;
        if (rec->m_goal) {
          double mg = INFINITY;
          if (valid) in_goal(o, xe, &mg);
          rec->m_goal[key] = mg;
        }
      }
    }
  }

  /* representatives of newly reached sub-regions: smallest key wins */
  unsigned char *claimed = (unsigned char *)xcalloc((size_t)o->n_sub, 1);
  for (int key = 0; key < S; ++key) {
    if ((fl[key] & 2) && !claimed[ss[key]]) {
      claimed[ss[key]] = 1;
      fl[key] |= 8;
    }
  }
  free(claimed);

  /* V_U: valid and (representative or P_accept draw) */
  int n_old = o->n, n_acc = 0;
  for (int key = 0; key < S; ++key) {
    unsigned char f = fl[key];
    if ((f & 1) && ((f & 8) || (f & 4))) fl[key] |= 16;
  }

  /* ----- Algorithm 4, new nodes: V_U -> T and V_E; goal test ----- */
  /* (appended before UpdateEstimates, reading R7) */
  for (int key = 0; key < S; ++key) {
    if (!(fl[key] & 16)) continue;
    int id = o->n++;
    ++n_acc;
    memcpy(o->x + (size_t)id * d, xs + (size_t)key * d, sizeof(double) * d);
    memcpy(o->u + (size_t)id * N, us + (size_t)key * N, sizeof(double) * N);
    o->parent[id] = ve[key / lambda];
    o->steps[id] = ks[key];
    o->region[id] = rs[key];
    o->sub[id] = ss[key];
    o->in_ve[id] = 1;
    o->visited[ss[key]] = 1;
    if (o->hv_feat && (fl[key] & 8) && o->hv_count < o->hv_cap) {
      const int h = o->hv_count++;
      memcpy(o->hv_feat + 32 * (size_t)h, feat + 32 * (size_t)(key / lambda), sizeof(double) * 32);
      for (int i = 0; i < 3; ++i)
        o->hv_target[4 * (size_t)h + i] =
            2.0 * (us[(size_t)key * N + i] - o->cfg.u_lo[i]) / (o->cfg.u_hi[i] - o->cfg.u_lo[i]) - 1.0;
      o->hv_target[4 * (size_t)h + 3] =
          o->cfg.k_max > o->cfg.k_min
              ? 2.0 * (double)(ks[key] - o->cfg.k_min) / (double)(o->cfg.k_max - o->cfg.k_min) - 1.0
              : 0.0;
    }
    if (in_goal(o, o->x + (size_t)id * d, NULL)) {
      fl[key] |= 32;
      if (o->goal_node < 0) o->goal_node = id;
    }
  }
  if (rec && rec->flags)
    for (int key = 0; key < S && key < rec->capacity; ++key) rec->flags[key] = fl[key];

  /* ---------------- Algorithm 3: UpdateEstimates ---------------- */
  refresh_region_sets(o);
  update_estimates(o);

  /* ----- Algorithm 4, old nodes: one draw per old node ----- */
  for (int v = 0; v < n_old; ++v) {
    uint32_t w[4];
    draw(o, it, (uint32_t)v, 0, 2, w);
    o->in_ve[v] = (uint64_t)w[0] < o->thr[o->region[v]] ? 1 : 0;
  }

  if (st) {
    st->iteration = (int32_t)it;
    st->n_ve = nve;
    st->lambda = lambda;
    st->n_samples = S;
    st->n_valid = n_valid_total;
    st->n_accepted = n_acc;
    st->n_nodes = o->n;
    st->goal_node = o->goal_node;
  }
  o->iteration += 1;
  if (o->goal_node >= 0) o->status = KPO_SOLVED;

  free(ve); free(xs); free(us); free(ks); free(rs); free(ss); free(fl);
  free(visited0); free(traj); free(feat); free(net);
  return o->status;
}

int32_t kpo_run(kpo *o, int32_t max_iters, int32_t *iters_done) {
  int done = 0;
  while (o->status == KPO_RUNNING && done < max_iters) {
    kpo_iterate(o, NULL, NULL);
    if (o->status == KPO_FULL) break;
    ++done;
  }
  if (iters_done) *iters_done = done;
  return o->status;
}

/* ------------------------------------------------------------------ */
/* state copy-out / copy-in                                             */
/* ------------------------------------------------------------------ */

void kpo_export(const kpo *o, double *state, int32_t *parent, double *ctrl,
                int32_t *steps, int32_t *region, int32_t *sub, uint8_t *in_ve,
                uint32_t *n_valid, uint32_t *n_invalid, uint32_t *cov,
                uint8_t *avail, uint64_t *thr, uint8_t *visited) {
  if (state) memcpy(state, o->x, sizeof(double) * (size_t)o->n * o->d);
  if (ctrl) memcpy(ctrl, o->u, sizeof(double) * (size_t)o->n * o->N);
  for (int v = 0; v < o->n; ++v) {
    if (parent) parent[v] = o->parent[v];
    if (steps) steps[v] = o->steps[v];
    if (region) region[v] = o->region[v];
    if (sub) sub[v] = o->sub[v];
    if (in_ve) in_ve[v] = o->in_ve[v];
  }
  for (int r = 0; r < o->R; ++r) {
    if (n_valid) n_valid[r] = (uint32_t)o->n_valid[r];
    if (n_invalid) n_invalid[r] = (uint32_t)o->n_invalid[r];
    if (cov) cov[r] = o->cov[r];
    if (avail) avail[r] = o->avail[r];
    if (thr) thr[r] = o->thr[r];
  }
  if (visited) memcpy(visited, o->visited, (size_t)o->n_sub);
}

int32_t kpo_import(kpo *o, int32_t n_nodes, int32_t iteration,
                   const float *state, const int32_t *parent,
                   const float *ctrl, const int32_t *steps,
                   const int32_t *region, const int32_t *sub,
                   const uint8_t *in_ve, const uint32_t *n_valid,
                   const uint32_t *n_invalid, const uint64_t *thr,
                   const uint8_t *visited) {
  if (n_nodes < 1 || n_nodes > o->cfg.t_e) return KPO_ERR;
  o->n = n_nodes;
  for (size_t i = 0; i < (size_t)n_nodes * o->d; ++i) o->x[i] = (double)state[i];
  for (size_t i = 0; i < (size_t)n_nodes * o->N; ++i) o->u[i] = (double)ctrl[i];
  for (int v = 0; v < n_nodes; ++v) {
    o->parent[v] = parent[v];
    o->steps[v] = steps[v];
    o->region[v] = region[v];
    o->sub[v] = sub[v];
    o->in_ve[v] = in_ve[v] ? 1 : 0;
  }
  for (int r = 0; r < o->R; ++r) {
    o->n_valid[r] = n_valid[r];
    o->n_invalid[r] = n_invalid[r];
    o->thr[r] = thr[r];
  }
  memcpy(o->visited, visited, (size_t)o->n_sub);
  refresh_region_sets(o);
  o->iteration = iteration;
  o->goal_node = -1;
  o->status = KPO_RUNNING;
  kpo_clear_work(o);
  return KPO_RUNNING;
}

void kpo_estimates(const kpo *o, double *score, double *p_accept,
                   double *score_sum) {
  if (score) memcpy(score, o->score, sizeof(double) * (size_t)o->R);
  if (p_accept) memcpy(p_accept, o->p_accept, sizeof(double) * (size_t)o->R);
  if (score_sum) *score_sum = o->score_sum;
}

int32_t kpo_path(const kpo *o, int32_t *nodes, int32_t cap) {
  if (o->goal_node < 0) return 0;
  int len = 0;
  for (int v = o->goal_node; v >= 0; v = o->parent[v]) ++len;
  int i = len - 1;
  for (int v = o->goal_node; v >= 0; v = o->parent[v], --i)
    if (i < cap) nodes[i] = v;
  return len;
}
