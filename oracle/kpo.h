/*
 * kpo.h -- FP64 CPU oracle for the Kino-PAX tree expansion.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, deliberately unoptimised
 * restatement of the Kino-PAX method (Perrault, Ho, Lahijanian, "Kino-PAX:
 * Highly Parallel Kinodynamic Sampling-based Planner", RA-L 2025) in double
 * precision.  It exists to check the CUDA implementation.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never calls it.  It shares no code, header or
 * constant table with the CUDA implementation.
 *
 * Paper anchors used below:
 *   Sec. II, Eq. 1-2 and Problem 1   dynamics, valid set, goal set
 *   Sec. III, Algorithm 1            main loop
 *   Sec. III, Algorithm 2            Propagate
 *   Sec. III, Algorithm 3, Eq. 3-5   UpdateEstimates (FreeVol, Score, P_accept)
 *   Sec. III, Algorithm 4            UpdateNodeSets
 *   Sec. IV-A, Eq. 6                 adaptive branching factor lambda
 *   Sec. V, Lemma 1                  P_accept >= eps
 */
#ifndef KPO_H
#define KPO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { KPO_DI = 0, KPO_DUBINS = 1, KPO_QUAD = 2 };

enum {
  KPO_RUNNING = 0,   /* loop may continue                                   */
  KPO_SOLVED = 1,    /* a goal node was appended (Algorithm 4, goal test)   */
  KPO_FULL = 2,      /* Eq. 6 gave lambda = 0: the tree cannot grow          */
  KPO_ERR = -1
};

/* Planner configuration.  All real values arrive as float32 inputs and are
 * promoted here, so the oracle and the device code start from identical
 * numbers and differ only in the precision of what they compute. */
typedef struct {
  int32_t system;               /* KPO_DI / KPO_DUBINS / KPO_QUAD          */
  double dt;                    /* integrator step                          */
  int32_t k_min, k_max;         /* duration = k * dt, k uniform in [min,max] */
  double x_lo[12], x_hi[12];    /* state box of the valid set (+-inf = free) */
  double u_lo[4], u_hi[4];      /* control box U                            */
  double phys[16];              /* quadrotor: m g l c Ixx Iyy Izz           */
  double ws_lo[3], ws_hi[3];    /* workspace W (position)                   */
  int32_t grid[3];              /* region cells per position axis           */
  int32_t speed_bins;           /* >= 1 speed bins in the region index      */
  double speed_hi;              /* speeds binned over [0, speed_hi]         */
  int32_t sub[3];               /* sub-region cells per region and axis     */
  int32_t fso;                  /* 1: regions are the leaves of a kd-tree
                                   split on obstacle faces (a free-space-
                                   obeying decomposition, Sec. IV-B); the
                                   position grid, speed bins and state grid
                                   are then unused                        */
  int32_t state_grid[12];       /* cells over state dimension d >= 3 in the
                                   region index (0 or 1: not decomposed);
                                   an unbounded dimension (an angle) is
                                   wrapped to [-pi, pi) first            */
  int32_t t_e;                  /* node cap (Sec. IV-A)                      */
  int32_t lambda_max;           /* Eq. 6                                     */
  double delta;                 /* Eq. 3                                     */
  double eps;                   /* Eq. 5                                     */
  uint64_t seed;                /* Philox key                                */
  double goal_c[3], goal_r;     /* goal set: closed ball on position        */
} kpo_config;

/* Per-sample record of one Propagate call (Algorithm 2), indexed by sample
 * key = (position in V_E) * lambda + j.  Any pointer may be NULL. */
typedef struct {
  int32_t capacity;
  int32_t *node;      /* expanded node id                                   */
  int32_t *k;         /* integration steps drawn                            */
  uint32_t *uraw;     /* [4*cap] raw Philox words of the control draw       */
  uint8_t *flags;     /* bit0 valid, bit1 contender, bit2 Bernoulli pass,
                         bit3 claim winner, bit4 accepted, bit5 goal         */
  int32_t *fail_step; /* 0 when valid, else first invalid step (1..k)       */
  int32_t *region;    /* region index                                       */
  int32_t *sub;       /* global sub-region index                            */
  double *state;      /* [d*cap] state at the end (or first invalid step)   */
  double *m_valid;    /* distance of the validity verdict from its boundary  */
  double *m_bin;      /* distance of the binned state from a cell face       */
  double *m_goal;     /* distance of the final position from the goal sphere */
} kpo_records;

typedef struct {
  int32_t iteration, n_ve, lambda, n_samples, n_valid, n_accepted, n_nodes,
      goal_node;
} kpo_iter_stats;

/* Algorithmic work of Propagate (Algorithm 2) since the last reset or
 * import, counted during replay (the counting rule is in work.c). */
typedef struct {
  uint64_t samples;   /* samples drawn                                       */
  uint64_t steps;     /* integrator steps run (to the first invalid one)     */
  uint64_t hulls;     /* steps whose end state is in the state box: their
                         hull is tested against the obstacles              */
  uint64_t box_scan;  /* hull-vs-box tests of a scan in box order that stops
                         at the first box met                              */
  uint64_t box_grid;  /* the same over the boxes of the grid cells the hull
                         overlaps (kpo_set_work_grid)                      */
  uint64_t ops;       /* lane operations: samples, steps, hulls and the
                         grid's box tests at their costs                   */
  /* box_scan, box_grid and their operations are counted only after
   * kpo_set_work_grid */
} kpo_work;

typedef struct kpo kpo;

kpo *kpo_create(const kpo_config *cfg, const float *boxes, int32_t n_boxes);
void kpo_destroy(kpo *o);
int32_t kpo_state_dim(const kpo *o);
int32_t kpo_control_dim(const kpo *o);
int32_t kpo_num_regions(const kpo *o);
int32_t kpo_num_subregions(const kpo *o);

/* Algorithm 1, initialisation.  Returns KPO_ERR when x_init is not valid. */
int32_t kpo_reset(kpo *o, const float *x_init);
/* One pass of the Algorithm 1 loop body.  Returns the planner status. */
int32_t kpo_iterate(kpo *o, kpo_records *rec, kpo_iter_stats *st);
/* Iterate until solved, full or max_iters passes.  Returns the status. */
int32_t kpo_run(kpo *o, int32_t max_iters, int32_t *iters_done);
int32_t kpo_status(const kpo *o);
int32_t kpo_goal_node(const kpo *o);
int32_t kpo_num_nodes(const kpo *o);
int32_t kpo_iteration(const kpo *o);

/* Tree / region state copy-out and copy-in (n_nodes entries; row-major
 * state [n][d] and control [n][N]).  Region arrays have kpo_num_regions
 * entries, visited has kpo_num_subregions entries. */
void kpo_export(const kpo *o, double *state, int32_t *parent, double *ctrl,
                int32_t *steps, int32_t *region, int32_t *sub, uint8_t *in_ve,
                uint32_t *n_valid, uint32_t *n_invalid, uint32_t *cov,
                uint8_t *avail, uint64_t *thr, uint8_t *visited);
int32_t kpo_import(kpo *o, int32_t n_nodes, int32_t iteration,
                   const float *state, const int32_t *parent,
                   const float *ctrl, const int32_t *steps,
                   const int32_t *region, const int32_t *sub,
                   const uint8_t *in_ve, const uint32_t *n_valid,
                   const uint32_t *n_invalid, const uint64_t *thr,
                   const uint8_t *visited);

/* Region estimates of the last UpdateEstimates call (Eq. 3-5). */
void kpo_estimates(const kpo *o, double *score, double *p_accept,
                   double *score_sum);

/* Root-to-goal chain: writes up to cap node ids (root first); returns the
 * chain length, 0 when there is no goal node. */
int32_t kpo_path(const kpo *o, int32_t *nodes, int32_t cap);

/* ---- learned proposal (an addition to the paper's uniform draw) ----
 * Node features (32 values, the last 8 zero) of node v under the current
 * region tables:
 *   [0..5]  state, each bounded entry mapped to [-1, 1]; an unbounded
 *           entry wrapped to [-pi, pi) and divided by pi
 *   [6..8]  goal centre minus position
 *   [9]     Cov / n'          [10] FreeVol / vol = (delta+nv)/(delta+nv+ni)
 *   [11]    log(1 + nv)       [12] log(1 + ni)
 *   [13]    P_accept = thr / 2^32
 *   [14..19] P_accept of the -x, +x, -y, +y, -z, +z neighbour regions in
 *           the position grid (0 outside the grid)
 * Targets: (u_i - lo_i) / (hi_i - lo_i) * 2 - 1 for the 3 controls and
 * (k - k_min) / (k_max - k_min) * 2 - 1 for the duration.
 * Learned draw of a sample (selector word < mix * 2^32): normals z_0..z_3
 * by Box-Muller from Philox purpose 3 words, q = clamp(mean + exp(log_std)
 * z, -1, 1), u_i = lo_i + (hi_i - lo_i)(q_i + 1)/2 for the controls; the
 * duration k stays the uniform draw (purpose 1, word 0), so a learned
 * sample costs the integrator steps a uniform one does.  Only 6D systems. */
int32_t kpo_mlp_num_params(void);
void kpo_mlp_forward(const double *p, const double *x, int32_t M, double *out);
double kpo_mlp_loss_grad(const double *p, const double *x, const double *t,
                         int32_t M, double *grad);
void kpo_adam(double *p, const double *g, double *m, double *v, int32_t n,
              double lr, double beta1, double beta2, double eps, int32_t t);
void kpo_features(const kpo *o, int32_t v, double *feat);
/* Enables the learned draw with the given parameter vector (NULL: off). */
int32_t kpo_set_mlp(kpo *o, const float *params, double mix);
/* Harvest: every representative of a newly reached sub-region appends its
 * parent's features and its own target; returns pairs written so far. */
int32_t kpo_set_harvest(kpo *o, double *feat, double *target, int32_t capacity);
int32_t kpo_harvest_count(const kpo *o);
void kpo_box_muller(const uint32_t w[4], double z[4]);

/* Work counting (work.c).  The grid of the pruned box count: g[a] cells
 * along position axis a over W (default 1 x 1 x 1: every box in one cell). */
void kpo_set_work_grid(kpo *o, const int32_t g[3]);
void kpo_get_work(const kpo *o, kpo_work *out);
/* The work grid's cell clearances in sixteenths of a cell (cells in index
 * order, x fastest); returns the cell count (0 before kpo_set_work_grid). */
int32_t kpo_work_clearance(const kpo *o, int32_t *out);
void kpo_clear_work(kpo *o);
/* Lane operations per unit: sample, integrator step, hull, box test. */
uint64_t kpo_work_ops_sample(const kpo *o);
uint64_t kpo_work_ops_step(const kpo *o);
uint64_t kpo_work_ops_hull(void);
uint64_t kpo_work_ops_box(void);

/* ---- building blocks, exported for the oracle's own pin tests ---- */
void kpo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* n blocks: counters ctr [n][4] under one key, words out [n][4]. */
void kpo_philox4x32_10_n(const uint32_t *ctr, const uint32_t key[2], uint32_t *out,
                         int64_t n);
/* Volume of every region as Eq. 3 takes it: the grid cell's, or the
 * kd-tree leaf's under the free-space-obeying decomposition. */
void kpo_region_volumes(const kpo *o, double *vol);
/* Advances x by one integrator step under control u (Eq. 1-2). */
void kpo_step(const kpo_config *cfg, const double *x, const double *u,
              double h, double *x_out);
/* Integrates k steps of cfg->dt, writing every state (k+1 rows) to traj. */
void kpo_propagate(const kpo_config *cfg, const double *x0, const double *u,
                   int32_t k, double *traj);
/* One step of the validity check: state bounds of x1 and the axis-aligned
 * box of positions {p(x0), p(x1)} against every obstacle.  Returns 1 when
 * valid; *margin receives the distance of the verdict from its boundary. */
int32_t kpo_step_valid(const kpo *o, const double *x0, const double *x1,
                       double *margin);
/* Region and global sub-region index of a state. */
void kpo_bin(const kpo *o, const double *x, int32_t *region, int32_t *sub,
             double *margin);
/* Eq. 3-5 on explicit arrays (n regions). */
void kpo_eq345(int32_t n, const uint32_t *n_valid, const uint32_t *n_invalid,
               const uint32_t *cov, const uint8_t *avail, double vol,
               double delta, double eps, double *score, double *p_accept,
               uint64_t *thr, double *score_sum);
/* The same with a volume per region (vol_r[i]; the free-space-obeying
 * decomposition, whose regions differ in size). */
void kpo_eq345_vol(int32_t n, const uint32_t *n_valid, const uint32_t *n_invalid,
                   const uint32_t *cov, const uint8_t *avail, const double *vol_r,
                   double delta, double eps, double *score, double *p_accept,
                   uint64_t *thr, double *score_sum);
/* Regions of the free-space-obeying decomposition (capacity). */
#define KPO_FSO_MAX_LEAVES 16384
/* Leaf boxes of that decomposition in region order (lo/hi: [cap][3]);
 * returns the number of leaves (0 when the regions are a grid). */
int32_t kpo_fso_leaves(const kpo *o, double *lo, double *hi, int32_t cap);
/* Eq. 6. */
int32_t kpo_lambda(int32_t t_e, int32_t n_tree, int32_t n_ve,
                   int32_t lambda_max);
/* Dense re-validation of one edge: 'sub' sub-steps per integrator step,
 * point-in-closed-box and state bounds at every sub-step.  Returns the
 * largest violation depth found (<= 0 means valid everywhere). */
double kpo_dense_check(const kpo *o, const double *x0, const double *u,
                       int32_t k, int32_t sub, double *x_end);

#ifdef __cplusplus
}
#endif
#endif
