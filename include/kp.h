/*
 * kp.h -- C ABI of the GB300 Kino-PAX planner.
 *
 * Kino-PAX (Perrault, Ho, Lahijanian, "Kino-PAX: Highly Parallel
 * Kinodynamic Sampling-based Planner", RA-L 2025) grows a tree of
 * trajectory segments in three data-parallel subroutines per iteration:
 * Propagate (Algorithm 2), UpdateEstimates (Algorithm 3, Eq. 3-5) and
 * UpdateNodeSets (Algorithm 4), with the branching factor of Eq. 6.  This
 * library runs that loop on one GPU, entirely on the device, and answers
 * the planning query of Problem 1 (Sec. II): given x_init and a goal set,
 * return a control trajectory whose induced state trajectory is valid and
 * reaches the goal.
 *
 * Conventions for every entry point:
 *  - Memory.  The library allocates no device memory.  All device state
 *    lives in one caller-owned arena of kp_required_bytes() bytes (for
 *    example a uint8 CUDA tensor); it must stay alive and untouched by the
 *    caller until kp_destroy().  Host inputs are copied during the call and
 *    may be freed when it returns.  Host outputs go to caller buffers.
 *  - Streams.  All device work is enqueued on the stream given to
 *    kp_create (NULL = the legacy default stream).  Calls that return host
 *    results synchronise that stream before returning.
 *  - Errors.  Every call returns a kp_status; nothing else crosses the ABI.
 *    KP_NO_SOLUTION is a normal outcome.  After KP_ERR_CUDA or
 *    KP_ERR_TIMEOUT the context is poisoned: every later call except
 *    kp_last_error and kp_destroy returns KP_ERR_STATE.
 *  - Threads.  A context belongs to one host thread at a time.
 *  - Units.  States, controls and boxes are in the units of kp_system and
 *    kp_workspace; all real inputs are float32.
 */
#ifndef KP_H
#define KP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KP_OK = 0,            /* call succeeded (kp_plan: a solution was found)   */
  KP_NO_SOLUTION = 1,   /* budget spent or tree full (Eq. 6 gave lambda 0)  */
  KP_ERR_ARG = -1,      /* invalid argument; nothing was changed            */
  KP_ERR_OOM = -2,      /* arena smaller than kp_required_bytes()           */
  KP_ERR_CUDA = -3,     /* a CUDA call failed; context poisoned             */
  KP_ERR_TIMEOUT = -4,  /* a bounded device wait expired; context poisoned  */
  KP_ERR_STATE = -5     /* call not allowed in the context's current state  */
} kp_status;

typedef enum {
  KP_DOUBLE_INTEGRATOR_6D = 0, /* x = (p, v), u = a; explicit Euler         */
  KP_DUBINS_AIRPLANE_6D = 1,   /* x = (x,y,z,yaw,pitch,speed),
                                  u = (yaw rate, pitch rate, accel); RK4    */
  KP_QUADROTOR_12D = 2         /* x = (p, roll,pitch,yaw, v_world,
                                  omega_body), u = 4 rotor thrusts; RK4     */
} kp_system_id;

/* Dynamics (Sec. II, Eq. 1-2) and the state/control boxes of the valid set.
 * A sample's duration is k integrator steps of dt, k uniform in
 * [k_min, k_max] (Algorithm 2 draws dt in (0, T_prop]).  Entries of
 * x_lo/x_hi beyond the state dimension are ignored; +-inf leaves a state
 * unbounded.  phys: quadrotor m, g, l, c, Ixx, Iyy, Izz (others unused). */
typedef struct {
  int32_t id;                 /* kp_system_id                              */
  float dt;                   /* integrator step, > 0                      */
  int32_t k_min, k_max;       /* 1 <= k_min <= k_max <= 255                 */
  float x_lo[12], x_hi[12];
  float u_lo[4], u_hi[4];
  float phys[16];
} kp_system;

/* Workspace W (Sec. II) and the decomposition R (Sec. III): a uniform grid
 * of grid[0]*grid[1]*grid[2] position cells times speed_bins speed bins over
 * [0, speed_hi] times state_grid[d] cells over each further state dimension
 * d >= 3 with state_grid[d] > 1 (a grid over the whole state space, as in
 * the paper's experiments, Sec. VI: a bounded dimension binned over
 * [x_lo, x_hi], an unbounded one, an angle, wrapped to [-pi, pi) first);
 * every region holds sub[0]*sub[1]*sub[2] sub-regions over position.
 * Region index: position fastest, then the speed bin, then the further
 * dimensions in increasing d.
 * fso = 1 replaces the grid by a free-space-obeying decomposition (Sec.
 * IV-B): the regions are the leaves of a kd-tree over W whose planes are
 * obstacle faces.  A cell is split while a face of a box meeting its
 * interior lies strictly inside it: on the axis with the most distinct such
 * coordinates (the lowest axis on a tie), at the lower median of them; so
 * every leaf lies inside an obstacle or meets none.  Leaves are numbered
 * depth first, the side below each plane first (a point on a plane goes
 * above it); each holds a sub[0]*sub[1]*sub[2] sub-grid over its own box,
 * and Eq. 3 takes its own volume.  grid, speed_bins and state_grid are then
 * ignored.  The tree is rebuilt by kp_set_obstacles; at most 16,384 leaves
 * and depth 64 (KP_ERR_ARG beyond).  Not available in kp_plan_static or
 * the server. */
typedef struct {
  float lo[3], hi[3];
  int32_t grid[3];            /* 1 .. 4096, and grid[a] * sub[a] <= 2^22    */
  int32_t speed_bins;         /* >= 1 (1: no speed bins)                    */
  float speed_hi;
  int32_t sub[3];
  int32_t state_grid[12];     /* 0 or 1: dimension not decomposed; entries
                                 0..2 and >= the state dimension ignored   */
  int32_t fso;                /* 1: free-space-obeying kd-tree regions      */
} kp_workspace;

/* Obstacle set O (Sec. II): closed axis-aligned boxes, host pointer to
 * n_boxes rows of {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z} with lo <= hi on
 * every axis (KP_ERR_ARG otherwise); copied. */
typedef struct {
  const float *boxes;
  int32_t n_boxes;            /* 0 .. KP_MAX_BOXES                          */
} kp_obstacles;

#define KP_MAX_BOXES 4096

/* Goal set X_goal: the closed ball of positions |p - center| <= radius. */
typedef struct {
  float center[3];
  float radius;
} kp_goal;

/* Planner constants: t_e node cap (Sec. IV-A), lambda_max (Eq. 6), delta
 * (Eq. 3), eps (Eq. 5, Lemma 1), 64-bit seed of the Philox stream. */
typedef struct {
  int32_t t_e;                /* 2 .. 2^28                                  */
  int32_t lambda_max;         /* 1 .. 1024                                   */
  double delta;               /* > 0                                         */
  double eps;                 /* (0, 1)                                      */
  uint64_t seed;
} kp_params;

/* Loop budget for kp_plan: stop after max_iters passes or max_ms of device
 * time (<= 0: no time limit), whichever comes first. */
typedef struct {
  int32_t max_iters;
  double max_ms;
} kp_budget;

/* Trajectory out: root-to-goal edges.  Caller buffers of 'capacity' rows:
 * states [capacity][12] (state at the end of each edge), ctrls
 * [capacity][4] (constant control of the edge), steps [capacity]
 * (integrator steps of the edge).  n_edges is set on return. */
typedef struct {
  int32_t capacity;
  int32_t n_edges;
  float *states;
  float *ctrls;
  int32_t *steps;
} kp_traj;

/* One loop pass (Algorithm 1 body). */
typedef struct {
  int32_t iteration;   /* pass index, from 0 after kp_reset                */
  int32_t n_ve;        /* |V_E| expanded in this pass                      */
  int32_t lambda;      /* branching factor of this pass (Eq. 6)            */
  int32_t n_samples;   /* |V_E| * lambda                                   */
  int32_t n_valid;     /* samples whose segment was valid                  */
  int32_t n_accepted;  /* |V_U| appended to the tree                       */
  int32_t n_nodes;     /* |T| after the pass                               */
  int32_t goal_node;   /* smallest new goal node id, -1 if none            */
  int32_t phase_ns[12]; /* device time of the pass's phases (ns) as seen by
                           one block, each phase's work then its barrier
                           wait: [0] Propagate, [1] wait, [2] accept flags
                           with Score (Eq. 3-4) alongside, [3] node
                           features and the network (learned form or
                           harvest, else 0), [4] wait, [5] 0, [6] wait
                           after [3], [7] 0, [8] P_accept (Eq. 5), the new
                           nodes appended to T and the node-set draws, [9]
                           wait, [10] V_E list and Eq. 6, [11] the previous
                           pass's final wait */
} kp_iter_stats;

/* Context status snapshot.  The work counters cover every pass since the
 * last kp_reset / kp_plan. */
typedef struct {
  int32_t n_nodes, n_ve, iteration, goal_node;
  int32_t state;       /* 0 running, 1 solved, 2 tree full, -1 error      */
  int32_t n_regions, n_subregions, state_dim, control_dim;
  int32_t n_boxes;     /* obstacle slots in use (padded to a multiple of 8) */
  int32_t grid_blocks; /* blocks of the persistent loop launch             */
  int64_t n_samples;   /* samples propagated and checked                   */
  int64_t n_steps;     /* integrator steps run (each one checked)          */
  int64_t n_hull_checks; /* step hulls tested against the obstacle set     */
  int64_t n_box_tests;   /* hull-vs-box tests made (after the broad phase)   */
  int32_t bp_cells;      /* broad-phase grid cells in all (1: every box)     */
  int32_t bp_grid[3];    /* broad-phase grid cells along x, y, z             */
  int64_t n_key_batches; /* key batches warps took from the grid-wide counter
                            after their first batch (the refill path)        */
  int64_t n_lane_refills; /* keys a lane started after finishing an earlier
                             key of the same pass                           */
} kp_info;

/* Host-side copy of the tree and decomposition (tests, checkpoints).
 * State rows are node-major: state[v * 12 + i], ctrl[v * 4 + i].  Arrays
 * must hold 'capacity' nodes / n_regions regions / n_subregions entries. */
typedef struct {
  int32_t capacity;
  int32_t n_nodes;      /* out (export) / in (import)                      */
  int32_t iteration;    /* out / in: next pass index                       */
  float *state;         /* [capacity][12]                                   */
  int32_t *parent;      /* -1 for the root                                  */
  float *ctrl;          /* [capacity][4]                                    */
  int32_t *steps;
  int32_t *region;
  int32_t *sub;         /* global sub-region index                          */
  uint8_t *in_ve;       /* 1: V_E, 0: V_O                                    */
  uint32_t *n_valid;    /* [n_regions] cumulative counters (Algorithm 2)    */
  uint32_t *n_invalid;
  uint32_t *cov;        /* [n_regions] visited sub-regions (export only)    */
  uint8_t *avail;       /* [n_regions] R_avail membership (export only)     */
  uint64_t *thr;        /* [n_regions] accept threshold: draw w < thr       */
  uint8_t *visited;     /* [n_subregions]                                    */
} kp_tree_view;

/* Per-sample record of the most recent pass (parity checks).  DEVICE
 * pointers, each with room for 'capacity' samples (uraw: 4 per sample,
 * state: 12 per sample, sample-major).  Sample key = position of the
 * expanded node in V_E (ascending node id) * lambda + j.  flags: bit0
 * valid, bit1 reached an unvisited sub-region, bit2 accept draw passed,
 * bit3 representative of its sub-region, bit4 appended, bit5 goal. */
typedef struct {
  int32_t capacity;
  int32_t *node;
  int32_t *k;
  uint32_t *uraw;
  uint8_t *flags;
  int32_t *fail_step;   /* 0 valid, else first invalid integrator step     */
  int32_t *region;
  int32_t *sub;
  float *state;         /* state at the end or at the first invalid step   */
} kp_sample_log;

typedef struct kp_ctx kp_ctx;

/* Bytes of device arena a context needs (room for KP_MAX_BOXES obstacles
 * is always reserved).  Returns 0 for invalid inputs. */
size_t kp_required_bytes(const kp_system *sys, const kp_workspace *ws,
                         int32_t n_boxes, const kp_params *prm);

/* Creates a context on the current CUDA device over the caller's arena
 * (256-byte aligned device pointer).  Copies the obstacles.  The tree is
 * empty until kp_reset.  Errors: KP_ERR_ARG (bad inputs, misaligned
 * arena), KP_ERR_OOM (arena too small), KP_ERR_CUDA. */
kp_status kp_create(const kp_system *sys, const kp_workspace *ws,
                    const kp_obstacles *obs, const kp_params *prm,
                    void *dev_arena, size_t arena_bytes, void *cuda_stream,
                    kp_ctx **out);

/* Replaces the obstacle set (up to KP_MAX_BOXES closed boxes, host rows
 * lo xyz, hi xyz) and resets the tree to empty.  On the host it builds the
 * broad-phase grid of the step-hull test (Algorithm 2 validity check):
 * 4096 cells shaped 16x16x16, 64x64x1 or 32x32x4 (or a rotation), the
 * shape with the smallest sum of squared per-cell box counts, coarser when
 * the box lists do not fit; under the kd-tree decomposition (Sec. IV-B)
 * it also rebuilds the tree.  Errors: KP_ERR_ARG (count above capacity,
 * NaN or lo > hi in a box, kd-tree above its leaf or depth limit; the
 * context keeps its previous obstacles), KP_ERR_CUDA. */
kp_status kp_set_obstacles(kp_ctx *ctx, const kp_obstacles *obs);

/* Algorithm 1, initialisation: tree = {x_init}, V_E = {x_init}, counters zero,
 * P_accept = 1 everywhere; the Philox key becomes 'seed'.  x_init is a
 * host array of the state dimension.  KP_ERR_ARG if x_init is not valid
 * (Problem 1 requires x_init in X_valid).  If x_init already lies in the
 * goal set the query is solved with zero edges. */
kp_status kp_reset(kp_ctx *ctx, const float *x_init, const kp_goal *goal,
                   uint64_t seed);

/* Runs up to n_iters passes of the Algorithm 1 loop body on the device
 * (fewer when a goal node is appended or Eq. 6 gives lambda = 0), in one
 * launch with no host synchronisation between passes.  Writes one record
 * per pass run to 'out' (nullable, room for n_iters).  Returns KP_OK. */
kp_status kp_expand_step(kp_ctx *ctx, int32_t n_iters, kp_iter_stats *out,
                         int32_t *n_run);

/* Problem 1 end to end: kp_reset, the loop until a goal node is appended or
 * the budget or the tree is exhausted, then the root-to-goal edge list.
 * Returns KP_OK with traj filled, KP_NO_SOLUTION, or KP_ERR_ARG when
 * traj->capacity is too small (traj->n_edges then holds the size needed). */
kp_status kp_plan(kp_ctx *ctx, const float *x_init, const kp_goal *goal,
                  const kp_budget *budget, kp_traj *traj);

/* kp_plan in two halves.  kp_plan_async validates its arguments and
 * enqueues the whole query (reset, loop, trajectory extraction: one launch
 * of the persistent loop kernel) on the context's stream without waiting;
 * traj_capacity is the number of
 * trajectory rows kp_plan_result will read back.  kp_plan_result waits
 * for that work and fills traj as kp_plan does (KP_ERR_STATE when no
 * kp_plan_async is pending). */
kp_status kp_plan_async(kp_ctx *ctx, const float *x_init, const kp_goal *goal,
                        const kp_budget *budget, int32_t traj_capacity);
kp_status kp_plan_result(kp_ctx *ctx, kp_traj *traj);

/* Device duration, in milliseconds, of the most recent launch of the
 * persistent loop kernel (for kp_plan and kp_plan_async that launch also
 * holds the reset and the trajectory extraction), from CUDA events the
 * library records on the context's stream around it (waits for it to
 * finish). */
kp_status kp_last_launch_ms(kp_ctx *ctx, float *ms);

/* Status snapshot (synchronises the stream). */
kp_status kp_get_info(kp_ctx *ctx, kp_info *out);

/* Copies the tree and decomposition to host buffers. */
kp_status kp_export_tree(kp_ctx *ctx, kp_tree_view *host_out);

/* Loads a tree and decomposition from host buffers (n_nodes, iteration,
 * state, parent, ctrl, steps, region, sub, in_ve, n_valid, n_invalid, thr,
 * visited are read; cov and R_avail are recomputed from visited and the
 * node regions).  The loop continues from there. */
kp_status kp_import_tree(kp_ctx *ctx, const kp_tree_view *host_in);

/* Enables (log != NULL) or disables per-sample records of each pass.  A
 * pass with more samples than log->capacity records only the first
 * capacity samples. */
/* Adaptive node cap (Sec. IV-A, Remark 1): moves the context to a larger
 * caller-owned arena (kp_required_bytes with the new t_e; 256-byte
 * aligned) and raises t_e, keeping the tree, the region and sub-region
 * tables, the loop state and the staged obstacles (a device-to-device copy
 * at HBM bandwidth; the tree's SoA rows move to the new stride).  The old
 * arena is no longer used when the call returns.  t_e may not shrink.
 * Typical use: kp_plan ends with KP_NO_SOLUTION and kp_get_info reports a
 * full tree (state 2); grow by a constant factor and call kp_resume. */
kp_status kp_grow(kp_ctx *ctx, void *dev_arena, size_t arena_bytes, int32_t t_e);
/* Continues the loop (Algorithm 1) from the context's current tree until a
 * goal node is appended, the tree is full (Eq. 6 gives lambda = 0) or the
 * budget is spent, then fills traj as kp_plan does.  KP_ERR_STATE without
 * a tree (kp_reset / kp_plan first). */
kp_status kp_resume(kp_ctx *ctx, const kp_budget *budget, kp_traj *traj);
kp_status kp_set_sample_log(kp_ctx *ctx, const kp_sample_log *log);

/* Upper bound, in nanoseconds, of every device-side wait (grid barrier,
 * bulk-copy completion).  On expiry the launch stops, the call returns
 * KP_ERR_TIMEOUT and the context is poisoned.  Default 2e9 (2 s). */
kp_status kp_set_wait_limit(kp_ctx *ctx, uint64_t ns);

/* Launch shape of the persistent loop (no counterpart in the paper: a
 * property of this implementation).  Caps the loop launch at max_blocks
 * blocks (0 restores the resident maximum of the device).  Results do not
 * depend on the launch shape: every sample's draw, integration, check and
 * binning follow from its key alone, claims are decided by the smallest
 * key and appends are made in key order.  With few blocks every lane runs
 * many keys of a pass, so the key-batch counter and lane refills (kp_info
 * n_key_batches, n_lane_refills) are exercised on small problems; tests use
 * this.  Errors: KP_ERR_ARG (negative, or a launch that cannot be resident;
 * the previous shape is kept). */
kp_status kp_set_grid_limit(kp_ctx *ctx, int32_t max_blocks);

/* Trajectory extraction (no counterpart in the paper: a testing aid).  A
 * query's root-to-goal chain is written by one block after the passes:
 * one thread walks the parent links from the goal node once and keeps the
 * node ids in the shared memory the passes no longer use, then the block
 * writes the rows; a chain longer than that room is written by the one
 * thread on a second walk.  This caps the ids kept at max_ids (0 restores
 * the room), so that tests can send short chains down the second path; the
 * rows are the same either way.  KP_ERR_ARG if negative. */
kp_status kp_set_extract_ids(kp_ctx *ctx, int32_t max_ids);

/* Bounds-checked build (no counterpart in the paper: a testing aid).  The
 * library compiled with KP_CHECK defined (paper_2409_06807_gb300/build.py,
 * check=True) checks every array index the loop kernel derives (node ids,
 * sample keys, regions, sub-regions, V_E positions, accepted-sample slots,
 * block slots, broad-phase cells, box lists and box ids) against its
 * array: an index out of range records the site, is replaced by 0 so that
 * no access leaves its array (nothing traps), and the launch stops at its
 * next barrier; the call then returns KP_ERR_CUDA with the site in
 * kp_last_error and the context is poisoned.  kp_bounds_checked returns 1
 * in that build, 0 otherwise.  kp_selftest_bounds looks up an index one
 * past the tree through the checked path and returns what the launch
 * reports (KP_ERR_CUDA, site 97, in the checked build); in the normal build
 * it launches nothing and returns KP_ERR_STATE. */
int32_t kp_bounds_checked(void);
kp_status kp_selftest_bounds(kp_ctx *ctx);

/* Test hook for the bounded-wait path: one block waits on a device flag
 * that nothing ever sets, for at most the context's wait limit, then
 * reports.  Returns KP_ERR_TIMEOUT (and poisons the context) when the wait
 * expired as designed. */
kp_status kp_selftest_wait_timeout(kp_ctx *ctx);

/* kp_plan for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment form of kp_plan.  Some callers may
 * not call cudaMalloc (or hand this library an arena) at all: a host
 * application that owns every byte of device memory through its own pool,
 * a plugin loaded into such a process, or a real-time control loop that
 * must not pay the implicit device synchronisation and unbounded latency of
 * an allocation.  This entry point runs the same query as kp_plan (same
 * kernels, same results) with no context, no arena and no allocation of any
 * kind: its device scratch is one static array of KP_STATIC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits.  The
 * caller still passes all inputs (host structs and arrays, as for
 * kp_create/kp_plan) and the output trajectory buffers.
 *  - Size limit: problems whose arena (kp_required_bytes) exceeds
 *    KP_STATIC_SCRATCH_BYTES return KP_ERR_OOM without touching the device.
 *  - Set-up: the first call on a device looks up the scratch's device
 *    address (once per device, with that device current).
 *  - Sharing: all calls on a device share the scratch, which keeps the last
 *    call's contents; every call clears what must start at zero.  Calls
 *    whose GPU work overlaps (other streams or host threads) race on the
 *    scratch and must be serialised by the caller.
 *  - Obstacles: the call builds the broad-phase grid of the step-hull test
 *    on the device in the scratch (the finest cube of 16^3, 8^3, 4^3, 2^3
 *    or 1 cell whose box lists fit), with the cells' clearances; verdicts
 *    equal testing every box, as in kp_plan.
 *  - Work is enqueued on cuda_stream (NULL = legacy default stream) and the
 *    call blocks until it is done (it synchronises that stream and copies
 *    to pageable host memory).  Returns as kp_plan (a replay mismatch of the
 *    sample log cannot occur here: the log is off); error codes carry no
 *    message; KP_ERR_ARG also when no block of the loop kernel can be
 *    resident with this problem's shared memory. */
#define KP_STATIC_SCRATCH_BYTES (16u << 20)
kp_status kp_plan_static(const kp_system *sys, const kp_workspace *ws,
                         const kp_obstacles *obs, const kp_params *prm,
                         const float *x_init, const kp_goal *goal,
                         const kp_budget *budget, kp_traj *traj,
                         void *cuda_stream);

/* ---- learned control proposal -------------------------------------------
 * Not in the paper: an addition on top of Algorithm 2's uniform control
 * draw.  A network maps 24 node features (zero padded to KP_MLP_INPUTS) to
 * a Gaussian over 4 normalised quantities (3 controls, the duration): two
 * ReLU layers of 256 units, outputs mean = tanh(o[0..3]) and log_std =
 * clamp(o[4..7], -4, 1).  BF16 weights and activations on the tensor
 * cores, FP32 accumulation, FP32 master weights and Adam moments.
 * Parameter vector (FP32, row-major): W1 [256][32], b1 [256], W2
 * [256][256], b2 [256], W3 [8][256], b3 [8].  A network context lives in a
 * caller-owned device arena (kp_mlp_required_bytes) and works on the
 * stream given at creation. */
#define KP_MLP_INPUTS 32
#define KP_MLP_OUTPUTS 8
typedef struct kp_mlp kp_mlp;
int32_t kp_mlp_num_params(void);
size_t kp_mlp_required_bytes(int32_t max_batch);
/* Copies host_params (kp_mlp_num_params floats); Adam state starts at 0. */
kp_status kp_mlp_create(void *dev_arena, size_t arena_bytes, int32_t max_batch,
                        const float *host_params, void *cuda_stream,
                        kp_mlp **out);
kp_status kp_mlp_set_params(kp_mlp *mlp, const float *host_params);
kp_status kp_mlp_get_params(kp_mlp *mlp, float *host_params);
/* dev_x: device [M][32] FP32 inputs; dev_out: device [M][8] FP32 (mean[4],
 * log_std[4]).  Enqueued only. */
kp_status kp_mlp_forward(kp_mlp *mlp, const float *dev_x, int32_t M,
                         float *dev_out);
/* Gradient of the batch-mean Gaussian negative log-likelihood of the device
 * targets dev_t [M][4] (normalised to [-1, 1]) w.r.t. every parameter, to
 * host_grad (nullable), and the loss (nullable).  Synchronises. */
kp_status kp_mlp_gradients(kp_mlp *mlp, const float *dev_x, const float *dev_t,
                           int32_t M, float *host_grad, float *host_loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss; host_loss
 * (nullable) receives the loss before the step (synchronises). */
kp_status kp_mlp_train_step(kp_mlp *mlp, const float *dev_x,
                            const float *dev_t, int32_t M, float lr,
                            float *host_loss);
/* One epoch of the same training on the device: rows perm[0..rows) of
 * dev_x [rows][32] / dev_t [rows][4] in mini-batches of max_batch rows (a
 * tail shorter than a batch is skipped), each batch gathered into the
 * network's own buffers and its whole step (forward, backward, Adam) run
 * as one CUDA graph launch; the graph is captured on the first call and
 * reused.  dev_perm is a device array of row indices.  host_loss (nullable)
 * receives the mean mini-batch loss.  Synchronises; KP_ERR_TIMEOUT if a
 * tensor-core kernel's bounded wait expired. */
kp_status kp_mlp_train_epoch(kp_mlp *mlp, const float *dev_x, const float *dev_t,
                             const int32_t *dev_perm, int64_t rows, float lr,
                             float *host_loss);
void kp_mlp_destroy(kp_mlp *mlp);
/* Planner use of a network (6D systems): each pass evaluates the network on
 * the features of every V_E node; a sample whose selector draw falls below
 * 'mix' draws its controls and duration from the node's Gaussian (Box-
 * Muller normals from its own Philox counter, clamped to the bounds), the
 * others from the uniform draw.  Propagation and validity are unchanged.
 * NULL detaches.  The network must outlive its use by the context. */
kp_status kp_attach_mlp(kp_ctx *ctx, const kp_mlp *mlp, float mix);
/* Harvest of training pairs (6D systems): every sample that becomes the
 * representative of a newly reached sub-region appends its parent's
 * features (dev_feat [capacity][32]) and its own normalised controls and
 * duration (dev_target [capacity][4]); *dev_count counts the pairs offered
 * (may exceed capacity; the caller zeroes it).  Device pointers; NULL
 * disables. */
kp_status kp_set_harvest(kp_ctx *ctx, float *dev_feat, float *dev_target,
                         int32_t capacity, uint32_t *dev_count);

/* ---- server: many queries in one persistent launch ------------------------
 * A server runs one persistent cooperative launch whose grid is split into
 * teams of team_blocks blocks; each team plans one query at a time (the
 * Algorithm 1 loop of kp_plan) and then takes the next.  Queries of any
 * system, obstacle count and t_e are submitted while others run (continuous
 * batching): a query is admitted when a descriptor slot and a slice of the
 * device pool for its arena (kp_required_bytes) are free, else it waits in
 * submission order.  A query's result depends only on its own inputs, so it
 * is the same alone or among others.  Teams that find no work for idle_ms
 * leave; the server launches again when work arrives.  All device memory
 * comes from the caller's pool (kp_server_required_bytes for the control
 * area plus the query arenas); host memory holds the rings and results.
 * Per query: at most 1,500 obstacle boxes (blob of 48 KB) and
 * kp_required_bytes regions up to 1024 * team_blocks in the padded count;
 * no sample log, learned proposal or harvest. */
typedef struct kp_server kp_server;
typedef struct {
  int32_t team_blocks;  /* blocks per team (>= 1); the grid is the resident
                           maximum rounded down to whole teams           */
  int32_t max_slots;    /* queries resident at once (1 .. 4096)          */
  double idle_ms;       /* a team leaves after this long without work    */
} kp_server_config;
typedef struct {
  int64_t id;
  int32_t status;       /* kp_status: KP_OK solved, KP_NO_SOLUTION, error */
  int32_t n_edges, iterations, n_nodes;
  int64_t samples;      /* samples propagated and checked                */
  double device_ms;     /* device time from its team's start to its end  */
  double latency_ms;    /* host time from submission to completion seen  */
} kp_server_done;
typedef struct {
  int32_t teams, team_blocks, pending, resident;
  int64_t submitted, completed;
  size_t pool_free;
  int32_t device_error;  /* first device-side error (code | site << 8)    */
  int32_t running;       /* 1 while the persistent launch is running      */
} kp_server_stats;
size_t kp_server_required_bytes(int32_t max_slots);
kp_status kp_server_create(const kp_server_config *cfg, void *dev_pool,
                           size_t pool_bytes, void *cuda_stream,
                           kp_server **out);
/* Copies every input; returns the query id in *id. */
kp_status kp_server_submit(kp_server *srv, const kp_system *sys,
                           const kp_workspace *ws, const kp_obstacles *obs,
                           const kp_params *prm, const float *x_init,
                           const kp_goal *goal, const kp_budget *budget,
                           int64_t *id);
/* Completed queries since the last call (up to capacity records); admits
 * waiting queries into the freed resources. */
kp_status kp_server_poll(kp_server *srv, kp_server_done *out, int32_t capacity,
                         int32_t *n_out);
/* Trajectory of a completed, solved query (once; KP_ERR_ARG if unknown or
 * if traj->capacity is too small, n_edges then holds the size needed). */
kp_status kp_server_result(kp_server *srv, int64_t id, kp_traj *traj);
kp_status kp_server_stats_get(kp_server *srv, kp_server_stats *out);
/* Asks the teams to leave after their current query and waits for them. */
void kp_server_destroy(kp_server *srv);

/* Lane-issue peak of the current device, measured: a project kernel in
 * which every thread runs eight independent FP32 fused multiply-add chains
 * (one lane operation each, enough independent work per warp that issue,
 * not latency, bounds the SM) on a full-occupancy grid, timed with CUDA
 * events on 'cuda_stream' (NULL = the legacy default stream), best of five
 * launches after a warm-up.  Writes lane operations per second to
 * *lane_ops_per_s.  This is the measured counterpart of the ALU roofline's
 * denominator (SMs x 128 FP32 lanes x clock).  Allocates no device memory;
 * synchronises the stream.  KP_ERR_ARG for a NULL output, KP_ERR_CUDA when
 * a CUDA call fails. */
kp_status kp_measure_lane_peak(void *cuda_stream, double *lane_ops_per_s);

/* Last error message of the context (never NULL). */
const char *kp_last_error(const kp_ctx *ctx);

/* Frees the context's host memory; the arena stays the caller's. */
void kp_destroy(kp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
