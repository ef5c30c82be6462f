// kp_layout.h -- layout shared by the host driver and the device kernels:
// the launch parameter block (KParams), the device control block (KCtl)
// and the per-sample log pointers (KLog).  Plain C++ (no CUDA types) so the
// host driver compiles it too.
#pragma once

#include <cstdint>

namespace kp {

enum { KP_SYS_DI = 0, KP_SYS_DUBINS = 1, KP_SYS_QUAD = 2 };

// planner state stored in KCtl::state
enum { KP_DEV_RUNNING = 0, KP_DEV_SOLVED = 1, KP_DEV_FULL = 2, KP_DEV_BAD_ROOT = -1 };
// launch errors stored in KCtl::err
// KP_DEV_ERR_REPLAY: with the sample log on, an accepted sample re-derived
// from its key when it is appended differed from its first derivation.
// KP_DEV_ERR_BOUNDS (bounds-checked build only): an array index outside its
// array; err_where holds the site.
enum { KP_DEV_OK = 0, KP_DEV_ERR_TIMEOUT = 1, KP_DEV_ERR_REPLAY = 2, KP_DEV_ERR_BOUNDS = 3 };
// per-sample flag bits
enum {
  KP_F_VALID = 1,
  KP_F_CONTENDER = 2,
  KP_F_BERN = 4,
  KP_F_WINNER = 8,
  KP_F_ACCEPTED = 16,
  KP_F_GOAL = 32
};

constexpr int KP_BLOCK = 256;          // threads per block of the loop kernel
constexpr int KP_MAX_GRID = 8192;      // upper bound on loop-kernel blocks
constexpr int KP_NO_GOAL = 0x7fffffff; // goal_node sentinel on the device
constexpr int KP_TRAJ_ROWS = 16384;    // longest root-to-goal chain returned
constexpr int KP_BP_MAX_G = 16;        // finest broad-phase grid per axis
constexpr int KP_BP_MAX_IDS = 32768;   // broad-phase (cell, box) entries
constexpr int KP_BLOB_BYTES = 4096 * 32 + (KP_BP_MAX_G * KP_BP_MAX_G * KP_BP_MAX_G + 4) * 4 +
                              KP_BP_MAX_IDS * 2 +
                              KP_BP_MAX_G * KP_BP_MAX_G * KP_BP_MAX_G;  // arena room for the obstacle blob
// per-cell clearance of the broad-phase grid: stored in 1/16 of a cell,
// computed up to KP_BP_CLEAR_CAP cells, less a margin for FP32 rounding
constexpr int KP_BP_CLEAR_CAP = 4;
constexpr double KP_BP_CLEAR_MARGIN = 1e-3;
constexpr int KP_FSO_MAX_LEAVES = 16384; // regions of a kd-tree decomposition
// floats per kept end state (one aligned row of whole 32-byte sectors per key)
__host__ __device__ constexpr int kp_xs_stride(int D) { return D <= 8 ? 8 : 16; }
constexpr int KP_FSO_MAX_DEPTH = 64;     // its deepest leaf

// Device control block (one per context, in the arena).
struct KCtl {
  // loop state, persistent across launches
  int32_t n_nodes;     // |T|
  int32_t n_ve;        // |V_E|
  int32_t iteration;   // next pass index
  int32_t goal_node;   // KP_NO_GOAL when none
  int32_t state;       // KP_DEV_*
  int32_t err;         // KP_DEV_ERR_* of the last launch
  int32_t err_where;
  int32_t n_run;       // passes run by the last launch
  int32_t stop;        // loop stop flag inside a launch
  uint32_t it_valid;   // valid samples of the current pass
  int32_t n_edges;     // trajectory extraction: edges on the chain
  int32_t work_next;   // next sample key handed out in the expand phase
  uint32_t t_done;     // region chunks whose thresholds are written, this pass
  uint32_t reset_done; // blocks of the reset launch that finished their clears
  double score_sum;    // sum of Eq. 5 over R_avail, this pass
  // work counters since the last reset (samples, integrator steps run,
  // segment hulls tested against the obstacle set)
  unsigned long long tot_samples;
  unsigned long long tot_steps;
  unsigned long long tot_hull;
  unsigned long long tot_box_tests;
  // launch-shape counters since the last reset: key batches taken from the
  // grid-wide counter (beyond each warp's first, fixed batch), and keys
  // started by a lane that had already run a key in the same pass
  unsigned long long tot_batches;
  unsigned long long tot_refills;
  // grid barrier word (top bit: phase) on its own 128-byte line
  uint32_t bar;
  uint32_t pad1[31];
  // never set: target of the bounded-wait self test
  uint32_t never_set;
  uint32_t pad3[31];
};

struct KLog {
  int32_t capacity;  // 0 = off
  int32_t* node;
  int32_t* k;
  uint32_t* uraw;    // [cap][4]
  uint8_t* flags;
  int32_t* fail_step;
  int32_t* region;
  int32_t* sub;
  float* state;      // [cap][12]
};

struct KStats {
  int32_t iteration, n_ve, lambda, n_samples, n_valid, n_accepted, n_nodes, goal_node;
  // device time of the pass as seen by block 0 (ns): work then barrier wait
  // of each phase: [0,1] Propagate, [2] accept + Score, [3] features and
  // network, [4] wait, [5] 0, [6] wait after [3], [7] 0, [8] P_accept,
  // new nodes and node sets, [9] wait, [10] V_E list and Eq. 6, [11]
  // previous pass's final wait
  int32_t phase_ns[12];
};

// x_init of a reset, passed by value.
// what a loop launch does around its passes
enum {
  KP_LOOP_RESET = 1,   // Algorithm 1's initialisation first (tables cleared, root)
  KP_LOOP_EXTRACT = 2  // the root-to-goal chain written to the trajectory rows after
};

struct RootState {
  float x[12];
};

// Launch parameters (passed by value; ~1 KB).
struct KParams {
  // system (Sec. II)
  int32_t sys;
  float dt;
  float dt_sixth;   // dt / 6 (RK4 combination), IEEE FP32 division on the host
  int32_t k_min;
  uint32_t k_span;  // k_max - k_min + 1
  float x_lo[12], x_hi[12];
  float u_lo[4], u_scale[4];  // u = u_lo + u_scale * r
  float phys[16];
  float recip[4];       // quadrotor 1/m, 1/Ixx, 1/Iyy, 1/Izz
  // decomposition (Sec. III)
  float ws_lo[3];
  float fine_scale[3];  // fine cells per unit length
  int32_t n_fine[3];    // grid * sub per axis
  float n_fine_last[3]; // n_fine - 1 per axis, as a float
  int32_t sub[3];
  int32_t sub_shift[3]; // log2(sub) when sub is a power of two, else -1
  int32_t grid[3];
  int32_t speed_bins;
  float speed_scale;    // speed_bins / speed_hi
  int32_t state_grid[12];  // cells over state dimension d (1: not decomposed)
  float state_scale[12];   // cells per unit of that dimension
  int32_t state_wrap[12];  // 1: an angle, wrapped to [-pi, pi) before binning
  // free-space-obeying decomposition (fso = 1): a kd-tree over position;
  // node i: (axis << 30) | right child for a split at kd_split[i] (the left
  // child is i + 1; a point below the plane goes left), (3 << 30) | leaf
  // for a leaf; leaf r: leaf_box[2r] = lo.xyz, leaf_box[2r+1] = sub-grid
  // cells per unit length; region_vol[r] = its volume (Eq. 3)
  int32_t fso;
  int32_t kd_n;         // tree nodes
  int32_t kd_smem_off;  // byte offset in the staged blob of a copy of the
                        // codes (kd_n) then the splits (kd_n); -1: global
  const int32_t* kd_node;
  const float* kd_split;
  const float4* leaf_box;
  const double* region_vol;
  int32_t n_sub_per;    // n'
  int32_t R;            // regions
  int32_t R_pad;        // next power of two >= R
  int32_t nch;          // region chunks of the score sum (power of two)
  // goal set
  float goal_c[3];
  float goal_r2;
  // constants
  int32_t t_e;
  int32_t lambda_max;
  double delta, eps, vol;
  uint32_t seed_lo, seed_hi;
  // obstacles: a blob staged whole into shared memory:
  //   [n_boxes_pad][8] floats (lo.xyz, pad, hi.xyz, pad), then the
  //   broad-phase grid: uint16 cell_start[bp_g[0] bp_g[1] bp_g[2] + 1], uint16 ids[...],
  //   then (optionally) uint8 clearance[cells]: q / 16 cells of free space
  //   around the cell in every axis (L-infinity, in each axis's cell units)
  const float* boxes;
  int32_t n_boxes_pad;
  int32_t blob_bytes;
  int32_t sd_bytes;      // score scratch after the blob; the network tile follows
  int32_t extract_cap;   // chain ids kept in shared memory at most (0: room only)
  int32_t bp_g[3];       // broad-phase cells along x, y, z (1 1 1: every box in one cell)
  int32_t bp_start_off;  // byte offsets inside the blob
  int32_t bp_ids_off;
  int32_t bp_clear_off;  // the cells' clearances (uint8), -1: none
  int32_t bp_n_ids;      // (cell, box) entries of the grid
  float bp_scale[3];     // cells per unit length, per axis
  float bp_last[3];      // bp_g - 1 per axis, as a float
  // tree, SoA over t_e nodes
  float* st;          // [D][t_e]
  int32_t* parent;
  float* ctrl;        // [N][t_e]
  uint8_t* steps;
  int32_t* region;
  int32_t* node_sub;  // global sub-region index of each node
  uint8_t* in_ve;
  // per-sample scratch, indexed by sample key (< t_e)
  int32_t* cs;        // sub-region of a contender (claim check)
  float* xs;          // [t_e][kp_xs_stride(D)] end state of a sample that may be accepted
  uint8_t* flags;     // KP_F_* of the sample
  // accepted samples: each accept warp compacts its keys (winner flag in
  // bit 31) at the start of its own key range, in key order
  uint32_t* acc_key;
  // decomposition tables
  uint32_t* n_valid;
  uint32_t* n_invalid;
  uint32_t* cov;
  uint8_t* avail;
  uint8_t* visited;   // [R * n']
  uint32_t* claim;    // [R * n'] smallest sample key, 0xffffffff = none
  double* score;
  uint64_t* thr;      // accept iff word < thr
  // loop scratch
  int32_t* ve;        // V_E list
  uint32_t* blk_a;    // [KP_MAX_GRID]
  uint32_t* blk_b;    // [KP_MAX_GRID]
  double* chunk_sum;  // [KP_MAX_GRID]
  KCtl* ctl;
  KStats* stats;
  int32_t stats_cap;
  float* traj;        // [KP_TRAJ_ROWS][17]: state 12, ctrl 4, steps
  KLog log;
  uint64_t wait_ns;
  // learned proposal and training-pair harvest (6D systems)
  const uint16_t* mlp_W1;  // bf16 [256][32]
  const float* mlp_b1;
  const uint16_t* mlp_W2;  // bf16 [256][256]
  const float* mlp_b2;
  const uint16_t* mlp_W3;  // bf16 [8][256]
  const float* mlp_b3;
  uint32_t mix_thr;        // learned draw iff selector word < mix_thr (0: off)
  int32_t features_on;     // node features computed each pass
  uint16_t* feat;          // bf16 [t_e][32]: features of the V_E positions
  float* net_raw;          // [t_e][8]: network outputs of the V_E positions
  float feat_scale[6];     // 2 / (hi - lo) of a bounded state entry, 0 if unbounded
  float* hv_feat;          // harvest: [hv_cap][32]
  float* hv_target;        // [hv_cap][4]
  uint32_t* hv_count;
  int32_t hv_cap;
};

// ---------------------------------------------------------------------------
// server: many queries in one persistent launch (teams of blocks)
// ---------------------------------------------------------------------------

constexpr int KS_MAX_TEAMS = 1024;
constexpr int KS_RING = 4096;          // submission / completion ring entries
constexpr uint32_t KS_EXIT = 0xffffffffu;
constexpr int KS_SD_DOUBLES = 1024;    // score scratch of a server block
constexpr int KS_BLOB_MAX = 49152;     // obstacle blob of a server query (bytes)

// One admitted query, written by the host into its descriptor slot.
struct KQuery {
  KParams P;           // constants and the query's arena slices
  RootState root;
  int32_t max_iters;
  int32_t id;
  uint64_t max_ns;
};

// Completion record, written by the device into host-mapped memory.
struct KDone {
  int32_t slot, state, err, n_edges;
  int32_t iterations, n_nodes, goal_node, pad;
  unsigned long long samples, t_start_ns, t_end_ns;
  uint32_t seq;        // written last: index + 1 of this record
  uint32_t pad2[3];
};

// Host-mapped area: submissions (host writes) and completions (device
// writes).
struct KServerHost {
  uint32_t posted;     // queries published so far
  uint32_t stop;       // the host asks the teams to leave
  int32_t error;       // device: first server error (code | site << 8), 0 if none
  uint32_t pad[29];
  uint32_t ring[KS_RING];  // descriptor slot of the i-th published query
  KDone done[KS_RING];
};

// Device control area of a server.
struct KServerDev {
  KCtl sctl;           // server-level error word and barrier scratch
  uint32_t taken;      // published queries claimed by teams
  uint32_t done_seq;   // completion records published
  uint32_t pad[30];
  uint32_t team_slot[KS_MAX_TEAMS];
  uint32_t team_bar[KS_MAX_TEAMS][32];  // [0] barrier word, one 128-byte line a team
};

struct KServerArgs {
  KServerDev* dev;
  KServerHost* host;   // device alias of the host-mapped area
  const KQuery* queries;
  int32_t team_blocks;
  int32_t pad;
  uint64_t idle_ns;    // a team leaves after this long without work
  uint64_t wait_ns;    // bound of every other device wait
};

}  // namespace kp
