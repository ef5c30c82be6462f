// kp_api.cu -- host driver behind the C ABI of include/kp.h: arena layout,
// context lifetime, launches of the loop kernel, tree import/export, and the
// small generic kernels (trajectory extraction, import fix-up, wait self
// test).  The library allocates no device memory: every device array is a
// slice of the caller's arena.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/kp.h"
#include "kp_device.cuh"
#include "kp_mlp.cuh"

struct kp_mlp;
namespace kp {
void mlp_device_weights(const kp_mlp* n, const void** W1, const float** b1, const void** W2,
                        const float** b2, const void** W3, const float** b3);
cudaError_t server_occupancy(size_t smem, int* blocks_per_sm);
cudaError_t launch_server(const KServerArgs& A, int grid, size_t smem, cudaStream_t stream);
// launchers defined in kp_sys_*.cu
#define KP_DECLARE_SYS(name)                                                                   \
  cudaError_t loop_occupancy_##name(bool log, size_t smem, int* blocks_per_sm);                \
  cudaError_t launch_loop_##name(const KParams& P, int grid, size_t smem, int max_iters,        \
                                 uint64_t max_ns, bool log, cudaStream_t stream,               \
                                 const RootState& root, int mode);                             \
  cudaError_t launch_reset_##name(const KParams& P, const RootState& root, cudaStream_t stream);
KP_DECLARE_SYS(di)
KP_DECLARE_SYS(dubins)
KP_DECLARE_SYS(quad)
#undef KP_DECLARE_SYS

// ---------------------------------------------------------------------------
// generic kernels
// ---------------------------------------------------------------------------

// Root-to-goal chain into P.traj rows (state 12, ctrl 4, steps), root first,
// as a launch of its own after the no-allocation entry's loop launch (the
// queries of a context do this inside their loop launch).
__global__ void kp_extract_kernel(KParams P) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  KCtl* ctl = P.ctl;
  const int g = ctl->goal_node;
  if (g == KP_NO_GOAL || g < 0 || g >= P.t_e) {
    ctl->n_edges = -1;
    return;
  }
  int len = 0;
  for (int v = g; v > 0 && len <= P.t_e; v = P.parent[v]) ++len;
  ctl->n_edges = len;
  if (len > KP_TRAJ_ROWS) return;
  const int D = P.sys == KP_SYS_QUAD ? 12 : 6;
  const int N = P.sys == KP_SYS_QUAD ? 4 : 3;
  int row = len - 1;
  for (int v = g; v > 0 && row >= 0; v = P.parent[v], --row) {
    float* out = P.traj + (size_t)row * 17;
    for (int i = 0; i < 12; ++i) out[i] = i < D ? P.st[(size_t)i * P.t_e + v] : 0.0f;
    for (int i = 0; i < 4; ++i) out[12 + i] = i < N ? P.ctrl[(size_t)i * P.t_e + v] : 0.0f;
    out[16] = (float)P.steps[v];
  }
}

// Import fix-up: Cov from the visited flags, R_avail cleared.
__global__ void kp_import_regions_kernel(KParams P) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += gridDim.x * blockDim.x) {
    uint32_t c = 0;
    for (int k = 0; k < P.n_sub_per; ++k) c += P.visited[(size_t)r * P.n_sub_per + k] ? 1u : 0u;
    P.cov[r] = c;
    P.avail[r] = 0;
  }
}

// Import fix-up: R_avail from the node regions.
__global__ void kp_import_avail_kernel(KParams P, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    P.avail[P.region[v]] = 1;
}

// The bounds check itself (checked build only): an index one past the
// tree is looked up through the checked-index path, which records the
// error and reads element 0 instead.
__global__ void kp_bounds_selftest_kernel(KParams P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
#ifdef KP_CHECK
  const int v = KP_IDX(P, P.t_e, P.t_e, 97);
  P.ctl->n_edges = (int)P.in_ve[v];
#endif
}

// Bounded wait on a flag that nothing sets; records the timeout.
__global__ void kp_wait_selftest_kernel(KParams P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  KCtl* ctl = P.ctl;
  const uint64_t t0 = global_ns();
  while (ld_acquire(&ctl->never_set) == 0) {
    if (global_ns() - t0 > P.wait_ns) {
      raise_error(ctl, KP_DEV_ERR_TIMEOUT, 99);
      return;
    }
  }
}

}  // namespace kp

using namespace kp;

// ---------------------------------------------------------------------------
// arena layout
// ---------------------------------------------------------------------------

namespace {

constexpr int kStatsCap = 4096;
constexpr int kFirstRows = 256;  // trajectory rows read with the header

struct Dims {
  int sys, D, N, R, R_pad, n_sub_per, t_e, boxes_pad;
  size_t n_sub;
  // the tables hold R_tab regions: R itself for a grid; for the kd-tree
  // decomposition the leaf capacity, R being the leaves of the current
  // obstacle set
  int fso, R_tab;
  size_t n_sub_tab;
};

struct Layout {
  size_t ctl, boxes, st, parent, ctrl, steps, region, sub, in_ve, cs, xs, flags, acc_key,
      n_valid, n_invalid, cov, avail, visited, claim, score, thr, ve, blk_a, blk_b, chunk_sum,
      stats, traj, feat, net_raw, kd_node, kd_split, leaf_box, region_vol, total;
};

// Bytes of the kd-tree slices (nodes, splits, leaf boxes, leaf volumes);
// they are contiguous in the arena from Layout::kd_node on.
constexpr size_t kKdNodes = 2 * (size_t)KP_FSO_MAX_LEAVES;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout make_layout(const Dims& d) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t te = (size_t)d.t_e;
  L.ctl = take(sizeof(KCtl));
  // room for any obstacle set and its grid (and a compact copy of a kd-tree
  // after it, staged with it when shared memory allows)
  L.boxes = take((size_t)KP_BLOB_BYTES + (d.fso ? kKdNodes * 8 : 0));
  L.st = take(te * d.D * 4);
  L.parent = take(te * 4);
  L.ctrl = take(te * d.N * 4);
  L.steps = take(te);
  L.region = take(te * 4);
  L.sub = take(te * 4);
  L.in_ve = take(te);
  L.cs = take(te * 4);
  L.xs = take(te * (size_t)kp_xs_stride(d.D) * 4);
  L.flags = take(te);
  L.acc_key = take(te * 4);
  L.n_valid = take((size_t)d.R_tab * 4);
  L.n_invalid = take((size_t)d.R_tab * 4);
  L.cov = take((size_t)d.R_tab * 4);
  L.avail = take((size_t)d.R_tab);
  L.visited = take(d.n_sub_tab);
  L.claim = take(d.n_sub_tab * 4);
  L.score = take((size_t)d.R_tab * 8);
  L.thr = take((size_t)d.R_tab * 8);
  L.ve = take(te * 4);
  L.blk_a = take((size_t)KP_MAX_GRID * 4);
  L.blk_b = take((size_t)KP_MAX_GRID * 4);
  L.chunk_sum = take((size_t)KP_MAX_GRID * 8);
  L.stats = take((size_t)kStatsCap * sizeof(KStats));
  L.traj = take((size_t)KP_TRAJ_ROWS * 17 * 4);
  L.feat = take(te * 32 * 2);     // bf16 node features of the V_E positions
  L.net_raw = take(te * 8 * 4);   // network outputs of the V_E positions
  if (d.fso) {
    L.kd_node = take(kKdNodes * 4);
    L.kd_split = take(kKdNodes * 4);
    L.leaf_box = take((size_t)KP_FSO_MAX_LEAVES * 32);
    L.region_vol = take((size_t)KP_FSO_MAX_LEAVES * 8);
  }
  L.total = off;
  return L;
}

bool finite_or_inf(float v) { return !std::isnan(v); }

// Validates the inputs; fills dims.  Returns an error message or nullptr.
const char* check_inputs(const kp_system* sys, const kp_workspace* ws, int32_t n_boxes,
                         const kp_params* prm, Dims* d) {
  if (!sys || !ws || !prm) return "null argument";
  if (sys->id < 0 || sys->id > 2) return "unknown system id";
  if (!(sys->dt > 0.0f) || !std::isfinite(sys->dt)) return "dt must be positive";
  if (sys->k_min < 1 || sys->k_max < sys->k_min || sys->k_max > 255) return "bad k range";
  d->sys = sys->id;
  d->D = sys->id == KP_QUADROTOR_12D ? 12 : 6;
  d->N = sys->id == KP_QUADROTOR_12D ? 4 : 3;
  for (int i = 0; i < d->D; ++i)
    if (!finite_or_inf(sys->x_lo[i]) || !finite_or_inf(sys->x_hi[i]) ||
        !(sys->x_lo[i] <= sys->x_hi[i]))
      return "bad state bounds";
  if (sys->id == KP_QUADROTOR_12D)
    for (int i : {0, 4, 5, 6})
      if (!(sys->phys[i] > 0.0f) || !std::isfinite(sys->phys[i])) return "quadrotor mass and inertia must be positive";
  for (int i = 0; i < d->N; ++i)
    if (!std::isfinite(sys->u_lo[i]) || !std::isfinite(sys->u_hi[i]) ||
        !(sys->u_lo[i] <= sys->u_hi[i]))
      return "bad control bounds";
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(ws->lo[a]) || !std::isfinite(ws->hi[a]) || !(ws->lo[a] < ws->hi[a]))
      return "bad workspace";
    if (ws->grid[a] < 1 || ws->sub[a] < 1 || ws->grid[a] > 4096 || ws->sub[a] > 4096)
      return "bad grid";
    // fine cells per axis below 2^22: the device floors cell coordinates by
    // an add of 2^23, exact below it
    if ((long long)ws->grid[a] * ws->sub[a] > (1 << 22)) return "bad grid";
  }
  if (ws->speed_bins < 1 || ws->speed_bins > 4096) return "bad speed bins";
  if (ws->speed_bins > 1 && !(ws->speed_hi > 0.0f)) return "bad speed range";
  if (n_boxes < 0 || n_boxes > KP_MAX_BOXES) return "bad box count";
  if (prm->t_e < 2 || prm->t_e > (1 << 28)) return "t_e out of range";
  if (prm->lambda_max < 1 || prm->lambda_max > 1024) return "lambda_max out of range";
  if (!(prm->delta > 0.0) || !(prm->eps > 0.0) || !(prm->eps < 1.0)) return "bad delta/eps";
  if (ws->fso != 0 && ws->fso != 1) return "fso must be 0 or 1";
  long long R = (long long)ws->grid[0] * ws->grid[1] * ws->grid[2] * ws->speed_bins;
  for (int dd = 3; dd < d->D; ++dd) {
    if (ws->state_grid[dd] < 0 || ws->state_grid[dd] > 4096) return "bad state grid";
    if (ws->state_grid[dd] > 1) R *= ws->state_grid[dd];
  }
  const long long nsp = (long long)ws->sub[0] * ws->sub[1] * ws->sub[2];
  d->fso = ws->fso;
  if (d->fso) R = KP_FSO_MAX_LEAVES;  // the leaf count comes with the obstacles
  if (R > (1 << 24) || R * nsp > (1ll << 30)) return "decomposition too large";
  d->R_tab = (int)R;
  d->n_sub_tab = (size_t)(R * nsp);
  d->R = d->fso ? 1 : (int)R;
  d->R_pad = 1;
  while (d->R_pad < d->R) d->R_pad *= 2;
  d->n_sub_per = (int)nsp;
  d->n_sub = (size_t)d->R * (size_t)nsp;
  d->t_e = prm->t_e;
  d->boxes_pad = (n_boxes + 7) / 8 * 8;
  return nullptr;
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct kp_ctx {
  Dims dims;
  Layout lay;
  kp_system sys;
  kp_workspace ws;
  kp_params prm;
  int n_boxes_cap;
  char* arena;
  size_t arena_bytes;
  cudaStream_t stream;
  int device;
  int num_sms;
  KParams P;  // pointers and constants; goal/seed/log per launch
  kp_goal goal;
  uint64_t seed;
  bool have_tree;
  bool poisoned;
  bool log_on;
  KLog log;
  uint64_t wait_ns;
  int grid[2];
  int grid_limit;  // 0: the resident maximum; else at most this many blocks
  size_t smem;
  int blob_base;  // blob bytes without the kd-tree copy
  int blob_kd;    // blob bytes with it (0: no tree)
  std::string err;
  void* pinned;
  size_t pinned_bytes;
  cudaEvent_t ev_loop0, ev_loop1;  // bracket every loop-kernel launch
  bool loop_timed;
  bool plan_pending;               // kp_plan_async issued, result not read
  int plan_rows;
};

namespace {

kp_status fail(kp_ctx* c, kp_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    if (s == KP_ERR_CUDA || s == KP_ERR_TIMEOUT) c->poisoned = true;
  }
  return s;
}

#define KP_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, KP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                 \
  } while (0)

cudaError_t occupancy(int sys, bool log, size_t smem, int* bps) {
  switch (sys) {
    case KP_SYS_DI: return loop_occupancy_di(log, smem, bps);
    case KP_SYS_DUBINS: return loop_occupancy_dubins(log, smem, bps);
    default: return loop_occupancy_quad(log, smem, bps);
  }
}

// mode: KP_LOOP_RESET (Algorithm 1's initialisation from root first) and
// KP_LOOP_EXTRACT (the root-to-goal chain after the passes), or 0.
cudaError_t launch_loop(kp_ctx* c, const KParams& P, int max_iters, uint64_t max_ns,
                        const RootState& root = RootState{}, int mode = 0) {
  const bool log = c->log_on;
  const int g = c->grid[log ? 1 : 0];
  cudaError_t e = cudaEventRecord(c->ev_loop0, c->stream);
  if (e != cudaSuccess) return e;
  switch (c->dims.sys) {
    case KP_SYS_DI:
      e = launch_loop_di(P, g, c->smem, max_iters, max_ns, log, c->stream, root, mode);
      break;
    case KP_SYS_DUBINS:
      e = launch_loop_dubins(P, g, c->smem, max_iters, max_ns, log, c->stream, root, mode);
      break;
    default: e = launch_loop_quad(P, g, c->smem, max_iters, max_ns, log, c->stream, root, mode);
  }
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(c->ev_loop1, c->stream);
  c->loop_timed = e == cudaSuccess;
  return e;
}

cudaError_t launch_reset(kp_ctx* c, const KParams& P, const RootState& root) {
  switch (c->dims.sys) {
    case KP_SYS_DI: return launch_reset_di(P, root, c->stream);
    case KP_SYS_DUBINS: return launch_reset_dubins(P, root, c->stream);
    default: return launch_reset_quad(P, root, c->stream);
  }
}

template <class T>
T* at(kp_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->arena + off);
}

// Launch parameters for the context's current goal, seed and log.
KParams params_now(kp_ctx* c) {
  KParams P = c->P;
  for (int a = 0; a < 3; ++a) P.goal_c[a] = c->goal.center[a];
  P.goal_r2 = (float)((double)c->goal.radius * (double)c->goal.radius);
  P.seed_lo = (uint32_t)(c->seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(c->seed >> 32);
  P.log = c->log_on ? c->log : KLog{};
  P.wait_ns = c->wait_ns;
  return P;
}

kp_status check_ctx(kp_ctx* c) {
  if (!c) return KP_ERR_ARG;
  if (c->poisoned) return KP_ERR_STATE;
  return KP_OK;
}

kp_status ensure_pinned(kp_ctx* ctx, size_t bytes) {
  if (ctx->pinned_bytes >= bytes) return KP_OK;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  KP_CUDA(cudaHostAlloc(&ctx->pinned, bytes, cudaHostAllocDefault));
  ctx->pinned_bytes = bytes;
  return KP_OK;
}

// Reads the control block back (synchronises the stream).
kp_status read_ctl(kp_ctx* ctx, KCtl* out) {
  kp_status s = ensure_pinned(ctx, sizeof(KCtl));
  if (s != KP_OK) return s;
  KP_CUDA(cudaMemcpyAsync(ctx->pinned, at<KCtl>(ctx, ctx->lay.ctl), sizeof(KCtl),
                          cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, ctx->pinned, sizeof(KCtl));
  return KP_OK;
}


size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

// Broad-phase cell of a coordinate: the device's bp_cell in host FP32.
int host_bp_cell(float v, float lo, float scale, int g) {
  const float t = (v - lo) * scale;
  return t >= 0.0f ? (t < (float)g ? (int)t : g - 1) : 0;
}

// Cell ranges of every padded box on the grid g (cells per axis), with the
// grid's scale; returns the (cell, box) entry count.
long long bp_ranges(const float* fb, int nb, const kp_workspace& ws, const int g[3],
                    float scale[3], std::vector<int>& lo3, std::vector<int>& hi3) {
  for (int a = 0; a < 3; ++a) scale[a] = (float)((double)g[a] / ((double)ws.hi[a] - (double)ws.lo[a]));
  lo3.resize((size_t)nb * 3);
  hi3.resize((size_t)nb * 3);
  long long entries = 0;
  for (int b = 0; b < nb; ++b) {
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
      lo3[(size_t)b * 3 + a] = host_bp_cell(fb[b * 8 + a], ws.lo[a], scale[a], g[a]);
      hi3[(size_t)b * 3 + a] = host_bp_cell(fb[b * 8 + 4 + a], ws.lo[a], scale[a], g[a]);
      cells *= hi3[(size_t)b * 3 + a] - lo3[(size_t)b * 3 + a] + 1;
    }
    entries += cells;
  }
  return entries;
}

// Writes the obstacle blob (padded boxes, then the broad-phase grid: cell
// start offsets and box ids of every cell a box overlaps) into 'blob' and
// sets the blob fields of P.
//
// The grid has 4096 cells in one of seven shapes: 16 x 16 x 16, 64 x 64 x 1
// (and its two rotations), 32 x 32 x 4 (and its two rotations).  The shape
// taken is the one with the smallest sum over cells of the squared box
// count, among those whose entries fit KP_BP_MAX_IDS and the byte budget:
// the lanes of a warp test the boxes of their own cells and wait for the
// longest list, so crowded cells cost more than their share.  Obstacles
// that span the workspace along an axis (trees of a forest) make that axis
// useless to the grid and the flat shapes win; boxes of every orientation
// keep the cube.  If no shape fits, the finest of 8^3, 4^3, 2^3 and 1 cell
// (every box) that fits is used.
//
// With 'clearance', a byte per cell follows: the cell's clearance, the
// smallest over boxes of the largest per-axis gap between the cell and the
// box, in that axis's cell units (an L-infinity distance), capped at
// KP_BP_CLEAR_CAP cells, less KP_BP_CLEAR_MARGIN, in sixteenths of a cell
// rounded down.  A hull inside its cell grown by that much on every side is
// separated from every box along some axis, so it meets none.
size_t build_blob(unsigned char* blob, const float* boxes, int nb, const kp_workspace& ws,
                  KParams& P, size_t max_bytes = KP_BLOB_BYTES, bool clearance = true) {
  const int pad = (nb + 7) / 8 * 8;
  float* fb = reinterpret_cast<float*>(blob);
  for (int b = 0; b < pad; ++b) {
    float* o = fb + (size_t)b * 8;
    if (b < nb) {
      const float* in = boxes + (size_t)b * 6;
      // + 0.0f: no negative zeros reach the sign-bit box test
      o[0] = in[0] + 0.0f; o[1] = in[1] + 0.0f; o[2] = in[2] + 0.0f; o[3] = 0.0f;
      o[4] = in[3] + 0.0f; o[5] = in[4] + 0.0f; o[6] = in[5] + 0.0f; o[7] = 0.0f;
    } else {  // padding: an empty box no hull can meet
      o[0] = o[1] = o[2] = INFINITY;
      o[4] = o[5] = o[6] = -INFINITY;
      o[3] = o[7] = 0.0f;
    }
  }
  auto blob_size = [&](const int g[3], long long entries) {
    return (size_t)pad * 32 + round16((size_t)(g[0] * g[1] * g[2] + 1) * 2) +
           round16((size_t)entries * 2);
  };
  auto fits = [&](const int g[3], long long entries) {
    return entries <= KP_BP_MAX_IDS && blob_size(g, entries) <= max_bytes;
  };
  static const int kShapes[7][3] = {{16, 16, 16}, {64, 64, 1}, {64, 1, 64}, {1, 64, 64},
                                    {32, 32, 4},  {32, 4, 32}, {4, 32, 32}};
  static_assert(KP_BP_MAX_G * KP_BP_MAX_G * KP_BP_MAX_G == 4096, "grid shapes hold 4096 cells");
  int g[3] = {1, 1, 1};
  float scale[3];
  std::vector<int> lo3, hi3;
  if (nb > 0) {
    long long best = -1;
    std::vector<int> count(4096);
    for (const auto& s : kShapes) {
      const long long entries = bp_ranges(fb, nb, ws, s, scale, lo3, hi3);
      if (!fits(s, entries)) continue;
      std::fill(count.begin(), count.end(), 0);
      for (int b = 0; b < nb; ++b)
        for (int z = lo3[(size_t)b * 3 + 2]; z <= hi3[(size_t)b * 3 + 2]; ++z)
          for (int y = lo3[(size_t)b * 3 + 1]; y <= hi3[(size_t)b * 3 + 1]; ++y)
            for (int x = lo3[(size_t)b * 3]; x <= hi3[(size_t)b * 3]; ++x)
              count[(size_t)x + (size_t)s[0] * ((size_t)y + (size_t)s[1] * z)] += 1;
      long long sq = 0;
      for (int c : count) sq += (long long)c * c;
      if (best < 0 || sq < best) {
        best = sq;
        for (int a = 0; a < 3; ++a) g[a] = s[a];
      }
    }
    if (best < 0)
      for (int gi = KP_BP_MAX_G / 2; gi >= 1; gi /= 2) {
        const int s[3] = {gi, gi, gi};
        if (fits(s, bp_ranges(fb, nb, ws, s, scale, lo3, hi3)) || gi == 1) {
          for (int a = 0; a < 3; ++a) g[a] = gi;
          break;
        }
      }
  }
  bp_ranges(fb, nb, ws, g, scale, lo3, hi3);
  const int C = g[0] * g[1] * g[2];
  const size_t start_off = (size_t)pad * 32;
  const size_t ids_off = start_off + round16((size_t)(C + 1) * 2);
  // cell starts fit in 16 bits: at most KP_BP_MAX_IDS (< 65536) ids, or the
  // box count for the single-cell grid
  uint16_t* start16 = reinterpret_cast<uint16_t*>(blob + start_off);
  uint16_t* ids = reinterpret_cast<uint16_t*>(blob + ids_off);
  auto cell = [&](int x, int y, int z) { return x + g[0] * (y + g[1] * z); };
  std::vector<int> start((size_t)C + 1, 0);
  for (int b = 0; b < nb; ++b)
    for (int z = lo3[(size_t)b * 3 + 2]; z <= hi3[(size_t)b * 3 + 2]; ++z)
      for (int y = lo3[(size_t)b * 3 + 1]; y <= hi3[(size_t)b * 3 + 1]; ++y)
        for (int x = lo3[(size_t)b * 3]; x <= hi3[(size_t)b * 3]; ++x) start[cell(x, y, z) + 1] += 1;
  for (int c = 0; c < C; ++c) start[c + 1] += start[c];
  for (int c = 0; c <= C; ++c) start16[c] = (uint16_t)start[c];
  std::vector<int> cursor(start.begin(), start.begin() + C);
  for (int b = 0; b < nb; ++b)
    for (int z = lo3[(size_t)b * 3 + 2]; z <= hi3[(size_t)b * 3 + 2]; ++z)
      for (int y = lo3[(size_t)b * 3 + 1]; y <= hi3[(size_t)b * 3 + 1]; ++y)
        for (int x = lo3[(size_t)b * 3]; x <= hi3[(size_t)b * 3]; ++x)
          ids[cursor[cell(x, y, z)]++] = (uint16_t)b;
  size_t bytes = ids_off + round16((size_t)start[C] * 2);
  P.bp_clear_off = -1;
  if (clearance && bytes + round16((size_t)C) <= max_bytes) {
    // every box lowers the clearance of the cells within the cap of it
    std::vector<double> rc((size_t)C, (double)KP_BP_CLEAR_CAP);
    double sc[3];
    for (int a = 0; a < 3; ++a) sc[a] = (double)g[a] / ((double)ws.hi[a] - (double)ws.lo[a]);
    for (int b = 0; b < nb; ++b) {
      double bl[3], bh[3];
      int c0[3], c1[3];
      for (int a = 0; a < 3; ++a) {
        bl[a] = ((double)fb[b * 8 + a] - (double)ws.lo[a]) * sc[a];
        bh[a] = ((double)fb[b * 8 + 4 + a] - (double)ws.lo[a]) * sc[a];
        const double f0 = std::floor(bl[a]) - KP_BP_CLEAR_CAP, f1 = std::floor(bh[a]) + KP_BP_CLEAR_CAP;
        c0[a] = f0 < 0.0 ? 0 : (f0 > g[a] - 1 ? g[a] - 1 : (int)f0);
        c1[a] = f1 < 0.0 ? 0 : (f1 > g[a] - 1 ? g[a] - 1 : (int)f1);
      }
      for (int z = c0[2]; z <= c1[2]; ++z)
        for (int y = c0[1]; y <= c1[1]; ++y)
          for (int x = c0[0]; x <= c1[0]; ++x) {
            const int cc[3] = {x, y, z};
            double gap = 0.0;
            for (int a = 0; a < 3; ++a) {
              const double ga = std::max(bl[a] - (double)(cc[a] + 1), (double)cc[a] - bh[a]);
              gap = std::max(gap, ga);
            }
            double& r = rc[(size_t)cell(x, y, z)];
            r = std::min(r, gap);
          }
    }
    unsigned char* q = blob + bytes;
    for (int c = 0; c < C; ++c) {
      const double v = (rc[c] - KP_BP_CLEAR_MARGIN) * 16.0;
      q[c] = v >= 1.0 ? (unsigned char)std::min(255.0, std::floor(v)) : 0;
    }
    std::memset(q + C, 0, round16((size_t)C) - (size_t)C);
    P.bp_clear_off = (int32_t)bytes;
    bytes += round16((size_t)C);
  }
  P.n_boxes_pad = pad;
  P.bp_n_ids = start[C];
  P.blob_bytes = (int32_t)bytes;
  for (int a = 0; a < 3; ++a) {
    P.bp_g[a] = g[a];
    P.bp_scale[a] = scale[a];
    P.bp_last[a] = (float)(g[a] - 1);
  }
  P.bp_start_off = (int32_t)start_off;
  P.bp_ids_off = (int32_t)ids_off;
  return bytes;
}

// Closed boxes need lo <= hi on every axis and no NaN.
const char* check_boxes(const float* boxes, int nb) {
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      const float lo = boxes[(size_t)b * 6 + a], hi = boxes[(size_t)b * 6 + 3 + a];
      if (std::isnan(lo) || std::isnan(hi)) return "NaN in a box";
      if (!(lo <= hi)) return "box with lo > hi";
    }
  return nullptr;
}

// Free-space-obeying decomposition (Sec. IV-B) as a kd-tree over the
// workspace whose planes are obstacle faces.  A cell is split while a face
// of a box meeting its interior lies strictly inside it: on the axis with
// the most distinct such coordinates (the lowest on a tie), at the lower
// median.  Nodes and leaves are numbered depth first, the side below the
// plane first.  A child sees only the boxes that met its parent.
struct KdTree {
  std::vector<int32_t> node;
  std::vector<float> split;
  std::vector<float> lo, hi;  // [leaves][3]
};

bool kd_cell(KdTree& T, const float* fb, const std::vector<int>& ids, const float lo[3],
             const float hi[3], int depth) {
  const size_t me = T.node.size();
  T.node.push_back(0);
  T.split.push_back(0.0f);
  std::vector<int> in;
  for (int b : ids) {
    const float* bx = fb + (size_t)b * 8;
    if (bx[0] < hi[0] && bx[4] > lo[0] && bx[1] < hi[1] && bx[5] > lo[1] && bx[2] < hi[2] &&
        bx[6] > lo[2])
      in.push_back(b);
  }
  int axis = -1;
  size_t most = 0;
  float at = 0.0f;
  std::vector<float> c;
  for (int a = 0; a < 3; ++a) {
    c.clear();
    for (int b : in)
      for (int s = 0; s < 2; ++s) {
        const float f = fb[(size_t)b * 8 + 4 * s + a];
        if (f > lo[a] && f < hi[a]) c.push_back(f);
      }
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    if (c.size() > most) {
      most = c.size();
      axis = a;
      at = c[(c.size() - 1) / 2];
    }
  }
  if (axis < 0) {  // no face crosses the cell: a leaf
    const size_t leaf = T.lo.size() / 3;
    if (leaf >= (size_t)KP_FSO_MAX_LEAVES) return false;
    T.node[me] = (int32_t)((3u << 30) | (uint32_t)leaf);
    T.lo.insert(T.lo.end(), lo, lo + 3);
    T.hi.insert(T.hi.end(), hi, hi + 3);
    return true;
  }
  if (depth >= KP_FSO_MAX_DEPTH) return false;
  T.split[me] = at;
  float clo[3] = {lo[0], lo[1], lo[2]}, chi[3] = {hi[0], hi[1], hi[2]};
  chi[axis] = at;
  if (!kd_cell(T, fb, in, lo, chi, depth + 1)) return false;
  T.node[me] = (int32_t)(((uint32_t)axis << 30) | (uint32_t)T.node.size());
  clo[axis] = at;
  return kd_cell(T, fb, in, clo, hi, depth + 1);
}

// Builds the tree over the padded blob boxes and writes the arena image of
// its slices to 'host' (kd_node, kd_split, leaf_box, region_vol at their
// offsets relative to lay.kd_node).  Returns the leaf count, 0 past the
// limits.
int build_kd(unsigned char* host, const float* fb, int nb, const kp_workspace& ws,
             const Layout& lay, int* n_nodes) {
  KdTree T;
  std::vector<int> all((size_t)nb);
  for (int b = 0; b < nb; ++b) all[(size_t)b] = b;
  if (!kd_cell(T, fb, all, ws.lo, ws.hi, 0)) return 0;
  const int leaves = (int)(T.lo.size() / 3);
  *n_nodes = (int)T.node.size();
  int32_t* node = reinterpret_cast<int32_t*>(host);
  float* split = reinterpret_cast<float*>(host + (lay.kd_split - lay.kd_node));
  float* box = reinterpret_cast<float*>(host + (lay.leaf_box - lay.kd_node));
  double* vol = reinterpret_cast<double*>(host + (lay.region_vol - lay.kd_node));
  for (size_t i = 0; i < T.node.size(); ++i) {
    node[i] = T.node[i];
    split[i] = T.split[i];
  }
  for (int r = 0; r < leaves; ++r) {
    float* o = box + (size_t)r * 8;
    for (int a = 0; a < 3; ++a) {
      const float l = T.lo[(size_t)r * 3 + a], h = T.hi[(size_t)r * 3 + a];
      o[a] = l;
      o[4 + a] = (float)((double)ws.sub[a] / ((double)h - (double)l));
    }
    o[3] = o[7] = 0.0f;
    const float* l = &T.lo[(size_t)r * 3];
    const float* h = &T.hi[(size_t)r * 3];
    vol[r] = ((double)h[0] - (double)l[0]) * ((double)h[1] - (double)l[1]) *
             ((double)h[2] - (double)l[2]);
  }
  return leaves;
}

kp_status configure_launch(kp_ctx* ctx);

// Region chunks of the Score sums (Eq. 5): a power of two, at most one per
// block, chunks of at least 32 regions (one per lane of the warp that
// scores them), at most 1024 chunks.  Any power of two gives the same
// pairwise tree.
int region_chunks(int blocks, int R_pad) {
  int nch = 1;
  while (nch * 2 <= blocks && nch * 2 * 32 <= R_pad && nch * 2 <= 1024) nch *= 2;
  return nch;
}

kp_status upload_boxes(kp_ctx* ctx, const kp_obstacles* obs) {
  const int nb = obs ? obs->n_boxes : 0;
  if (nb < 0 || nb > ctx->n_boxes_cap) return fail(ctx, KP_ERR_ARG, "box count above capacity");
  if (nb > 0 && !obs->boxes) return fail(ctx, KP_ERR_ARG, "null boxes");
  if (const char* m = check_boxes(nb > 0 ? obs->boxes : nullptr, nb)) return fail(ctx, KP_ERR_ARG, "%s", m);
  // build the blob (and the kd-tree) in pinned host memory first; nothing
  // of the context changes unless both succeed
  const Layout& L = ctx->lay;
  const size_t kd_bytes = ctx->dims.fso ? L.total - L.kd_node : 0;
  kp_status ps = ensure_pinned(ctx, (size_t)KP_BLOB_BYTES + (ctx->dims.fso ? kKdNodes * 8 : 0) +
                                        kd_bytes + sizeof(KCtl));
  if (ps != KP_OK) return ps;
  KP_CUDA(cudaStreamSynchronize(ctx->stream));  // the staging buffer is free
  unsigned char* host = static_cast<unsigned char*>(ctx->pinned);
  KParams Pn = ctx->P;
  const size_t bytes = build_blob(host, nb > 0 ? obs->boxes : nullptr, nb, ctx->ws, Pn);
  unsigned char* kd = host + (size_t)KP_BLOB_BYTES + kKdNodes * 8;
  int leaves = 0, n_nodes = 0, blob_kd = 0;
  if (ctx->dims.fso) {
    leaves = build_kd(kd, reinterpret_cast<const float*>(host), nb, ctx->ws, L, &n_nodes);
    if (leaves == 0)
      return fail(ctx, KP_ERR_ARG, "kd-tree decomposition above %d leaves or depth %d",
                  KP_FSO_MAX_LEAVES, KP_FSO_MAX_DEPTH);
    // the compact copy (codes, then splits) right after the blob
    const size_t at = round16(bytes);
    std::memset(host + bytes, 0, at - bytes);
    std::memcpy(host + at, kd, (size_t)n_nodes * 4);
    std::memcpy(host + at + (size_t)n_nodes * 4, kd + (L.kd_split - L.kd_node), (size_t)n_nodes * 4);
    blob_kd = (int)round16(at + (size_t)n_nodes * 8);
  }
  // commit
  KP_CUDA(cudaMemcpyAsync(ctx->arena + L.boxes, host, blob_kd > 0 ? (size_t)blob_kd : bytes,
                          cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->dims.fso)
    KP_CUDA(cudaMemcpyAsync(ctx->arena + L.kd_node, kd, kd_bytes, cudaMemcpyHostToDevice,
                            ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->P = Pn;
  ctx->blob_base = (int)bytes;
  ctx->blob_kd = blob_kd;
  if (ctx->dims.fso) {
    ctx->P.kd_n = n_nodes;
    Dims& d = ctx->dims;
    d.R = leaves;
    d.R_pad = 1;
    while (d.R_pad < d.R) d.R_pad *= 2;
    d.n_sub = (size_t)d.R * (size_t)d.n_sub_per;
    ctx->P.R = d.R;
    ctx->P.R_pad = d.R_pad;
  }
  ctx->dims.boxes_pad = ctx->P.n_boxes_pad;
  ctx->have_tree = false;
  return configure_launch(ctx);
}

kp_status configure_launch(kp_ctx* ctx) {
  const Dims& d = ctx->dims;
  ctx->P.blob_bytes = ctx->blob_base;
  ctx->P.kd_smem_off = -1;
  // shared memory: boxes + the double scratch of the region-score sums (a
  // chunk's scores, then the chunk sums) + the network tile (learned form)
  auto grids = [&](int sd) -> kp_status {
    ctx->P.sd_bytes = sd * 8;
    ctx->smem = (size_t)ctx->P.blob_bytes + (size_t)sd * 8 +
                (ctx->P.features_on ? (size_t)MLP_LOOP_TILE_SMEM : 0);
    for (int log = 0; log < 2; ++log) {
      int bps = 0;
      KP_CUDA(occupancy(d.sys, log != 0, ctx->smem, &bps));
      if (bps < 1) return fail(ctx, KP_ERR_ARG, "loop kernel cannot be resident");
      int g = bps * ctx->num_sms;
      if (g > KP_MAX_GRID) g = KP_MAX_GRID;
      if (ctx->grid_limit > 0 && g > ctx->grid_limit) g = ctx->grid_limit;
      ctx->grid[log] = g;
    }
    return KP_OK;
  };
  // first with room for any chunking (chunks of at least R_pad / 1024
  // regions, at most 1024 chunk sums) ...
  const int min_ch = d.R_pad / (d.R_pad < 1024 ? d.R_pad : 1024);
  kp_status s = grids(min_ch > 1024 ? min_ch : 1024);
  if (s != KP_OK) return s;
  // region chunks: a power of two <= the smaller grid, <= R_pad, <= 1024
  const int gmin = ctx->grid[0] < ctx->grid[1] ? ctx->grid[0] : ctx->grid[1];
  const int nch = region_chunks(gmin, d.R_pad);
  ctx->P.nch = nch;
  // ... then with the scratch this chunking needs (smaller shared memory
  // never lowers the grid, so nch stays at most the grid)
  const int need = d.R_pad / nch > nch ? d.R_pad / nch : nch;
  s = grids(need);
  if (s != KP_OK || ctx->blob_kd == 0) return s;
  // the kd-tree goes into shared memory with the blob when that keeps the
  // resident blocks (it is read at every binning)
  const size_t smem_kd = ctx->smem + (size_t)(ctx->blob_kd - ctx->blob_base);
  for (int log = 0; log < 2; ++log) {
    int bps = 0;
    KP_CUDA(occupancy(d.sys, log != 0, smem_kd, &bps));
    int g = bps * ctx->num_sms;
    if (g > KP_MAX_GRID) g = KP_MAX_GRID;
    if (ctx->grid_limit > 0 && g > ctx->grid_limit) g = ctx->grid_limit;
    if (g < ctx->grid[log]) return KP_OK;
  }
  ctx->P.blob_bytes = ctx->blob_kd;
  ctx->P.kd_smem_off = (int)round16((size_t)ctx->blob_base);
  ctx->smem = smem_kd;
  return KP_OK;
}

// Algorithm 1's initialisation: one launch clears the tables and writes
// the root (kp_reset_kernel).
kp_status enqueue_reset(kp_ctx* ctx, const float* x_init) {
  for (int i = 0; i < ctx->dims.D; ++i)
    if (std::isnan(x_init[i])) return fail(ctx, KP_ERR_ARG, "NaN in x_init");
  RootState root{};
  for (int i = 0; i < ctx->dims.D; ++i) root.x[i] = x_init[i];
  KParams P = params_now(ctx);
  KP_CUDA(launch_reset(ctx, P, root));
  ctx->have_tree = true;
  return KP_OK;
}

// Launch constants and arena slices of a validated problem.
void fill_params(KParams& P, const Dims& d, const Layout& lay, const kp_system* sys,
                 const kp_workspace* ws, const kp_params* prm, char* A) {
  P = KParams{};
  P.sys = d.sys;
  P.dt = sys->dt;
  P.dt_sixth = sys->dt / 6.0f;  // the same correctly rounded FP32 division the device made
  P.k_min = sys->k_min;
  P.k_span = (uint32_t)(sys->k_max - sys->k_min + 1);
  for (int i = 0; i < 12; ++i) {
    P.x_lo[i] = i < d.D ? sys->x_lo[i] : -INFINITY;
    P.x_hi[i] = i < d.D ? sys->x_hi[i] : INFINITY;
  }
  for (int i = 0; i < 4; ++i) {
    P.u_lo[i] = sys->u_lo[i];
    P.u_scale[i] = sys->u_hi[i] - sys->u_lo[i];
  }
  for (int i = 0; i < 16; ++i) P.phys[i] = sys->phys[i];
  if (d.sys == KP_SYS_QUAD)
    for (int i = 0; i < 4; ++i) {
      const float q = sys->phys[i == 0 ? 0 : 3 + i];  // m, Ixx, Iyy, Izz
      P.recip[i] = q != 0.0f ? 1.0f / q : 0.0f;
    }
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    P.ws_lo[a] = ws->lo[a];
    P.n_fine[a] = ws->grid[a] * ws->sub[a];
    P.n_fine_last[a] = (float)(P.n_fine[a] - 1);
    P.sub_shift[a] = -1;
    for (int b = 0; b < 16; ++b)
      if (ws->sub[a] == (1 << b)) P.sub_shift[a] = b;
    P.fine_scale[a] = (float)((double)P.n_fine[a] / ((double)ws->hi[a] - (double)ws->lo[a]));
    P.sub[a] = ws->sub[a];
    P.grid[a] = ws->grid[a];
    vol *= ((double)ws->hi[a] - (double)ws->lo[a]) / (double)ws->grid[a];
  }
  P.speed_bins = ws->speed_bins;
  // further state dimensions of the region index (cells per unit of the
  // dimension; an unbounded one is binned over [-pi, pi) after wrapping)
  for (int dd = 0; dd < 12; ++dd) {
    const int n = dd >= 3 && dd < d.D && ws->state_grid[dd] > 1 ? ws->state_grid[dd] : 1;
    P.state_grid[dd] = n;
    P.state_scale[dd] = 0.0f;
    if (n > 1) {
      const bool bounded = std::isfinite(sys->x_lo[dd]) && std::isfinite(sys->x_hi[dd]);
      P.state_scale[dd] =
          bounded ? (float)((double)n / ((double)sys->x_hi[dd] - (double)sys->x_lo[dd]))
                  : (float)((double)n / (2.0 * 3.14159265358979323846));
      P.state_wrap[dd] = bounded ? 0 : 1;
    }
  }
  P.speed_scale = ws->speed_bins > 1 ? (float)((double)ws->speed_bins / (double)ws->speed_hi) : 0.0f;
  P.n_sub_per = d.n_sub_per;
  P.R = d.R;
  P.R_pad = d.R_pad;
  P.t_e = d.t_e;
  P.lambda_max = prm->lambda_max;
  P.delta = prm->delta;
  P.eps = prm->eps;
  P.vol = vol;
  P.fso = d.fso;
  P.kd_smem_off = -1;
  P.bp_clear_off = -1;
  if (d.fso) {
    P.kd_node = reinterpret_cast<const int32_t*>(A + lay.kd_node);
    P.kd_split = reinterpret_cast<const float*>(A + lay.kd_split);
    P.leaf_box = reinterpret_cast<const float4*>(A + lay.leaf_box);
    P.region_vol = reinterpret_cast<const double*>(A + lay.region_vol);
  }
  P.boxes = reinterpret_cast<const float*>(A + lay.boxes);
  P.st = reinterpret_cast<float*>(A + lay.st);
  P.parent = reinterpret_cast<int32_t*>(A + lay.parent);
  P.ctrl = reinterpret_cast<float*>(A + lay.ctrl);
  P.steps = reinterpret_cast<uint8_t*>(A + lay.steps);
  P.region = reinterpret_cast<int32_t*>(A + lay.region);
  P.node_sub = reinterpret_cast<int32_t*>(A + lay.sub);
  P.in_ve = reinterpret_cast<uint8_t*>(A + lay.in_ve);
  P.cs = reinterpret_cast<int32_t*>(A + lay.cs);
  P.xs = reinterpret_cast<float*>(A + lay.xs);
  P.acc_key = reinterpret_cast<uint32_t*>(A + lay.acc_key);
  P.flags = reinterpret_cast<uint8_t*>(A + lay.flags);
  P.n_valid = reinterpret_cast<uint32_t*>(A + lay.n_valid);
  P.n_invalid = reinterpret_cast<uint32_t*>(A + lay.n_invalid);
  P.cov = reinterpret_cast<uint32_t*>(A + lay.cov);
  P.avail = reinterpret_cast<uint8_t*>(A + lay.avail);
  P.visited = reinterpret_cast<uint8_t*>(A + lay.visited);
  P.claim = reinterpret_cast<uint32_t*>(A + lay.claim);
  P.score = reinterpret_cast<double*>(A + lay.score);
  P.thr = reinterpret_cast<uint64_t*>(A + lay.thr);
  P.ve = reinterpret_cast<int32_t*>(A + lay.ve);
  P.blk_a = reinterpret_cast<uint32_t*>(A + lay.blk_a);
  P.blk_b = reinterpret_cast<uint32_t*>(A + lay.blk_b);
  P.chunk_sum = reinterpret_cast<double*>(A + lay.chunk_sum);
  P.ctl = reinterpret_cast<KCtl*>(A + lay.ctl);
  P.stats = reinterpret_cast<KStats*>(A + lay.stats);
  P.stats_cap = kStatsCap;
  P.traj = reinterpret_cast<float*>(A + lay.traj);
  P.feat = reinterpret_cast<uint16_t*>(A + lay.feat);
  P.net_raw = reinterpret_cast<float*>(A + lay.net_raw);
  for (int i = 0; i < 6; ++i) {
    const float lo = i < d.D ? sys->x_lo[i] : 0.0f, hi = i < d.D ? sys->x_hi[i] : 0.0f;
    P.feat_scale[i] =
        std::isfinite(lo) && std::isfinite(hi) && hi > lo ? (float)(2.0 / ((double)hi - (double)lo)) : 0.0f;
  }
}

kp_status check_launch(kp_ctx* ctx, const KCtl& h) {
  if (h.err == KP_DEV_ERR_TIMEOUT)
    return fail(ctx, KP_ERR_TIMEOUT, "device wait exceeded %llu ns (site %d)",
                (unsigned long long)ctx->wait_ns, h.err_where);
  if (h.err == KP_DEV_ERR_REPLAY)
    return fail(ctx, KP_ERR_STATE, "appended sample differs from its first derivation (site %d)",
                h.err_where);
  if (h.err == KP_DEV_ERR_BOUNDS)
    return fail(ctx, KP_ERR_CUDA, "array index out of range (site %d)", h.err_where);
  if (h.err != 0) return fail(ctx, KP_ERR_CUDA, "device error %d", h.err);
  return KP_OK;
}

}  // namespace

extern "C" {

size_t kp_required_bytes(const kp_system* sys, const kp_workspace* ws, int32_t n_boxes,
                         const kp_params* prm) {
  Dims d{};
  if (check_inputs(sys, ws, n_boxes, prm, &d)) return 0;
  return make_layout(d).total;
}

kp_status kp_create(const kp_system* sys, const kp_workspace* ws, const kp_obstacles* obs,
                    const kp_params* prm, void* dev_arena, size_t arena_bytes, void* cuda_stream,
                    kp_ctx** out) {
  if (!out) return KP_ERR_ARG;
  *out = nullptr;
  Dims d{};
  const int nb = obs ? obs->n_boxes : 0;
  if (check_inputs(sys, ws, nb, prm, &d)) return KP_ERR_ARG;
  if (!dev_arena || ((uintptr_t)dev_arena & 255u)) return KP_ERR_ARG;
  const Layout lay = make_layout(d);
  if (arena_bytes < lay.total) return KP_ERR_OOM;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, dev_arena) != cudaSuccess ||
      attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return KP_ERR_ARG;
  }

  kp_ctx* ctx = new (std::nothrow) kp_ctx();
  if (!ctx) return KP_ERR_OOM;
  ctx->dims = d;
  ctx->lay = lay;
  ctx->sys = *sys;
  ctx->ws = *ws;
  ctx->prm = *prm;
  ctx->n_boxes_cap = KP_MAX_BOXES;
  ctx->arena = static_cast<char*>(dev_arena);
  ctx->arena_bytes = arena_bytes;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->device = attr.device;
  ctx->seed = prm->seed;
  ctx->wait_ns = 2000000000ull;
  ctx->goal = kp_goal{{0, 0, 0}, 0};
  kp_status s = KP_OK;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return KP_ERR_CUDA;
    }
  }

  fill_params(ctx->P, d, lay, sys, ws, prm, ctx->arena);
  char* A = ctx->arena;

  {
    cudaError_t e = cudaMemsetAsync(A + lay.ctl, 0, sizeof(KCtl), ctx->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_loop0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_loop1);
    if (e != cudaSuccess) s = fail(ctx, KP_ERR_CUDA, "create: %s", cudaGetErrorString(e));
  }
  if (s == KP_OK) s = upload_boxes(ctx, obs);
  if (s != KP_OK) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->ev_loop0) cudaEventDestroy(ctx->ev_loop0);
    if (ctx->ev_loop1) cudaEventDestroy(ctx->ev_loop1);
    delete ctx;
    return s;
  }
  *out = ctx;
  return KP_OK;
}

kp_status kp_set_obstacles(kp_ctx* ctx, const kp_obstacles* obs) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  return upload_boxes(ctx, obs);
}

kp_status kp_reset(kp_ctx* ctx, const float* x_init, const kp_goal* goal, uint64_t seed) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!x_init || !goal) return fail(ctx, KP_ERR_ARG, "null argument");
  if (!(goal->radius >= 0.0f) || std::isnan(goal->center[0]) || std::isnan(goal->center[1]) ||
      std::isnan(goal->center[2]))
    return fail(ctx, KP_ERR_ARG, "bad goal");
  ctx->goal = *goal;
  ctx->seed = seed;
  s = enqueue_reset(ctx, x_init);
  if (s != KP_OK) return s;
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  if (h.state == KP_DEV_BAD_ROOT) {
    ctx->have_tree = false;
    return fail(ctx, KP_ERR_ARG, "x_init is not a valid state");
  }
  return KP_OK;
}

kp_status kp_expand_step(kp_ctx* ctx, int32_t n_iters, kp_iter_stats* out, int32_t* n_run) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (n_run) *n_run = 0;
  if (!ctx->have_tree) return fail(ctx, KP_ERR_STATE, "no tree: call kp_reset first");
  if (n_iters < 1 || n_iters > kStatsCap) return fail(ctx, KP_ERR_ARG, "n_iters out of range");
  KParams P = params_now(ctx);
  KP_CUDA(launch_loop(ctx, P, n_iters, 0));
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  s = check_launch(ctx, h);
  if (s != KP_OK) return s;
  if (n_run) *n_run = h.n_run;
  if (out && h.n_run > 0) {
    static_assert(sizeof(KStats) == sizeof(kp_iter_stats), "stats layout");
    KP_CUDA(cudaMemcpyAsync(out, ctx->arena + ctx->lay.stats, sizeof(KStats) * h.n_run,
                            cudaMemcpyDeviceToHost, ctx->stream));
    KP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return KP_OK;
}

kp_status kp_plan_async(kp_ctx* ctx, const float* x_init, const kp_goal* goal,
                        const kp_budget* budget, int32_t traj_capacity) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!x_init || !goal || !budget) return fail(ctx, KP_ERR_ARG, "null argument");
  if (budget->max_iters < 1) return fail(ctx, KP_ERR_ARG, "max_iters must be >= 1");
  if (traj_capacity < 0) return fail(ctx, KP_ERR_ARG, "negative capacity");
  if (!(goal->radius >= 0.0f) || std::isnan(goal->center[0]) || std::isnan(goal->center[1]) ||
      std::isnan(goal->center[2]))
    return fail(ctx, KP_ERR_ARG, "bad goal");
  const int rows = traj_capacity < KP_TRAJ_ROWS ? traj_capacity : KP_TRAJ_ROWS;
  const size_t traj_bytes = (size_t)rows * 17 * 4;
  // every copy through the staging buffer completes before its call
  // returns, so it is free here
  if (ctx->plan_pending) return fail(ctx, KP_ERR_STATE, "kp_plan_result not called");
  s = ensure_pinned(ctx, sizeof(KCtl) + traj_bytes);
  if (s != KP_OK) return s;
  for (int i = 0; i < ctx->dims.D; ++i)
    if (std::isnan(x_init[i])) return fail(ctx, KP_ERR_ARG, "NaN in x_init");
  ctx->goal = *goal;
  RootState root{};
  for (int i = 0; i < ctx->dims.D; ++i) root.x[i] = x_init[i];
  KParams P = params_now(ctx);
  const uint64_t max_ns = budget->max_ms > 0.0 ? (uint64_t)(budget->max_ms * 1e6) : 0ull;
  // one launch: initialisation, the passes, the chain
  KP_CUDA(launch_loop(ctx, P, budget->max_iters, max_ns, root, KP_LOOP_RESET | KP_LOOP_EXTRACT));
  ctx->have_tree = true;
  ctx->plan_pending = true;
  ctx->plan_rows = rows;
  return KP_OK;
}

kp_status kp_plan_result(kp_ctx* ctx, kp_traj* traj) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!traj) return fail(ctx, KP_ERR_ARG, "null argument");
  if (!ctx->plan_pending) return fail(ctx, KP_ERR_STATE, "no kp_plan_async pending");
  const int rows = ctx->plan_rows < traj->capacity ? ctx->plan_rows : traj->capacity;
  if (rows > 0 && (!traj->states || !traj->ctrls || !traj->steps))
    return fail(ctx, KP_ERR_ARG, "bad trajectory buffers");
  ctx->plan_pending = false;
  // header and the first rows in one round trip; longer chains in a second
  const int first = rows < kFirstRows ? rows : kFirstRows;
  char* pin = static_cast<char*>(ctx->pinned);
  float* prow = reinterpret_cast<float*>(pin + sizeof(KCtl));
  KP_CUDA(cudaMemcpyAsync(pin, ctx->arena + ctx->lay.ctl, sizeof(KCtl), cudaMemcpyDeviceToHost,
                          ctx->stream));
  if (first > 0)
    KP_CUDA(cudaMemcpyAsync(prow, ctx->arena + ctx->lay.traj, (size_t)first * 17 * 4,
                            cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  KCtl h;
  std::memcpy(&h, pin, sizeof(KCtl));
  if (h.state == KP_DEV_SOLVED && h.n_edges > first && h.n_edges <= rows) {
    KP_CUDA(cudaMemcpyAsync(prow + (size_t)first * 17,
                            ctx->arena + ctx->lay.traj + (size_t)first * 17 * 4,
                            (size_t)(h.n_edges - first) * 17 * 4, cudaMemcpyDeviceToHost,
                            ctx->stream));
    KP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  s = check_launch(ctx, h);
  if (s != KP_OK) return s;
  if (h.state == KP_DEV_BAD_ROOT) {
    ctx->have_tree = false;
    return fail(ctx, KP_ERR_ARG, "x_init is not a valid state");
  }
  traj->n_edges = 0;
  if (h.state != KP_DEV_SOLVED || h.n_edges < 0) return KP_NO_SOLUTION;
  traj->n_edges = h.n_edges;
  if (h.n_edges > rows) return fail(ctx, KP_ERR_ARG, "trajectory needs %d rows", h.n_edges);
  const float* src = prow;
  for (int e = 0; e < h.n_edges; ++e) {
    std::memcpy(traj->states + (size_t)e * 12, src + (size_t)e * 17, 12 * 4);
    std::memcpy(traj->ctrls + (size_t)e * 4, src + (size_t)e * 17 + 12, 4 * 4);
    traj->steps[e] = (int32_t)src[(size_t)e * 17 + 16];
  }
  return KP_OK;
}

kp_status kp_plan(kp_ctx* ctx, const float* x_init, const kp_goal* goal, const kp_budget* budget,
                  kp_traj* traj) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!traj || traj->capacity < 0) return fail(ctx, KP_ERR_ARG, "bad trajectory");
  s = kp_plan_async(ctx, x_init, goal, budget, traj->capacity);
  if (s != KP_OK) return s;
  return kp_plan_result(ctx, traj);
}

kp_status kp_get_info(kp_ctx* ctx, kp_info* out) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!out) return KP_ERR_ARG;
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  out->n_nodes = ctx->have_tree ? h.n_nodes : 0;
  out->n_ve = ctx->have_tree ? h.n_ve : 0;
  out->iteration = h.iteration;
  out->goal_node = h.goal_node == KP_NO_GOAL ? -1 : h.goal_node;
  out->state = ctx->have_tree ? (h.state == KP_DEV_BAD_ROOT ? -1 : h.state) : -1;
  out->n_regions = ctx->dims.R;
  out->n_subregions = (int32_t)ctx->dims.n_sub;
  out->state_dim = ctx->dims.D;
  out->control_dim = ctx->dims.N;
  out->n_samples = ctx->have_tree ? (int64_t)h.tot_samples : 0;
  out->n_steps = ctx->have_tree ? (int64_t)h.tot_steps : 0;
  out->n_hull_checks = ctx->have_tree ? (int64_t)h.tot_hull : 0;
  out->n_box_tests = ctx->have_tree ? (int64_t)h.tot_box_tests : 0;
  out->bp_cells = ctx->P.bp_g[0] * ctx->P.bp_g[1] * ctx->P.bp_g[2];
  for (int a = 0; a < 3; ++a) out->bp_grid[a] = ctx->P.bp_g[a];
  out->n_key_batches = ctx->have_tree ? (int64_t)h.tot_batches : 0;
  out->n_lane_refills = ctx->have_tree ? (int64_t)h.tot_refills : 0;
  out->n_boxes = ctx->P.n_boxes_pad;
  out->grid_blocks = ctx->grid[ctx->log_on ? 1 : 0];
  return KP_OK;
}

kp_status kp_export_tree(kp_ctx* ctx, kp_tree_view* v) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!v) return KP_ERR_ARG;
  if (!ctx->have_tree) return fail(ctx, KP_ERR_STATE, "no tree");
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  const int n = h.n_nodes, D = ctx->dims.D, N = ctx->dims.N, te = ctx->dims.t_e;
  v->n_nodes = n;
  v->iteration = h.iteration;
  if (n > v->capacity) return fail(ctx, KP_ERR_ARG, "view holds %d nodes, tree has %d", v->capacity, n);
  const Layout& L = ctx->lay;
  auto d2h = [&](void* dst, size_t off, size_t bytes) -> kp_status {
    if (!dst || !bytes) return KP_OK;
    KP_CUDA(cudaMemcpyAsync(dst, ctx->arena + off, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return KP_OK;
  };
  std::vector<float> st((size_t)D * n), ct((size_t)N * n);
  std::vector<uint8_t> steps(n);
  for (int i = 0; i < D; ++i)
    if ((s = d2h(st.data() + (size_t)i * n, L.st + (size_t)i * te * 4, (size_t)n * 4)) != KP_OK) return s;
  for (int i = 0; i < N; ++i)
    if ((s = d2h(ct.data() + (size_t)i * n, L.ctrl + (size_t)i * te * 4, (size_t)n * 4)) != KP_OK) return s;
  if ((s = d2h(steps.data(), L.steps, n)) != KP_OK) return s;
  if ((s = d2h(v->parent, L.parent, (size_t)n * 4)) != KP_OK) return s;
  if ((s = d2h(v->region, L.region, (size_t)n * 4)) != KP_OK) return s;
  if ((s = d2h(v->sub, L.sub, (size_t)n * 4)) != KP_OK) return s;
  if ((s = d2h(v->in_ve, L.in_ve, (size_t)n)) != KP_OK) return s;
  const size_t R = ctx->dims.R;
  if ((s = d2h(v->n_valid, L.n_valid, R * 4)) != KP_OK) return s;
  if ((s = d2h(v->n_invalid, L.n_invalid, R * 4)) != KP_OK) return s;
  if ((s = d2h(v->cov, L.cov, R * 4)) != KP_OK) return s;
  if ((s = d2h(v->avail, L.avail, R)) != KP_OK) return s;
  if ((s = d2h(v->thr, L.thr, R * 8)) != KP_OK) return s;
  if ((s = d2h(v->visited, L.visited, ctx->dims.n_sub)) != KP_OK) return s;
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int u = 0; u < n; ++u) {
    if (v->state)
      for (int i = 0; i < 12; ++i) v->state[(size_t)u * 12 + i] = i < D ? st[(size_t)i * n + u] : 0.0f;
    if (v->ctrl)
      for (int i = 0; i < 4; ++i) v->ctrl[(size_t)u * 4 + i] = i < N ? ct[(size_t)i * n + u] : 0.0f;
    if (v->steps) v->steps[u] = steps[u];
  }
  return KP_OK;
}

kp_status kp_import_tree(kp_ctx* ctx, const kp_tree_view* v) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!v || !v->state || !v->parent || !v->ctrl || !v->steps || !v->region || !v->sub ||
      !v->in_ve || !v->n_valid || !v->n_invalid || !v->thr || !v->visited)
    return fail(ctx, KP_ERR_ARG, "null array in tree view");
  const int n = v->n_nodes, D = ctx->dims.D, N = ctx->dims.N, te = ctx->dims.t_e;
  if (n < 1 || n > te || v->iteration < 0) return fail(ctx, KP_ERR_ARG, "bad node count");
  const int R = ctx->dims.R;
  for (int u = 0; u < n; ++u) {
    if (v->region[u] < 0 || v->region[u] >= R || v->sub[u] < 0 ||
        (size_t)v->sub[u] >= ctx->dims.n_sub || v->parent[u] >= u || (u > 0 && v->parent[u] < 0) ||
        v->steps[u] < 0 || v->steps[u] > 255)
      return fail(ctx, KP_ERR_ARG, "bad node %d", u);
  }
  const Layout& L = ctx->lay;
  std::vector<float> st((size_t)D * n), ct((size_t)N * n);
  std::vector<uint8_t> steps(n), inve(n);
  for (int u = 0; u < n; ++u) {
    for (int i = 0; i < D; ++i) st[(size_t)i * n + u] = v->state[(size_t)u * 12 + i];
    for (int i = 0; i < N; ++i) ct[(size_t)i * n + u] = v->ctrl[(size_t)u * 4 + i];
    steps[u] = (uint8_t)v->steps[u];
    inve[u] = v->in_ve[u] ? 1 : 0;
  }
  auto h2d = [&](size_t off, const void* src, size_t bytes) -> kp_status {
    KP_CUDA(cudaMemcpyAsync(ctx->arena + off, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return KP_OK;
  };
  for (int i = 0; i < D; ++i)
    if ((s = h2d(L.st + (size_t)i * te * 4, st.data() + (size_t)i * n, (size_t)n * 4)) != KP_OK) return s;
  for (int i = 0; i < N; ++i)
    if ((s = h2d(L.ctrl + (size_t)i * te * 4, ct.data() + (size_t)i * n, (size_t)n * 4)) != KP_OK) return s;
  if ((s = h2d(L.steps, steps.data(), n)) != KP_OK) return s;
  if ((s = h2d(L.in_ve, inve.data(), n)) != KP_OK) return s;
  if ((s = h2d(L.parent, v->parent, (size_t)n * 4)) != KP_OK) return s;
  if ((s = h2d(L.region, v->region, (size_t)n * 4)) != KP_OK) return s;
  if ((s = h2d(L.sub, v->sub, (size_t)n * 4)) != KP_OK) return s;
  if ((s = h2d(L.n_valid, v->n_valid, (size_t)R * 4)) != KP_OK) return s;
  if ((s = h2d(L.n_invalid, v->n_invalid, (size_t)R * 4)) != KP_OK) return s;
  if ((s = h2d(L.thr, v->thr, (size_t)R * 8)) != KP_OK) return s;
  if ((s = h2d(L.visited, v->visited, ctx->dims.n_sub)) != KP_OK) return s;
  KP_CUDA(cudaMemsetAsync(ctx->arena + L.claim, 0xff, ctx->dims.n_sub * 4, ctx->stream));
  KParams P = params_now(ctx);
  kp_import_regions_kernel<<<(R + 255) / 256 < 1024 ? (R + 255) / 256 : 1024, 256, 0, ctx->stream>>>(P);
  KP_CUDA(cudaGetLastError());
  kp_import_avail_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, ctx->stream>>>(P, n);
  KP_CUDA(cudaGetLastError());
  KCtl h{};
  h.n_nodes = n;
  h.n_ve = 0;
  h.iteration = v->iteration;
  h.goal_node = KP_NO_GOAL;
  h.state = KP_DEV_RUNNING;
  // the barrier word starts at 0 (no launch is in flight)
  kp_status rs = ensure_pinned(ctx, sizeof(KCtl));
  if (rs != KP_OK) return rs;
  std::memcpy(ctx->pinned, &h, sizeof(KCtl));
  KP_CUDA(cudaMemcpyAsync(ctx->arena + L.ctl, ctx->pinned, sizeof(KCtl), cudaMemcpyHostToDevice,
                          ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->have_tree = true;
  return KP_OK;
}

kp_status kp_grow(kp_ctx* ctx, void* dev_arena, size_t arena_bytes, int32_t t_e) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!dev_arena || ((uintptr_t)dev_arena & 255u)) return fail(ctx, KP_ERR_ARG, "bad arena");
  if (ctx->plan_pending) return fail(ctx, KP_ERR_STATE, "kp_plan_result not called");
  if (t_e < ctx->dims.t_e || t_e > (1 << 28)) return fail(ctx, KP_ERR_ARG, "bad node cap");
  Dims nd = ctx->dims;
  nd.t_e = t_e;
  const Layout nl = make_layout(nd);
  if (arena_bytes < nl.total) return fail(ctx, KP_ERR_OOM, "arena too small for the new node cap");
  char* src = ctx->arena;
  char* dst = static_cast<char*>(dev_arena);
  const Layout& ol = ctx->lay;
  const Dims& od = ctx->dims;
  // the loop state, to know how many nodes to carry over
  s = ensure_pinned(ctx, sizeof(KCtl));
  if (s != KP_OK) return s;
  KP_CUDA(cudaMemcpyAsync(ctx->pinned, src + ol.ctl, sizeof(KCtl), cudaMemcpyDeviceToHost,
                          ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  KCtl h;
  std::memcpy(&h, ctx->pinned, sizeof(KCtl));
  const size_t n = ctx->have_tree ? (size_t)h.n_nodes : 0;
  auto d2d = [&](size_t dst_off, size_t src_off, size_t bytes) -> kp_status {
    if (bytes)
      KP_CUDA(cudaMemcpyAsync(dst + dst_off, src + src_off, bytes, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    return KP_OK;
  };
  // control region (loop state, barrier words; a tree that was full can
  // grow again) and the staged obstacles
  if (h.state == KP_DEV_FULL) h.state = KP_DEV_RUNNING;
  std::memcpy(ctx->pinned, &h, sizeof(KCtl));
  KP_CUDA(cudaMemcpyAsync(dst + nl.ctl, ctx->pinned, sizeof(KCtl), cudaMemcpyHostToDevice,
                          ctx->stream));
  const int blob_all = ctx->blob_kd > ctx->blob_base ? ctx->blob_kd : ctx->blob_base;
  if ((s = d2d(nl.boxes, ol.boxes, (size_t)blob_all)) != KP_OK) return s;
  if (od.fso && (s = d2d(nl.kd_node, ol.kd_node, ol.total - ol.kd_node)) != KP_OK) return s;
  // the tree: SoA rows move to the new stride
  if (n) {
    KP_CUDA(cudaMemcpy2DAsync(dst + nl.st, (size_t)nd.t_e * 4, src + ol.st, (size_t)od.t_e * 4,
                              n * 4, (size_t)od.D, cudaMemcpyDeviceToDevice, ctx->stream));
    KP_CUDA(cudaMemcpy2DAsync(dst + nl.ctrl, (size_t)nd.t_e * 4, src + ol.ctrl,
                              (size_t)od.t_e * 4, n * 4, (size_t)od.N, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    if ((s = d2d(nl.parent, ol.parent, n * 4)) != KP_OK) return s;
    if ((s = d2d(nl.steps, ol.steps, n)) != KP_OK) return s;
    if ((s = d2d(nl.region, ol.region, n * 4)) != KP_OK) return s;
    if ((s = d2d(nl.sub, ol.sub, n * 4)) != KP_OK) return s;
    if ((s = d2d(nl.in_ve, ol.in_ve, n)) != KP_OK) return s;
  }
  // decomposition tables (sizes do not depend on the node cap)
  if ((s = d2d(nl.n_valid, ol.n_valid, (size_t)od.R * 4)) != KP_OK) return s;
  if ((s = d2d(nl.n_invalid, ol.n_invalid, (size_t)od.R * 4)) != KP_OK) return s;
  if ((s = d2d(nl.cov, ol.cov, (size_t)od.R * 4)) != KP_OK) return s;
  if ((s = d2d(nl.avail, ol.avail, (size_t)od.R)) != KP_OK) return s;
  if ((s = d2d(nl.score, ol.score, (size_t)od.R * 8)) != KP_OK) return s;
  if ((s = d2d(nl.thr, ol.thr, (size_t)od.R * 8)) != KP_OK) return s;
  if ((s = d2d(nl.visited, ol.visited, od.n_sub)) != KP_OK) return s;
  if ((s = d2d(nl.claim, ol.claim, od.n_sub * 4)) != KP_OK) return s;
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  // rebind: pointers from the new layout; what the layout does not give
  // (staged obstacles, chunking, network, harvest) carries over
  const KParams old = ctx->P;
  ctx->prm.t_e = t_e;
  fill_params(ctx->P, nd, nl, &ctx->sys, &ctx->ws, &ctx->prm, dst);
  KParams& P = ctx->P;
  P.n_boxes_pad = old.n_boxes_pad;
  P.blob_bytes = old.blob_bytes;
  P.kd_n = old.kd_n;
  P.kd_smem_off = old.kd_smem_off;
  for (int a = 0; a < 3; ++a) P.bp_g[a] = old.bp_g[a];
  P.bp_start_off = old.bp_start_off;
  P.bp_ids_off = old.bp_ids_off;
  P.bp_clear_off = old.bp_clear_off;
  P.bp_n_ids = old.bp_n_ids;
  for (int a = 0; a < 3; ++a) P.bp_scale[a] = old.bp_scale[a];
  for (int a = 0; a < 3; ++a) P.bp_last[a] = old.bp_last[a];
  P.nch = old.nch;
  P.sd_bytes = old.sd_bytes;
  P.extract_cap = old.extract_cap;
  P.mlp_W1 = old.mlp_W1;
  P.mlp_b1 = old.mlp_b1;
  P.mlp_W2 = old.mlp_W2;
  P.mlp_b2 = old.mlp_b2;
  P.mlp_W3 = old.mlp_W3;
  P.mlp_b3 = old.mlp_b3;
  P.mix_thr = old.mix_thr;
  P.features_on = old.features_on;
  P.hv_feat = old.hv_feat;
  P.hv_target = old.hv_target;
  P.hv_count = old.hv_count;
  P.hv_cap = old.hv_cap;
  ctx->dims = nd;
  ctx->lay = nl;
  ctx->arena = dst;
  ctx->arena_bytes = arena_bytes;
  return configure_launch(ctx);
}

kp_status kp_resume(kp_ctx* ctx, const kp_budget* budget, kp_traj* traj) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!budget || !traj) return fail(ctx, KP_ERR_ARG, "null argument");
  if (!ctx->have_tree) return fail(ctx, KP_ERR_STATE, "no tree: call kp_reset or kp_plan first");
  if (ctx->plan_pending) return fail(ctx, KP_ERR_STATE, "kp_plan_result not called");
  if (budget->max_iters < 1) return fail(ctx, KP_ERR_ARG, "max_iters must be >= 1");
  if (traj->capacity < 0) return fail(ctx, KP_ERR_ARG, "negative capacity");
  const int rows = traj->capacity < KP_TRAJ_ROWS ? traj->capacity : KP_TRAJ_ROWS;
  s = ensure_pinned(ctx, sizeof(KCtl) + (size_t)rows * 17 * 4);
  if (s != KP_OK) return s;
  KParams P = params_now(ctx);
  const uint64_t max_ns = budget->max_ms > 0.0 ? (uint64_t)(budget->max_ms * 1e6) : 0ull;
  KP_CUDA(launch_loop(ctx, P, budget->max_iters, max_ns, RootState{}, KP_LOOP_EXTRACT));
  ctx->plan_pending = true;
  ctx->plan_rows = rows;
  return kp_plan_result(ctx, traj);
}

kp_status kp_set_sample_log(kp_ctx* ctx, const kp_sample_log* log) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!log) {
    ctx->log_on = false;
    ctx->log = KLog{};
    return KP_OK;
  }
  if (log->capacity < 0 || !log->node || !log->k || !log->uraw || !log->flags ||
      !log->fail_step || !log->region || !log->sub || !log->state)
    return fail(ctx, KP_ERR_ARG, "bad sample log");
  ctx->log = KLog{log->capacity, log->node, log->k, log->uraw, log->flags, log->fail_step,
                  log->region, log->sub, log->state};
  ctx->log_on = true;
  return KP_OK;
}

kp_status kp_set_wait_limit(kp_ctx* ctx, uint64_t ns) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (ns < 1000) return fail(ctx, KP_ERR_ARG, "wait limit below 1 us");
  ctx->wait_ns = ns;
  return KP_OK;
}

kp_status kp_set_extract_ids(kp_ctx* ctx, int32_t max_ids) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (max_ids < 0) return fail(ctx, KP_ERR_ARG, "negative id cap");
  ctx->P.extract_cap = max_ids;
  return KP_OK;
}

kp_status kp_set_grid_limit(kp_ctx* ctx, int32_t max_blocks) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (max_blocks < 0) return fail(ctx, KP_ERR_ARG, "negative grid limit");
  const int old = ctx->grid_limit;
  ctx->grid_limit = max_blocks;
  s = configure_launch(ctx);
  if (s != KP_OK) {
    ctx->grid_limit = old;
    kp_status r = configure_launch(ctx);
    return r != KP_OK ? r : s;
  }
  return KP_OK;
}

kp_status kp_selftest_bounds(kp_ctx* ctx) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
#ifndef KP_CHECK
  return fail(ctx, KP_ERR_STATE, "not the bounds-checked build");
#else
  KP_CUDA(cudaMemsetAsync(ctx->arena + ctx->lay.ctl + offsetof(KCtl, err), 0, 8, ctx->stream));
  KParams P = params_now(ctx);
  kp_bounds_selftest_kernel<<<1, 32, 0, ctx->stream>>>(P);
  KP_CUDA(cudaGetLastError());
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  return check_launch(ctx, h);
#endif
}

kp_status kp_selftest_wait_timeout(kp_ctx* ctx) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  KP_CUDA(cudaMemsetAsync(ctx->arena + ctx->lay.ctl + offsetof(KCtl, never_set), 0, 4, ctx->stream));
  KP_CUDA(cudaMemsetAsync(ctx->arena + ctx->lay.ctl + offsetof(KCtl, err), 0, 8, ctx->stream));
  KParams P = params_now(ctx);
  kp_wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(P);
  KP_CUDA(cudaGetLastError());
  KCtl h;
  s = read_ctl(ctx, &h);
  if (s != KP_OK) return s;
  return check_launch(ctx, h);
}

kp_status kp_attach_mlp(kp_ctx* ctx, const kp_mlp* mlp, float mix) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  KParams& P = ctx->P;
  if (!mlp) {
    P.mix_thr = 0;
    P.mlp_W1 = P.mlp_W2 = P.mlp_W3 = nullptr;
    P.mlp_b1 = P.mlp_b2 = P.mlp_b3 = nullptr;
  } else {
    if (ctx->dims.D != 6) return fail(ctx, KP_ERR_ARG, "the learned proposal needs a 6D system");
    if (!(mix >= 0.0f && mix <= 1.0f)) return fail(ctx, KP_ERR_ARG, "mix must be in [0, 1]");
    const void *W1, *W2, *W3;
    mlp_device_weights(mlp, &W1, &P.mlp_b1, &W2, &P.mlp_b2, &W3, &P.mlp_b3);
    P.mlp_W1 = static_cast<const uint16_t*>(W1);
    P.mlp_W2 = static_cast<const uint16_t*>(W2);
    P.mlp_W3 = static_cast<const uint16_t*>(W3);
    const double thr = std::floor((double)mix * 4294967296.0);
    P.mix_thr = thr >= 4294967295.0 ? 0xffffffffu : (uint32_t)thr;
    if (P.mix_thr == 0) P.mlp_W1 = nullptr;
  }
  P.features_on = (P.mix_thr != 0 || P.hv_cap > 0) ? 1 : 0;
  return configure_launch(ctx);
}

kp_status kp_set_harvest(kp_ctx* ctx, float* dev_feat, float* dev_target, int32_t capacity,
                         uint32_t* dev_count) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  KParams& P = ctx->P;
  if (!dev_feat || !dev_target || !dev_count || capacity <= 0) {
    P.hv_feat = P.hv_target = nullptr;
    P.hv_count = nullptr;
    P.hv_cap = 0;
  } else {
    if (ctx->dims.D != 6) return fail(ctx, KP_ERR_ARG, "the harvest needs a 6D system");
    P.hv_feat = dev_feat;
    P.hv_target = dev_target;
    P.hv_count = dev_count;
    P.hv_cap = capacity;
  }
  P.features_on = (P.mix_thr != 0 || P.hv_cap > 0) ? 1 : 0;
  return configure_launch(ctx);
}

const char* kp_last_error(const kp_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void kp_destroy(kp_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->ev_loop0) cudaEventDestroy(ctx->ev_loop0);
  if (ctx->ev_loop1) cudaEventDestroy(ctx->ev_loop1);
  delete ctx;
}

kp_status kp_last_launch_ms(kp_ctx* ctx, float* ms) {
  kp_status s = check_ctx(ctx);
  if (s != KP_OK) return s;
  if (!ms) return KP_ERR_ARG;
  if (!ctx->loop_timed) return fail(ctx, KP_ERR_STATE, "no loop launch recorded");
  KP_CUDA(cudaEventSynchronize(ctx->ev_loop1));
  KP_CUDA(cudaEventElapsedTime(ms, ctx->ev_loop0, ctx->ev_loop1));
  return KP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// kp_plan_static: kp_plan without any allocation, over a static scratch
// ---------------------------------------------------------------------------

namespace {

// Scratch of kp_plan_static.  Every GPU that loads this library holds one
// copy until the process exits.  All kp_plan_static calls on a device share
// it and it keeps the last call's contents, so each call clears what must
// start at zero; calls whose GPU work overlaps (other streams, other host
// threads) race on it.
static __device__ __align__(256) unsigned char g_kp_static_scratch[KP_STATIC_SCRATCH_BYTES];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_base[kStaticMaxDevices];  // device address of the scratch, per device

// Raw {lo, hi} box rows -> the obstacle blob the loop kernel reads: padded
// boxes, then a uniform broad-phase grid of g[0] g[1] g[2] cells (cell
// starts, box ids of each cell in box order) and each cell's clearance, the
// same structure the host builder makes for a context, built here by one
// block of the device (the no-allocation path has no host staging).  A box
// is listed in every cell of its range on each axis, the cell of a
// coordinate v being the FP32 (v - lo) * scale clamped to [0, g - 1], as in
// the hull test.  The clearance of a cell: the smallest over boxes of the
// largest per-axis gap between the cell and the box in cell units, at most
// KP_BP_CLEAR_CAP cells, less KP_BP_CLEAR_MARGIN, in sixteenths, rounded
// down.  Shared memory: C + 1 ints of cell counts, then offsets.
__global__ void __launch_bounds__(1024) kp_static_blob_kernel(
    unsigned char* blob, const float* raw, int n, int pad, int gx, int gy, int gz, float sx,
    float sy, float sz, float lx, float ly, float lz, int start_off, int ids_off, int clear_off) {
  extern __shared__ int kcount[];
  float* dst = reinterpret_cast<float*>(blob);
  uint16_t* start = reinterpret_cast<uint16_t*>(blob + start_off);
  uint16_t* ids = reinterpret_cast<uint16_t*>(blob + ids_off);
  const int C = gx * gy * gz;
  const int g3[3] = {gx, gy, gz};
  const float s3[3] = {sx, sy, sz}, l3[3] = {lx, ly, lz};
  for (int b = threadIdx.x; b < pad; b += blockDim.x) {
    float* o = dst + (size_t)b * 8;
    if (b < n) {
      const float* in = raw + (size_t)b * 6;
      o[0] = in[0] + 0.0f; o[1] = in[1] + 0.0f; o[2] = in[2] + 0.0f; o[3] = 0.0f;
      o[4] = in[3] + 0.0f; o[5] = in[4] + 0.0f; o[6] = in[5] + 0.0f; o[7] = 0.0f;
    } else {
      o[0] = o[1] = o[2] = INFINITY;
      o[4] = o[5] = o[6] = -INFINITY;
      o[3] = o[7] = 0.0f;
    }
  }
  __syncthreads();
  auto in_range = [&](int b, const int* cc) {
    for (int a = 0; a < 3; ++a) {
      float f;
      const float last = (float)(g3[a] - 1);
      const int c0 = bp_cell_of(__fmul_rn(__fsub_rn(dst[b * 8 + a], l3[a]), s3[a]), last, &f);
      const int c1 = bp_cell_of(__fmul_rn(__fsub_rn(dst[b * 8 + 4 + a], l3[a]), s3[a]), last, &f);
      if (cc[a] < c0 || cc[a] > c1) return false;
    }
    return true;
  };
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int cc[3] = {c % gx, (c / gx) % gy, c / (gx * gy)};
    int k = 0;
    double r = (double)KP_BP_CLEAR_CAP;
    for (int b = 0; b < n; ++b) {
      k += in_range(b, cc) ? 1 : 0;
      double gap = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double bl = ((double)dst[b * 8 + a] - (double)l3[a]) * (double)s3[a];
        const double bh = ((double)dst[b * 8 + 4 + a] - (double)l3[a]) * (double)s3[a];
        gap = fmax(gap, fmax(bl - (double)(cc[a] + 1), (double)cc[a] - bh));
      }
      r = fmin(r, gap);
    }
    kcount[c] = k;
    const double v = (r - KP_BP_CLEAR_MARGIN) * 16.0;
    blob[clear_off + c] = v >= 1.0 ? (unsigned char)fmin(255.0, floor(v)) : (unsigned char)0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // cell starts: an exclusive prefix over the counts
    int acc = 0;
    for (int c = 0; c < C; ++c) {
      start[c] = (uint16_t)acc;
      acc += kcount[c];
    }
    start[C] = (uint16_t)acc;
  }
  __syncthreads();
  // the ids, within the room the host counted for them (the same FP32 cell
  // arithmetic gives the same count; the bound only guards the blob)
  const int room = (clear_off - ids_off) / 2;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int cc[3] = {c % gx, (c / gx) % gy, c / (gx * gy)};
    int pos = start[c];
    for (int b = 0; b < n && pos < room; ++b)
      if (in_range(b, cc)) ids[pos++] = (uint16_t)b;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// measured lane-issue peak (denominator of the ALU roofline)
// ---------------------------------------------------------------------------

namespace {

static __device__ float g_kp_peak_sink[KP_MAX_GRID];

// Eight independent FMA chains per thread; 'iters' rounds of eight FMAs.
__global__ void __launch_bounds__(256) kp_lane_peak_kernel(int iters) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1.0e-3f * (float)(threadIdx.x + 7 * j);
  const float m = 0.99990f, c = 1.0e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = __fmaf_rn(a[j], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 1234.5f) g_kp_peak_sink[blockIdx.x % KP_MAX_GRID] = s;  // keeps the chains
}

}  // namespace

extern "C" int32_t kp_bounds_checked(void) {
#ifdef KP_CHECK
  return 1;
#else
  return 0;
#endif
}

extern "C" kp_status kp_measure_lane_peak(void* cuda_stream, double* lane_ops_per_s) {
  if (!lane_ops_per_s) return KP_ERR_ARG;
  *lane_ops_per_s = 0.0;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kp_lane_peak_kernel, 256, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    return KP_ERR_CUDA;
  }
  const int grid = n_sm * (bps > 0 ? bps : 1);
  const int iters = 8192;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, stream);
    if (e == cudaSuccess) {
      kp_lane_peak_kernel<<<grid, 256, 0, stream>>>(iters);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;  // rep 0 warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || best <= 0.0f) {
    cudaGetLastError();
    return KP_ERR_CUDA;
  }
  *lane_ops_per_s = (double)grid * 256.0 * (double)iters * 8.0 / ((double)best * 1e-3);
  return KP_OK;
}

extern "C" kp_status kp_plan_static(const kp_system* sys, const kp_workspace* ws,
                                    const kp_obstacles* obs, const kp_params* prm,
                                    const float* x_init, const kp_goal* goal,
                                    const kp_budget* budget, kp_traj* traj, void* cuda_stream) {
  if (!sys || !ws || !prm || !x_init || !goal || !budget || !traj) return KP_ERR_ARG;
  const int nb = obs ? obs->n_boxes : 0;
  Dims d{};
  if (check_inputs(sys, ws, nb, prm, &d)) return KP_ERR_ARG;
  if (d.fso) return KP_ERR_ARG;  // grid regions only
  if (nb > 0 && !obs->boxes) return KP_ERR_ARG;
  if (check_boxes(nb > 0 ? obs->boxes : nullptr, nb)) return KP_ERR_ARG;
  for (int i = 0; i < d.D; ++i)
    if (std::isnan(x_init[i])) return KP_ERR_ARG;
  if (!(goal->radius >= 0.0f) || std::isnan(goal->center[0]) || std::isnan(goal->center[1]) ||
      std::isnan(goal->center[2]))
    return KP_ERR_ARG;
  if (budget->max_iters < 1 || traj->capacity < 0 ||
      (traj->capacity > 0 && (!traj->states || !traj->ctrls || !traj->steps)))
    return KP_ERR_ARG;
  const Layout lay = make_layout(d);
  if (lay.total > (size_t)KP_STATIC_SCRATCH_BYTES) return KP_ERR_OOM;

  // one-time set-up per device: the device address of the scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
    cudaGetLastError();
    return KP_ERR_CUDA;
  }
  char* A = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[dev]) {
      void* base = nullptr;
      if (cudaGetSymbolAddress(&base, g_kp_static_scratch) != cudaSuccess || !base) {
        cudaGetLastError();
        return KP_ERR_CUDA;
      }
      g_static_base[dev] = base;
    }
    A = static_cast<char*>(g_static_base[dev]);
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  KParams P{};
  fill_params(P, d, lay, sys, ws, prm, A);
  const int pad = (nb + 7) / 8 * 8;
  P.n_boxes_pad = pad;
  // the broad-phase grid: the finest cube of 16^3, 8^3, 4^3, 2^3, 1 whose
  // (cell, box) entries and blob fit (counted here, built on the device)
  int gc = KP_BP_MAX_G;
  for (;; gc /= 2) {
    float sc[3];
    long long entries = 0;
    for (int a = 0; a < 3; ++a) sc[a] = (float)((double)gc / ((double)ws->hi[a] - (double)ws->lo[a]));
    for (int b = 0; b < nb; ++b) {
      long long cells = 1;
      for (int a = 0; a < 3; ++a) {
        const float lo = obs->boxes[(size_t)b * 6 + a] + 0.0f, hi = obs->boxes[(size_t)b * 6 + 3 + a] + 0.0f;
        cells *= host_bp_cell(hi, ws->lo[a], sc[a], gc) - host_bp_cell(lo, ws->lo[a], sc[a], gc) + 1;
      }
      entries += cells;
    }
    const size_t cells3 = (size_t)gc * gc * gc;
    const size_t bytes = (size_t)pad * 32 + round16((cells3 + 1) * 2) + round16((size_t)entries * 2) +
                         round16(cells3);
    if (gc == 1 || (entries <= KP_BP_MAX_IDS && bytes <= (size_t)KP_BLOB_BYTES)) {
      for (int a = 0; a < 3; ++a) {
        P.bp_g[a] = gc;
        P.bp_scale[a] = sc[a];
        P.bp_last[a] = (float)(gc - 1);
      }
      P.bp_start_off = pad * 32;
      P.bp_ids_off = P.bp_start_off + (int32_t)round16((cells3 + 1) * 2);
      P.bp_clear_off = P.bp_ids_off + (int32_t)round16((size_t)entries * 2);
      P.bp_n_ids = (int32_t)entries;
      P.blob_bytes = P.bp_clear_off + (int32_t)round16(cells3);
      break;
    }
  }
  for (int a = 0; a < 3; ++a) P.goal_c[a] = goal->center[a];
  P.goal_r2 = (float)((double)goal->radius * (double)goal->radius);
  P.seed_lo = (uint32_t)(prm->seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(prm->seed >> 32);
  P.log = KLog{};
  P.wait_ns = 2000000000ull;

  // launch shape, as for a context with this obstacle count
  int num_sms = 0, bps = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return KP_ERR_CUDA;
  }
  // as configure_launch: the grid with room for any chunking, the chunks
  // of that grid, then the score scratch those chunks need
  int grid = 0;
  auto shape = [&](int sd) -> kp_status {
    const size_t smem = (size_t)P.blob_bytes + (size_t)sd * 8;
    if (occupancy(d.sys, false, smem, &bps) != cudaSuccess) {
      cudaGetLastError();
      return KP_ERR_CUDA;
    }
    if (bps < 1) return KP_ERR_ARG;  // no block of this shape can be resident
    grid = bps * num_sms;
    if (grid > KP_MAX_GRID) grid = KP_MAX_GRID;
    P.sd_bytes = sd * 8;
    return KP_OK;
  };
  const int min_ch = d.R_pad / (d.R_pad < 1024 ? d.R_pad : 1024);
  kp_status ss = shape(min_ch > 1024 ? min_ch : 1024);
  if (ss != KP_OK) return ss;
  P.nch = region_chunks(grid, d.R_pad);
  ss = shape(d.R_pad / P.nch > P.nch ? d.R_pad / P.nch : P.nch);
  if (ss != KP_OK) return ss;
  const size_t smem = (size_t)P.blob_bytes + (size_t)P.sd_bytes;

  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
    return e == cudaSuccess;
  };
  // obstacles: raw rows into the (not yet used) trajectory rows, padded on
  // the device into the box slots
  if (nb > 0)
    ok(cudaMemcpyAsync(A + lay.traj, obs->boxes, (size_t)nb * 24, cudaMemcpyHostToDevice, stream));
  kp_static_blob_kernel<<<1, 1024, (size_t)(P.bp_g[0] * P.bp_g[1] * P.bp_g[2] + 1) * 4, stream>>>(
      reinterpret_cast<unsigned char*>(A + lay.boxes), reinterpret_cast<const float*>(A + lay.traj),
      nb, pad, P.bp_g[0], P.bp_g[1], P.bp_g[2], P.bp_scale[0], P.bp_scale[1], P.bp_scale[2],
      ws->lo[0], ws->lo[1], ws->lo[2], P.bp_start_off, P.bp_ids_off, P.bp_clear_off);
  ok(cudaGetLastError());
  // everything that must start from zero (the scratch keeps old contents)
  ok(cudaMemsetAsync(A + lay.ctl, 0, sizeof(KCtl), stream));
  ok(cudaMemsetAsync(A + lay.visited, 0, d.n_sub, stream));
  ok(cudaMemsetAsync(A + lay.claim, 0xff, d.n_sub * 4, stream));
  ok(cudaMemsetAsync(A + lay.n_valid, 0, (size_t)d.R * 4, stream));
  ok(cudaMemsetAsync(A + lay.n_invalid, 0, (size_t)d.R * 4, stream));
  ok(cudaMemsetAsync(A + lay.cov, 0, (size_t)d.R * 4, stream));
  ok(cudaMemsetAsync(A + lay.avail, 0, (size_t)d.R, stream));
  RootState root{};
  for (int i = 0; i < d.D; ++i) root.x[i] = x_init[i];
  const uint64_t max_ns = budget->max_ms > 0.0 ? (uint64_t)(budget->max_ms * 1e6) : 0ull;
  if (e == cudaSuccess) {
    switch (d.sys) {
      case KP_SYS_DI:
        ok(launch_reset_di(P, root, stream));
        ok(launch_loop_di(P, grid, smem, budget->max_iters, max_ns, false, stream, root, 0));
        break;
      case KP_SYS_DUBINS:
        ok(launch_reset_dubins(P, root, stream));
        ok(launch_loop_dubins(P, grid, smem, budget->max_iters, max_ns, false, stream, root,
                              0));
        break;
      default:
        ok(launch_reset_quad(P, root, stream));
        ok(launch_loop_quad(P, grid, smem, budget->max_iters, max_ns, false, stream, root, 0));
    }
  }
  if (e == cudaSuccess) {
    kp_extract_kernel<<<1, 32, 0, stream>>>(P);
    ok(cudaGetLastError());
  }
  KCtl h{};
  ok(cudaMemcpyAsync(&h, A + lay.ctl, sizeof(KCtl), cudaMemcpyDeviceToHost, stream));
  ok(cudaStreamSynchronize(stream));
  if (e != cudaSuccess) return KP_ERR_CUDA;
  if (h.err == KP_DEV_ERR_TIMEOUT) return KP_ERR_TIMEOUT;
  if (h.err == KP_DEV_ERR_REPLAY) return KP_ERR_STATE;  // as kp_plan reports it
  if (h.err != 0) return KP_ERR_CUDA;
  if (h.state == KP_DEV_BAD_ROOT) return KP_ERR_ARG;
  traj->n_edges = 0;
  if (h.state != KP_DEV_SOLVED || h.n_edges < 0) return KP_NO_SOLUTION;
  traj->n_edges = h.n_edges;
  if (h.n_edges > traj->capacity || h.n_edges > KP_TRAJ_ROWS) return KP_ERR_ARG;
  const int n = h.n_edges;
  if (n > 0) {
    const char* rows = A + lay.traj;
    ok(cudaMemcpy2DAsync(traj->states, 12 * 4, rows, 17 * 4, 12 * 4, n, cudaMemcpyDeviceToHost,
                         stream));
    ok(cudaMemcpy2DAsync(traj->ctrls, 4 * 4, rows + 12 * 4, 17 * 4, 4 * 4, n,
                         cudaMemcpyDeviceToHost, stream));
    ok(cudaMemcpy2DAsync(traj->steps, 4, rows + 16 * 4, 17 * 4, 4, n, cudaMemcpyDeviceToHost,
                         stream));
    ok(cudaStreamSynchronize(stream));
    if (e != cudaSuccess) return KP_ERR_CUDA;
    for (int i = 0; i < n; ++i) {  // the rows carry the step count as a float
      float f;
      std::memcpy(&f, &traj->steps[i], 4);
      traj->steps[i] = (int32_t)f;
    }
  }
  return KP_OK;
}

// ---------------------------------------------------------------------------
// server: host runtime
// ---------------------------------------------------------------------------

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct PendingQuery {
  int64_t id;
  kp_system sys;
  kp_workspace ws;
  kp_params prm;
  std::vector<float> boxes;
  RootState root;
  kp_goal goal;
  kp_budget budget;
  double t_submit;
};

struct SlotState {
  bool used = false;
  int64_t id = -1;
  size_t off = 0, bytes = 0;
  Layout lay{};
  double t_submit = 0;
};

struct StoredResult {
  kp_status status;
  std::vector<float> rows;  // n_edges x 17
  int32_t n_edges;
};

}  // namespace

struct kp_server {
  kp_server_config cfg{};
  char* pool = nullptr;
  size_t pool_bytes = 0;
  cudaStream_t stream = nullptr;  // the persistent launch
  cudaStream_t copy = nullptr;    // uploads and read-backs beside it
  KServerDev* dev = nullptr;
  KQuery* queries = nullptr;
  KServerHost* host_h = nullptr;  // host view of the mapped area
  KServerHost* host_d = nullptr;  // device view
  int team_blocks = 0, n_teams = 0, grid = 0, num_sms = 0;
  size_t smem = 0;
  std::map<size_t, size_t> free_list;  // offset -> bytes
  std::vector<SlotState> slots;
  std::deque<PendingQuery> pending;
  std::unordered_map<int64_t, StoredResult> results;
  std::deque<kp_server_done> ready;
  uint32_t posted = 0, consumed = 0;
  int64_t next_id = 0, submitted = 0, completed = 0;
  cudaEvent_t ev_kernel = nullptr;
  bool launched = false;
  bool poisoned = false;
  std::vector<unsigned char> blob;
};

namespace {

size_t server_ctl_bytes(int max_slots) {
  return align256(sizeof(KServerDev)) + align256((size_t)max_slots * sizeof(KQuery));
}

// First fit in the pool's free list (256-byte granules).
bool pool_alloc(kp_server* s, size_t bytes, size_t* off) {
  bytes = align256(bytes);
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t o = it->first + bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[o] = rest;
      return true;
    }
  }
  return false;
}

void pool_free(kp_server* s, size_t off, size_t bytes) {
  bytes = align256(bytes);
  auto it = s->free_list.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != s->free_list.end() && it->first + it->second == next->first) {
    it->second += next->second;
    s->free_list.erase(next);
  }
  if (it != s->free_list.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      s->free_list.erase(it);
    }
  }
}

void finish_now(kp_server* s, int64_t id, kp_status st, double t_submit) {
  kp_server_done d{};
  d.id = id;
  d.status = st;
  d.latency_ms = now_ms() - t_submit;
  s->ready.push_back(d);
  s->results[id] = StoredResult{st, {}, 0};
  s->completed += 1;
}

// Admits the query if a slot and pool memory are free: uploads its blob and
// descriptor (copy stream) and publishes it.  Returns false to keep it
// waiting; an invalid query completes at once with KP_ERR_ARG.
bool try_admit(kp_server* s, PendingQuery& q) {
  int slot = -1;
  for (int i = 0; i < (int)s->slots.size(); ++i)
    if (!s->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return false;
  Dims d{};
  if (check_inputs(&q.sys, &q.ws, (int)(q.boxes.size() / 6), &q.prm, &d)) {
    finish_now(s, q.id, KP_ERR_ARG, q.t_submit);
    return true;
  }
  const Layout lay = make_layout(d);
  size_t off = 0;
  if (!pool_alloc(s, lay.total, &off)) {
    if (s->free_list.empty() || lay.total > s->pool_bytes) {
      finish_now(s, q.id, KP_ERR_OOM, q.t_submit);
      return true;
    }
    return false;
  }
  KQuery kq{};
  KParams& P = kq.P;
  fill_params(P, d, lay, &q.sys, &q.ws, &q.prm, s->pool + off);
  for (int a = 0; a < 3; ++a) P.goal_c[a] = q.goal.center[a];
  P.goal_r2 = (float)((double)q.goal.radius * (double)q.goal.radius);
  P.seed_lo = (uint32_t)(q.prm.seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(q.prm.seed >> 32);
  P.wait_ns = 2000000000ull;
  const int nch = region_chunks(s->team_blocks, d.R_pad);
  P.nch = nch;
  P.sd_bytes = KS_SD_DOUBLES * 8;
  // no cell clearances: the host would spend milliseconds per query on them
  const size_t blob_bytes = build_blob(s->blob.data(), q.boxes.empty() ? nullptr : q.boxes.data(),
                                       (int)(q.boxes.size() / 6), q.ws, P, KS_BLOB_MAX, false);
  if (blob_bytes > (size_t)KS_BLOB_MAX || d.R_pad / nch > KS_SD_DOUBLES) {
    pool_free(s, off, lay.total);
    finish_now(s, q.id, KP_ERR_ARG, q.t_submit);
    return true;
  }
  kq.root = q.root;
  kq.max_iters = q.budget.max_iters;
  kq.id = (int32_t)q.id;
  kq.max_ns = q.budget.max_ms > 0.0 ? (uint64_t)(q.budget.max_ms * 1e6) : 0ull;
  bool ok = cudaMemcpyAsync(s->pool + off + lay.boxes, s->blob.data(), blob_bytes,
                            cudaMemcpyHostToDevice, s->copy) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(s->queries + slot, &kq, sizeof(KQuery), cudaMemcpyHostToDevice,
                             s->copy) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(s->copy) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    s->poisoned = true;
    pool_free(s, off, lay.total);
    finish_now(s, q.id, KP_ERR_CUDA, q.t_submit);
    return true;
  }
  SlotState& ss = s->slots[slot];
  ss.used = true;
  ss.id = q.id;
  ss.off = off;
  ss.bytes = lay.total;
  ss.lay = lay;
  ss.t_submit = q.t_submit;
  // publish: ring entry first, then the count
  s->host_h->ring[s->posted % KS_RING] = (uint32_t)slot;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  reinterpret_cast<volatile uint32_t*>(&s->host_h->posted)[0] = s->posted + 1;
  s->posted += 1;
  return true;
}

void admit_pending(kp_server* s) {
  while (!s->pending.empty()) {
    if (!try_admit(s, s->pending.front())) break;
    s->pending.pop_front();
  }
}

bool any_resident(const kp_server* s) {
  for (const auto& ss : s->slots)
    if (ss.used) return true;
  return false;
}

// Launches the persistent server when queries are resident and no launch
// is running (teams leave after idle_ms without work).
kp_status ensure_running(kp_server* s) {
  if (reinterpret_cast<volatile int32_t*>(&s->host_h->error)[0] != 0) {
    s->poisoned = true;  // a bounded device wait expired: no relaunch
    return KP_ERR_TIMEOUT;
  }
  if (s->launched) {
    const cudaError_t q = cudaEventQuery(s->ev_kernel);
    if (q == cudaErrorNotReady) return KP_OK;
    if (q != cudaSuccess) {
      cudaGetLastError();
      s->poisoned = true;
      return KP_ERR_CUDA;
    }
    s->launched = false;
  }
  if (!any_resident(s)) return KP_OK;
  KServerArgs A{};
  A.dev = s->dev;
  A.host = s->host_d;
  A.queries = s->queries;
  A.team_blocks = s->team_blocks;
  A.idle_ns = (uint64_t)(s->cfg.idle_ms * 1e6);
  A.wait_ns = 2000000000ull;
  if (launch_server(A, s->grid, s->smem, s->stream) != cudaSuccess ||
      cudaEventRecord(s->ev_kernel, s->stream) != cudaSuccess) {
    cudaGetLastError();
    s->poisoned = true;
    return KP_ERR_CUDA;
  }
  s->launched = true;
  return KP_OK;
}

// Reads new completion records; frees their slots and pool memory.
kp_status collect(kp_server* s) {
  for (;;) {
    KDone* d = &s->host_h->done[s->consumed % KS_RING];
    const uint32_t seq = reinterpret_cast<volatile uint32_t*>(&d->seq)[0];
    if (seq != s->consumed + 1) break;
    std::atomic_thread_fence(std::memory_order_acquire);
    const KDone r = *d;
    s->consumed += 1;
    if (r.slot < 0 || r.slot >= (int)s->slots.size() || !s->slots[r.slot].used) {
      s->poisoned = true;
      return KP_ERR_STATE;
    }
    SlotState& ss = s->slots[r.slot];
    kp_status st = r.err ? KP_ERR_TIMEOUT
                         : (r.state == KP_DEV_SOLVED ? KP_OK
                                                     : (r.state == KP_DEV_BAD_ROOT ? KP_ERR_ARG
                                                                                   : KP_NO_SOLUTION));
    StoredResult res{st, {}, 0};
    if (st == KP_OK && r.n_edges >= 0 && r.n_edges <= KP_TRAJ_ROWS) {
      res.n_edges = r.n_edges;
      res.rows.resize((size_t)r.n_edges * 17);
      if (r.n_edges > 0 &&
          (cudaMemcpyAsync(res.rows.data(), s->pool + ss.off + ss.lay.traj,
                           (size_t)r.n_edges * 17 * 4, cudaMemcpyDeviceToHost,
                           s->copy) != cudaSuccess ||
           cudaStreamSynchronize(s->copy) != cudaSuccess)) {
        cudaGetLastError();
        s->poisoned = true;
        return KP_ERR_CUDA;
      }
    }
    kp_server_done out{};
    out.id = ss.id;
    out.status = st;
    out.n_edges = r.n_edges;
    out.iterations = r.iterations;
    out.n_nodes = r.n_nodes;
    out.samples = (int64_t)r.samples;
    out.device_ms = (double)(r.t_end_ns - r.t_start_ns) * 1e-6;
    out.latency_ms = now_ms() - ss.t_submit;
    s->ready.push_back(out);
    s->results[ss.id] = std::move(res);
    s->completed += 1;
    pool_free(s, ss.off, ss.bytes);
    ss = SlotState{};
  }
  return KP_OK;
}

}  // namespace

extern "C" {

size_t kp_server_required_bytes(int32_t max_slots) {
  if (max_slots < 1 || max_slots > KS_RING) return 0;
  return server_ctl_bytes(max_slots);
}

kp_status kp_server_create(const kp_server_config* cfg, void* dev_pool, size_t pool_bytes,
                           void* cuda_stream, kp_server** out) {
  if (!cfg || !out || !dev_pool || ((uintptr_t)dev_pool & 255u)) return KP_ERR_ARG;
  *out = nullptr;
  if (cfg->team_blocks < 1 || cfg->max_slots < 1 || cfg->max_slots > KS_RING ||
      !(cfg->idle_ms > 0.0))
    return KP_ERR_ARG;
  const size_t ctl = server_ctl_bytes(cfg->max_slots);
  if (pool_bytes < ctl + 256) return KP_ERR_OOM;
  kp_server* s = new (std::nothrow) kp_server();
  if (!s) return KP_ERR_OOM;
  s->cfg = *cfg;
  s->pool = static_cast<char*>(dev_pool);
  s->pool_bytes = pool_bytes;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->dev = reinterpret_cast<KServerDev*>(s->pool);
  s->queries = reinterpret_cast<KQuery*>(s->pool + align256(sizeof(KServerDev)));
  s->free_list[ctl] = (pool_bytes - ctl) & ~(size_t)255;
  s->slots.resize(cfg->max_slots);
  s->blob.resize(KP_BLOB_BYTES);
  s->team_blocks = cfg->team_blocks;
  auto bad = [&](kp_status st) {
    cudaGetLastError();
    if (s->host_h) cudaFreeHost(s->host_h);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->ev_kernel) cudaEventDestroy(s->ev_kernel);
    delete s;
    return st;
  };
  int dev = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bad(KP_ERR_CUDA);
  s->smem = ((sizeof(KParams) + 127) & ~(size_t)127) + (size_t)KS_BLOB_MAX +
            (size_t)KS_SD_DOUBLES * 8;
  if (server_occupancy(s->smem, &bps) != cudaSuccess || bps < 1) return bad(KP_ERR_CUDA);
  const int resident = bps * s->num_sms;
  s->n_teams = resident / s->team_blocks;
  if (s->n_teams < 1) return bad(KP_ERR_ARG);
  if (s->n_teams > KS_MAX_TEAMS) s->n_teams = KS_MAX_TEAMS;
  s->grid = s->n_teams * s->team_blocks;
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->host_h), sizeof(KServerHost),
                    cudaHostAllocMapped) != cudaSuccess)
    return bad(KP_ERR_CUDA);
  std::memset(s->host_h, 0, sizeof(KServerHost));
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->host_d), s->host_h, 0) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_kernel, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemsetAsync(s->dev, 0, sizeof(KServerDev), s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return bad(KP_ERR_CUDA);
  *out = s;
  return KP_OK;
}

kp_status kp_server_submit(kp_server* s, const kp_system* sys, const kp_workspace* ws,
                           const kp_obstacles* obs, const kp_params* prm, const float* x_init,
                           const kp_goal* goal, const kp_budget* budget, int64_t* id) {
  if (!s || !sys || !ws || !prm || !x_init || !goal || !budget || !id) return KP_ERR_ARG;
  if (s->poisoned) return KP_ERR_STATE;
  const int nb = obs ? obs->n_boxes : 0;
  Dims d{};
  if (check_inputs(sys, ws, nb, prm, &d)) return KP_ERR_ARG;
  if (d.fso) return KP_ERR_ARG;  // grid regions only
  if (nb > 0 && (!obs->boxes || check_boxes(obs->boxes, nb))) return KP_ERR_ARG;
  if (budget->max_iters < 1 || !(goal->radius >= 0.0f)) return KP_ERR_ARG;
  for (int i = 0; i < d.D; ++i)
    if (std::isnan(x_init[i])) return KP_ERR_ARG;
  PendingQuery q;
  q.id = s->next_id++;
  q.sys = *sys;
  q.ws = *ws;
  q.prm = *prm;
  if (nb > 0) q.boxes.assign(obs->boxes, obs->boxes + (size_t)nb * 6);
  q.root = RootState{};
  for (int i = 0; i < d.D; ++i) q.root.x[i] = x_init[i];
  q.goal = *goal;
  q.budget = *budget;
  q.t_submit = now_ms();
  *id = q.id;
  s->submitted += 1;
  s->pending.push_back(std::move(q));
  admit_pending(s);
  return ensure_running(s);
}

kp_status kp_server_poll(kp_server* s, kp_server_done* out, int32_t capacity, int32_t* n_out) {
  if (!s || !n_out || capacity < 0 || (capacity > 0 && !out)) return KP_ERR_ARG;
  *n_out = 0;
  if (s->poisoned) return KP_ERR_STATE;
  kp_status st = collect(s);
  if (st != KP_OK) return st;
  admit_pending(s);
  st = ensure_running(s);
  if (st != KP_OK) return st;
  int n = 0;
  while (n < capacity && !s->ready.empty()) {
    out[n++] = s->ready.front();
    s->ready.pop_front();
  }
  *n_out = n;
  return KP_OK;
}

kp_status kp_server_result(kp_server* s, int64_t id, kp_traj* traj) {
  if (!s || !traj) return KP_ERR_ARG;
  auto it = s->results.find(id);
  if (it == s->results.end()) return KP_ERR_ARG;
  const StoredResult& r = it->second;
  traj->n_edges = r.n_edges;
  if (r.status != KP_OK) {
    const kp_status st = r.status;
    s->results.erase(it);
    return st;
  }
  if (r.n_edges > traj->capacity) return KP_ERR_ARG;
  for (int e = 0; e < r.n_edges; ++e) {
    std::memcpy(traj->states + (size_t)e * 12, r.rows.data() + (size_t)e * 17, 12 * 4);
    std::memcpy(traj->ctrls + (size_t)e * 4, r.rows.data() + (size_t)e * 17 + 12, 4 * 4);
    traj->steps[e] = (int32_t)r.rows[(size_t)e * 17 + 16];
  }
  s->results.erase(it);
  return KP_OK;
}

kp_status kp_server_stats_get(kp_server* s, kp_server_stats* out) {
  if (!s || !out) return KP_ERR_ARG;
  out->teams = s->n_teams;
  out->team_blocks = s->team_blocks;
  out->pending = (int32_t)s->pending.size();
  int res = 0;
  for (const auto& ss : s->slots) res += ss.used ? 1 : 0;
  out->resident = res;
  out->submitted = s->submitted;
  out->completed = s->completed;
  size_t f = 0;
  for (const auto& kv : s->free_list) f += kv.second;
  out->pool_free = f;
  out->device_error = reinterpret_cast<volatile int32_t*>(&s->host_h->error)[0];
  out->running = s->launched && cudaEventQuery(s->ev_kernel) == cudaErrorNotReady ? 1 : 0;
  cudaGetLastError();
  return KP_OK;
}

void kp_server_destroy(kp_server* s) {
  if (!s) return;
  if (s->host_h) {
    reinterpret_cast<volatile uint32_t*>(&s->host_h->stop)[0] = 1u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
  cudaStreamSynchronize(s->stream);
  if (s->copy) {
    cudaStreamSynchronize(s->copy);
    cudaStreamDestroy(s->copy);
  }
  if (s->ev_kernel) cudaEventDestroy(s->ev_kernel);
  if (s->host_h) cudaFreeHost(s->host_h);
  delete s;
}

}  // extern "C"
