// kp_loop.cuh -- the Kino-PAX loop as one persistent cooperative kernel, plus
// the small reset / import / trajectory kernels.  Instantiated once per
// system by kp_sys_*.cu.
//
// One pass of the loop body (Algorithm 1) runs as four grid phases separated
// by bounded grid barriers, with no host involvement:
//   E  Propagate (Algorithm 2): lanes carry one sample (V_E position, j)
//      each and are refilled from a grid-wide key counter; draw u and k,
//      integrate k steps in FP32 registers, check each step against the
//      state box and the obstacle boxes staged in shared memory, bin the
//      end (or first invalid) state, count n_valid / n_invalid, claim newly
//      reached sub-regions (smallest sample key wins), keep the end state
//      of a sample that may still be accepted.
//   A  accept decisions (representative or P_accept draw), accepted keys
//      compacted per warp in key order; alongside, on warp 0:
//   S  Score per region (Eq. 3-4, FP64, rounded exactly as written) and
//      the pairwise partial sum of each aligned region chunk (Eq. 5's sum).
//   N  first, on warp 0 of each region-chunk block, T: the sum of Eq. 5
//      from the partial sums and P_accept with its integer accept threshold
//      per region; each block appends its own accepted samples (Algorithm
//      4, to T and V_E) at their key-order node ids, from the kept end
//      states, with the goal test; then one selection draw per old node
//      against its region's new threshold (Algorithm 4, V_E <-> V_O) and
//      per-block V_E counts.
//   L  V_E list in ascending node id, lambda for the next pass (Eq. 6),
//      stop decision.
// With a network attached (learned proposal) a phase F before E evaluates
// it on every V_E node.
#pragma once

#include <cstdint>

#include "kp_device.cuh"
#include "kp_mlp.cuh"

namespace kp {

constexpr int KP_WARPS = KP_BLOCK / 32;

struct LoopShared {
  ScanSmem scan;
  unsigned long long red[64];
  uint64_t mbar;
  int flag;
  int bcast[2];
  int32_t phase_ns[12];  // per-pass phase timers (block 0, thread 0)
  // accepted samples of this block, from the accept phase to the node-set
  // phase: warp w compacted acc_n[w] keys at acc_key[acc_a[w]...], which
  // are the block's accepted samples acc_off[w] .. acc_off[w] + acc_n[w] - 1
  int acc_a[KP_WARPS], acc_n[KP_WARPS], acc_off[KP_WARPS];
  int acc_tot;
};

// Stage the obstacle blob (boxes and broad-phase grid) into shared memory
// with bulk asynchronous copies (TMA engine) completing on one mbarrier.
// Returns false on a wait timeout.
__device__ __forceinline__ bool stage_boxes(const KParams& P, float4* sbox, LoopShared& sh) {
  const uint32_t bytes = (uint32_t)P.blob_bytes;  // multiple of 16
  if (bytes == 0) return true;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&sh.mbar);
  const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(sbox);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
    const uint32_t piece = 16384u;  // several copies of <= 16 KB each
    for (uint32_t off = 0; off < bytes; off += piece) {
      const uint32_t n = bytes - off < piece ? bytes - off : piece;  // multiple of 16
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
          "[%3];" ::"r"(dst0 + off),
          "l"(reinterpret_cast<const char*>(P.boxes) + off), "r"(n), "r"(mb)
          : "memory");
    }
    // bounded wait for phase 0 of the mbarrier
    int ok = 0;
    const uint64_t t0 = global_ns();
    for (uint32_t spin = 0;; ++spin) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(mb)
          : "memory");
      if (done) { ok = 1; break; }
      if (global_ns() - t0 > P.wait_ns) break;
    }
    if (!ok) {
      raise_error(P.ctl, KP_DEV_ERR_TIMEOUT, 1);
      // wait once more, again bounded, for the copies still in flight
      const uint64_t t1 = global_ns();
      for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mb)
            : "memory");
        if (done || global_ns() - t1 > P.wait_ns) break;
      }
    }
    // invalidate the object so that a later staging (the server stages one
    // blob per query) initialises a fresh mbarrier
    if (ok) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
    sh.flag = ok;
  }
  __syncthreads();
  return sh.flag != 0;
}

__device__ __forceinline__ int eq6_lambda(int t_e, int n_tree, int n_ve, int lambda_max) {
  if (n_ve <= 0) return lambda_max;
  int room = t_e - n_tree;
  if (room < 0) room = 0;
  const int lam = room / n_ve;
  return lam < lambda_max ? lam : lambda_max;
}

// Node chunk [v0, v1) of this block over n nodes.
__device__ __forceinline__ void chunk_of(const Team& T, int n, int* c0, int* c1) {
  const int per = (n + T.nb - 1) / T.nb;
  const long long a = (long long)T.b * per;
  *c0 = (int)(a < n ? a : n);
  *c1 = (int)(a + per < n ? a + per : n);
}

// Sum of blk[0..G) and of blk[0..blockIdx.x), by one warp (no block sync).
__device__ __forceinline__ void warp_prefix(const Team& T, const uint32_t* blk,
                                            unsigned long long* before,
                                            unsigned long long* total) {
  unsigned long long pre = 0, tot = 0;
  for (int i = (int)(threadIdx.x & 31u); i < T.nb; i += 32) {
    const unsigned long long c = __ldcg(blk + i);
    tot += c;
    if (i < T.b) pre += c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pre += __shfl_xor_sync(0xffffffffu, pre, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  *before = pre;
  *total = tot;
}

// Sum of blk[0..G) and of blk[0..blockIdx.x).
__device__ __forceinline__ void block_prefix(const Team& T, const uint32_t* blk, LoopShared& sh,
                                             unsigned long long* before,
                                             unsigned long long* total) {
  unsigned long long pre = 0, tot = 0;
  for (int i = threadIdx.x; i < T.nb; i += blockDim.x) {
    const unsigned long long c = __ldcg(blk + i);
    tot += c;
    if (i < T.b) pre += c;
  }
  block_sum2(pre, tot, sh.red, before, total);
}

// Nodes of a block's chunk are visited in tiles of blockDim.x: node v0 +
// tile * blockDim.x + threadIdx.x, so that a warp's loads and stores of the
// per-node arrays are coalesced.

// Block sum of one int per thread (every thread gets it).
__device__ __forceinline__ int block_sum(int c, LoopShared& sh) {
  unsigned long long a, dummy;
  block_sum2((unsigned long long)c, 0, sh.red, &a, &dummy);
  return (int)a;
}

// Phase N': count V_E members of this block's node chunk (no draws) and
// publish the count.
__device__ __forceinline__ void count_ve(const KParams& P, const Team& T, int n, LoopShared& sh) {
  int v0, v1;
  chunk_of(T, n, &v0, &v1);
  int c = 0;
  for (int v = v0 + (int)threadIdx.x; v < v1; v += (int)blockDim.x)
    c += P.in_ve[KP_IDX(P, v, P.t_e, 1)] ? 1 : 0;
  const int tot = block_sum(c, sh);
  if (threadIdx.x == 0) P.blk_b[KP_IDX(P, T.b, KP_MAX_GRID, 2)] = (uint32_t)tot;
}

// Phase L: write the V_E list (ascending node id) from the per-block counts:
// the block's offset is the sum of the counts before it; inside the chunk
// each tile is compacted in node order (warp ballots, then the warps'
// counts in order).  Returns |V_E|.
__device__ __forceinline__ int write_ve(const KParams& P, const Team& T, int n, LoopShared& sh) {
  int v0, v1;
  chunk_of(T, n, &v0, &v1);
  unsigned long long off, total;
  block_prefix(T, P.blk_b, sh, &off, &total);
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
  int base = (int)off;
  for (int t0 = v0; t0 < v1; t0 += (int)blockDim.x) {
    const int v = t0 + (int)threadIdx.x;
    const bool m = v < v1 && P.in_ve[KP_IDX(P, v, P.t_e, 3)];
    const uint32_t bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) sh.scan.warp[w] = __popc(bal);
    __syncthreads();
    int before = 0, tile = 0;
    for (int q = 0; q < nw; ++q) {
      const int cq = sh.scan.warp[q];
      before += q < (int)w ? cq : 0;
      tile += cq;
    }
    if (m) P.ve[KP_IDX(P, base + before + __popc(bal & ((1u << lane) - 1u)), P.t_e, 4)] = v;
    base += tile;
    __syncthreads();
  }
  return (int)total;
}

// ---------------------------------------------------------------------------
// learned proposal: node features and the network (6D systems)
// ---------------------------------------------------------------------------

// Features 2q and 2q+1 (q = 0..15) of node v under the current region
// tables; the 32 features are: bounded state entries mapped to [-1, 1], an
// unbounded one wrapped to [-pi, pi) and divided by pi; goal minus
// position; Cov / n'; FreeVol / vol; log(1 + n_valid); log(1 + n_invalid);
// P_accept of the node's region and of its six face neighbours in the
// position grid (0 outside, and 0 under the kd-tree decomposition); zeros
// from feature 20 on.
__device__ __forceinline__ float state_feature(const KParams& P, int i, float x) {
  if (P.feat_scale[i] > 0.0f) return (x - P.x_lo[i]) * P.feat_scale[i] - 1.0f;
  const float y = x - 6.28318530717958648f * floorf((x + 3.14159265358979324f) *
                                                    0.159154943091895336f);
  return y * 0.318309886183790672f;
}

__device__ __forceinline__ float neighbour_accept(const KParams& P, int r, int k) {
  const int gx = P.grid[0], gy = P.grid[1], gz = P.grid[2];
  const int cx = r % gx, cy = (r / gx) % gy, cz = (r / (gx * gy)) % gz, sb = r / (gx * gy * gz);
  const int nx = cx + (k == 0 ? -1 : k == 1 ? 1 : 0);
  const int ny = cy + (k == 2 ? -1 : k == 3 ? 1 : 0);
  const int nz = cz + (k == 4 ? -1 : k == 5 ? 1 : 0);
  if (nx < 0 || nx >= gx || ny < 0 || ny >= gy || nz < 0 || nz >= gz) return 0.0f;
  return (float)P.thr[nx + gx * (ny + gy * (nz + gz * sb))] * 2.3283064365386963e-10f;
}

__device__ __forceinline__ void node_feature_pair(const KParams& P, int v, int q, float* f2) {
  f2[0] = f2[1] = 0.0f;
  if (q < 3) {
    f2[0] = state_feature(P, 2 * q, P.st[(size_t)(2 * q) * P.t_e + v]);
    f2[1] = state_feature(P, 2 * q + 1, P.st[(size_t)(2 * q + 1) * P.t_e + v]);
    return;
  }
  if (q == 3) {
    f2[0] = P.goal_c[0] - P.st[v];
    f2[1] = P.goal_c[1] - P.st[(size_t)P.t_e + v];
    return;
  }
  if (q >= 10) return;
  const int r = P.region[v];
  const float nv = (float)P.n_valid[r], ni = (float)P.n_invalid[r], dl = (float)P.delta;
  switch (q) {
    case 4:
      f2[0] = P.goal_c[2] - P.st[(size_t)2 * P.t_e + v];
      f2[1] = (float)P.cov[r] / (float)P.n_sub_per;
      break;
    case 5:
      f2[0] = (dl + nv) / (dl + nv + ni);
      f2[1] = log1pf(nv);
      break;
    case 6:
      f2[0] = log1pf(ni);
      f2[1] = (float)P.thr[r] * 2.3283064365386963e-10f;
      break;
    default:  // q = 7, 8, 9: neighbours 2(q-7) and 2(q-7)+1 (none for kd-tree regions)
      if (P.fso) break;
      f2[0] = neighbour_accept(P, r, 2 * (q - 7));
      f2[1] = neighbour_accept(P, r, 2 * (q - 7) + 1);
  }
}

// Phase F: features of every V_E position (kept for the harvest) and, with
// a network attached, its outputs, in tiles of 32 positions per block; 16
// threads share the features of one position.  Not inlined: it runs once
// per pass, and as a call it gets the register budget of the loop kernel
// to itself instead of sharing it with the loop state live around it.
static __device__ __noinline__ void phase_features(const KParams& P, const Team& T, int n_ve,
                                                   unsigned char* mtile) {
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(mtile);
  __nv_bfloat16* sH = sX + MLP_LOOP_TILE * MLP_XS;
  MlpWeights w;
  w.W1 = reinterpret_cast<const __nv_bfloat16*>(P.mlp_W1);
  w.b1 = P.mlp_b1;
  w.W2 = reinterpret_cast<const __nv_bfloat16*>(P.mlp_W2);
  w.b2 = P.mlp_b2;
  w.W3 = reinterpret_cast<const __nv_bfloat16*>(P.mlp_W3);
  w.b3 = P.mlp_b3;
  const int n_tiles = (n_ve + MLP_LOOP_TILE - 1) / MLP_LOOP_TILE;
  const int q = threadIdx.x & 15;  // 16 rows x 16 feature pairs per round
  for (int tile = T.b; tile < n_tiles; tile += T.nb) {
    const int p0 = tile * MLP_LOOP_TILE;
    const int rows = n_ve - p0 < MLP_LOOP_TILE ? n_ve - p0 : MLP_LOOP_TILE;
#pragma unroll
    for (int rr = 0; rr < MLP_LOOP_TILE; rr += 16) {
      const int row = rr + (threadIdx.x >> 4);
      float f2[2] = {0.0f, 0.0f};
      if (row < rows) node_feature_pair(P, P.ve[p0 + row], q, f2);
      const uint32_t v2 = pack_bf16(f2[0], f2[1]);
      *reinterpret_cast<uint32_t*>(sX + row * MLP_XS + 2 * q) = v2;
      if (row < rows) *reinterpret_cast<uint32_t*>(P.feat + (size_t)(p0 + row) * 32 + 2 * q) = v2;
    }
    __syncthreads();
    if (P.mix_thr)
      mlp_tile_forward<MLP_LOOP_TILE / 16, true>(w, sX, sH, P.net_raw, p0, rows, nullptr, nullptr);
    __syncthreads();
  }
}

// Standard normals z[0..3] from four Philox words (Box-Muller, pairs of
// words: radius from the first, angle from the second).
__device__ __forceinline__ void box_muller4(uint4 w, float* z) {
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const float r1 = (float)((ws[2 * pr] >> 8) + 1u) * 5.9604644775390625e-08f;  // (0, 1]
    const float r2 = (float)(ws[2 * pr + 1] >> 8) * 5.9604644775390625e-08f;     // [0, 1)
    const float rad = sqrtf(-2.0f * logf(r1));
    float s, c;
    sincospif(2.0f * r2, &s, &c);
    z[2 * pr] = rad * c;
    z[2 * pr + 1] = rad * s;
  }
}

// The draw of sample key (V_E position p = key / lam, j = key - p lam) in
// pass it (Algorithm 2: random control in U, random duration): returns the
// parent's node id.  Counter (it, node, j, purpose): purpose 0 the control
// words (kept in wr), purpose 1 (duration, accept word, selector); with a
// network attached and the selector below the mix threshold, the control
// comes from the node's Gaussian with normals from purpose 3 (the duration
// keeps the uniform draw).
// The expand phase and the node-set phase (which appends accepted samples
// by their keys) both draw through this function, so both see the same
// numbers.
template <int SYS>
__device__ __forceinline__ int draw_controls(const KParams& P, uint32_t it, int key, int lam,
                                             float* u, int* k, uint32_t* wacc, uint32_t* wr) {
  constexpr int N = System<SYS>::N;
  const int p = key / lam;
  const int j = key - p * lam;
  const int v = KP_IDX(P, P.ve[KP_IDX(P, p, P.t_e, 5)], P.t_e, 6);
  const uint4 w0 = philox4x32_10(make_uint4(it, (uint32_t)v, (uint32_t)j, 0u), P.seed_lo, P.seed_hi);
  const uint4 w1 = philox4x32_10(make_uint4(it, (uint32_t)v, (uint32_t)j, 1u), P.seed_lo, P.seed_hi);
  wr[0] = w0.x; wr[1] = w0.y; wr[2] = w0.z; wr[3] = w0.w;
#pragma unroll
  for (int d = 0; d < N; ++d) u[d] = __fmaf_rn(P.u_scale[d], unit24(wr[d]), P.u_lo[d]);
  *k = P.k_min + (int)__umulhi(w1.x, P.k_span);
  if (w1.z < P.mix_thr) {
    // learned draw from the node's Gaussian (normals: purpose 3)
    const uint4 w3 = philox4x32_10(make_uint4(it, (uint32_t)v, (uint32_t)j, 3u), P.seed_lo, P.seed_hi);
    float z[4], mean[MLP_NQ], ls[MLP_NQ], q[4];
    box_muller4(w3, z);
    mlp_heads(P.net_raw + (size_t)p * MLP_OUT, mean, ls);
#pragma unroll
    for (int d = 0; d < N; ++d) q[d] = fminf(fmaxf(__fmaf_rn(expf(ls[d]), z[d], mean[d]), -1.0f), 1.0f);
#pragma unroll
    for (int d = 0; d < N; ++d)
      u[d] = __fmaf_rn(P.u_scale[d], __fmul_rn(__fadd_rn(q[d], 1.0f), 0.5f), P.u_lo[d]);
  }
  *wacc = w1.y;
  return v;
}

// The draw of sample 'key' and its parent's state (the start of the
// segment).
template <int SYS>
__device__ __forceinline__ int draw_sample(const KParams& P, uint32_t it, int key, int lam, float* x,
                                           float* u, int* k, uint32_t* wacc, uint32_t* wr) {
  constexpr int D = System<SYS>::D;
  const int v = draw_controls<SYS>(P, it, key, lam, u, k, wacc, wr);
#pragma unroll
  for (int d = 0; d < D; ++d) x[d] = P.st[(size_t)d * P.t_e + v];
  return v;
}

// Phase E: Algorithm 2 for every sample key in [0, S).
//
// Lanes integrate step by step and are refilled as they finish: a warp
// takes keys in batches from a grid-wide counter, every lane carries one
// sample (k steps, or fewer when a step is invalid), and when enough lanes
// of the warp have finished they are finalised (binning, counters, claim,
// flags) and given new keys together, so that the divergent finalise /
// start-up work is shared by many lanes and no lane idles while a long
// sample runs next to it.  Every sample's arithmetic depends on its key
// alone, so the result does not depend on which lane ran it.
constexpr int KP_KEY_BATCH = 128; // keys a warp takes from the grid counter

template <int SYS, bool LOG>
__device__ __forceinline__ void phase_expand(const KParams& P, const Team& T,
                                             const unsigned char* sblob, uint32_t it, int lam,
                                             int S, LoopShared& sh) {
  using Sys = System<SYS>;
  constexpr int D = Sys::D, N = Sys::N;
  const float4* sbox = reinterpret_cast<const float4*>(sblob);
  const uint16_t* sstart = reinterpret_cast<const uint16_t*>(sblob + P.bp_start_off);
  const uint16_t* sids = reinterpret_cast<const uint16_t*>(sblob + P.bp_ids_off);
  const uint8_t* sclear = P.bp_clear_off >= 0 ? sblob + P.bp_clear_off : nullptr;
  const uint32_t FULL = 0xffffffffu;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;

  // per-thread counts of one pass: a thread runs at most 2^28 / 256 keys of
  // at most 255 steps each, so 32 bits hold them; n_refill counts the keys
  // a lane starts after its first one, n_batch (lane 0) the batches its
  // warp takes from the grid counter
  uint32_t n_steps = 0, n_hull = 0, n_box = 0, n_refill = 0, n_batch = 0;
  bool ran = false;
  // lane state: the sample being integrated
  int key = -1, v = 0, k = 0, i = 0, fail = 0;
  bool done = false;
  float x[D], u[N];
  uint32_t wacc = 0, wr[4] = {0, 0, 0, 0};
  // warp state (uniform): the current batch of keys.  The first batch of
  // every warp is fixed by the warp's index (keys [gw b0, (gw + 1) b0), the
  // size the live sizing below gives at the start of a pass), so no warp
  // queues on the counter to start; later batches come from the counter,
  // offset past the statically handed-out keys.
  const int n_warps = T.nb * (int)(blockDim.x >> 5);
  const int gw = T.b * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
  int b0 = S / (2 * n_warps);
  b0 = b0 < Sys::FIRST_BATCH_MIN ? Sys::FIRST_BATCH_MIN : (b0 > KP_KEY_BATCH ? KP_KEY_BATCH : b0);
  const int static_end = n_warps * b0 < S ? n_warps * b0 : S;
  int pool_next = gw * b0 < S ? gw * b0 : S;
  int pool_end = pool_next + b0 < S ? pool_next + b0 : S;
  bool exhausted = S <= 0;
  // bound on the phase's device time, checked warp-uniformly at every
  // refill (a sample runs at most 255 steps, so refills are at most 255
  // iterations apart)
  const uint64_t t_phase = global_ns();

  for (;;) {
    // finished lanes are finalised together: REFILL_MIN of them while keys
    // remain (they are refilled at once), and once the pass's keys are all
    // handed out, only when every lane has finished, so that the warp's
    // last samples cost one finalise instead of one per finishing step
    const uint32_t m_free = __ballot_sync(FULL, key < 0 || done);
    if (exhausted ? m_free == FULL : __popc(m_free) >= Sys::REFILL_MIN) {
      const uint64_t now = __shfl_sync(FULL, global_ns(), 0);
      if (now - t_phase > P.wait_ns) {
        if (lane == 0) raise_error(P.ctl, KP_DEV_ERR_TIMEOUT, 30);
        break;
      }
      // ---- finalise the lanes that finished -------------------------------
      if (key >= 0 && done) {
        // steps run, and hull tests (every step but one that left the
        // state box)
        n_steps += (uint32_t)i;
        n_hull += (uint32_t)(fail < 0 ? i - 1 : i);
        int r, s;
        bin_state<SYS>(x, P, &r, &s, sblob);
        const bool valid = fail == 0;
        uint32_t f = 0;
        if (valid) {
          r = KP_IDX(P, r, P.R, 7);
          s = KP_IDX(P, s, (long long)P.R * P.n_sub_per, 8);
          key = KP_IDX(P, key, P.t_e, 9);
          atomicAdd(&P.n_valid[r], 1u);
          f = KP_F_VALID;
          const bool cont = P.visited[s] == 0;
          const bool bern = (uint64_t)wacc < P.thr[r];
          bool may_win = false;
          if (cont) {
            f |= KP_F_CONTENDER;
            // the first claimant of a sub-region knows it is newly reached:
            // it will get exactly one representative in region r; a
            // claimant that finds a smaller key there has already lost
            const uint32_t prev = atomicMin(&P.claim[s], (uint32_t)key);
            if (prev == 0xffffffffu) {
              atomicAdd(&P.cov[r], 1u);
              P.avail[r] = 1;
            }
            may_win = prev > (uint32_t)key;
          }
          if (bern) {
            f |= KP_F_BERN;
            P.avail[r] = 1;
          }
          // a sample that may still be accepted (a contender not yet beaten,
          // or past its draw) keeps its end state for the append, and a
          // contender its sub-region for the claim check
          if (cont) P.cs[key] = s;
          if (may_win || bern) {
            float4* row = reinterpret_cast<float4*>(P.xs + (size_t)key * kp_xs_stride(D));
#pragma unroll
            for (int q = 0; q < kp_xs_stride(D) / 4; ++q)
              row[q] = make_float4(4 * q < D ? x[4 * q] : 0.0f, 4 * q + 1 < D ? x[4 * q + 1] : 0.0f,
                                   4 * q + 2 < D ? x[4 * q + 2] : 0.0f,
                                   4 * q + 3 < D ? x[4 * q + 3] : 0.0f);
          }
        } else {
          atomicAdd(&P.n_invalid[KP_IDX(P, r, P.R, 10)], 1u);
        }
        P.flags[KP_IDX(P, key, P.t_e, 11)] = (uint8_t)f;
        if (LOG && key < P.log.capacity) {
          P.log.node[key] = v;
          P.log.k[key] = k;
#pragma unroll
          for (int d = 0; d < 4; ++d) P.log.uraw[4 * (size_t)key + d] = wr[d];
          P.log.fail_step[key] = fail < 0 ? -fail : fail;
          P.log.region[key] = r;
          P.log.sub[key] = s;
#pragma unroll
          for (int d = 0; d < 12; ++d) P.log.state[12 * (size_t)key + d] = d < D ? x[d] : 0.0f;
        }
        key = -1;
      }
      // ---- hand new keys to the free lanes --------------------------------
      uint32_t m_idle = __ballot_sync(FULL, key < 0);
      while (m_idle && !exhausted) {
        if (pool_next >= pool_end) {
          // batches shrink towards the end of the pass so that warps run
          // out of work together
          // (at the very end a warp takes only what its idle lanes can
          // start now, so no warp is left with a second round of samples)
          // (the batch is sized from the counter's current value: a warp
          // that last took keys long ago must not size it from a stale
          // position and leave with a large batch just before the end)
          const int n_idle_now = __popc(m_idle);
          int base = S;
          if (lane == 0 && static_end < S) {
            const int cur = static_end + *((volatile int*)&P.ctl->work_next);
            int want = (S - cur) / (Sys::GUIDED_DIV * n_warps);
            want = want < n_idle_now ? n_idle_now : (want > KP_KEY_BATCH ? KP_KEY_BATCH : want);
            base = static_end + atomicAdd(&P.ctl->work_next, want);
            base = base < S ? base : S;
            n_batch += base < S ? 1u : 0u;
            pool_end = base + want < S ? base + want : S;
          }
          base = __shfl_sync(FULL, base, 0);
          const int end_now = __shfl_sync(FULL, pool_end, 0);
          if (base >= S) {
            exhausted = true;
            break;
          }
          pool_next = base;
          pool_end = end_now;
        }
        const int avail = pool_end - pool_next;
        const int rank = __popc(m_idle & lt);
        if (key < 0 && rank < avail) {
          key = pool_next + rank;
          n_refill += ran ? 1u : 0u;
          ran = true;
          v = draw_sample<SYS>(P, it, key, lam, x, u, &k, &wacc, wr);
          i = 0;
          fail = 0;
          done = false;
        }
        const int n_idle = __popc(m_idle);
        pool_next += n_idle < avail ? n_idle : avail;
        m_idle = __ballot_sync(FULL, key < 0);
      }
      if (__ballot_sync(FULL, key >= 0) == 0) break;
    }
    // ---- one integrator step (PropagateODE) and its validity check --------
    if (key >= 0 && !done) {
      const float px = x[0], py = x[1], pz = x[2];
      Sys::step(x, u, P.dt, P);
      ++i;
      const bool inbox = in_state_box<D>(x, P);
      bool ok = inbox;
      if (inbox) {
        // hull of the step; + 0.0f turns a -0 into +0 for the box test
        ok = !hull_hits_grid(P, sbox, sstart, sids, sclear, fminf(px, x[0]) + 0.0f,
                             fminf(py, x[1]) + 0.0f, fminf(pz, x[2]) + 0.0f,
                             fmaxf(px, x[0]) + 0.0f, fmaxf(py, x[1]) + 0.0f,
                             fmaxf(pz, x[2]) + 0.0f, &n_box);
      }
      if (!ok) {
        done = true;
        fail = inbox ? i : -i;  // negative: the end state left the state box
      } else if (i >= k) {
        done = true;
      }
    }
  }
  unsigned long long bs, bh, bb, brf, bbt, dummy;
  block_sum2((unsigned long long)n_steps, (unsigned long long)n_hull, sh.red, &bs, &bh);
  block_sum2((unsigned long long)n_box, (unsigned long long)n_refill, sh.red, &bb, &brf);
  block_sum2((unsigned long long)n_batch, 0, sh.red, &bbt, &dummy);
  if (threadIdx.x == 0 && bs) {
    atomicAdd(&P.ctl->tot_steps, bs);
    atomicAdd(&P.ctl->tot_hull, bh);
    atomicAdd(&P.ctl->tot_box_tests, bb);
    if (brf) atomicAdd(&P.ctl->tot_refills, brf);
    if (bbt) atomicAdd(&P.ctl->tot_batches, bbt);
  }
}

// Contiguous key range [a, b) of warp w >= 1 inside the block's chunk
// [c0, c1) (warp 0 runs the region estimates and gets none).
__device__ __forceinline__ void warp_range(int c0, int c1, int* a, int* b) {
  const int nw = (int)(blockDim.x >> 5) - 1;
  const int w = (int)(threadIdx.x >> 5) - 1;
  if (w < 0) {
    *a = *b = c0;
    return;
  }
  const int per = (c1 - c0 + nw - 1) / nw;
  const long long lo = (long long)c0 + (long long)w * per;
  *a = (int)(lo < c1 ? lo : c1);
  *b = (int)(lo + per < c1 ? lo + per : c1);
}

// Phase A (warps 1..): accept decisions of this block's key chunk.  Each
// warp walks its own key range in tiles of 32 x KP_ACC_KPL keys (lane l
// takes keys t0 + 32q + l: every load is coalesced), with the loads of a
// tile's flags, contenders' sub-regions and their claims issued together,
// and compacts its accepted keys (claim winners marked in bit 31) in key
// order at the start of its range in acc_key.  Phase S (warp 0) runs
// alongside.  Publishes the block's accepted count, adds the valid count to
// the pass, and leaves where each warp's accepted keys are, and their
// offsets among the block's, in shared memory for the node-set phase.
constexpr int KP_ACC_KPL = 8;

__device__ __forceinline__ void phase_scores(const KParams& P, const Team& T, int nch, double* sd);

template <bool LOG>
__device__ __forceinline__ void phase_accept(const KParams& P, const Team& T, int S, int nch,
                                             double* sd, LoopShared& sh) {
  if (threadIdx.x < 32) phase_scores(P, T, nch, sd);
  const uint32_t FULL = 0xffffffffu;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  int k0, k1, a, b;
  chunk_of(T, S, &k0, &k1);
  warp_range(k0, k1, &a, &b);
  int n_acc = 0;
  uint32_t n_valid = 0;
  for (int t0 = a; t0 < b; t0 += 32 * KP_ACC_KPL) {
    uint32_t f[KP_ACC_KPL], c[KP_ACC_KPL];
    int s[KP_ACC_KPL];
#pragma unroll
    for (int q = 0; q < KP_ACC_KPL; ++q) {
      const int key = t0 + 32 * q + (int)lane;
      f[q] = key < b ? P.flags[key] : 0u;
    }
#pragma unroll
    for (int q = 0; q < KP_ACC_KPL; ++q)
      s[q] = (f[q] & KP_F_CONTENDER) ? P.cs[KP_IDX(P, t0 + 32 * q + (int)lane, P.t_e, 12)] : 0;
#pragma unroll
    for (int q = 0; q < KP_ACC_KPL; ++q)
      c[q] = (f[q] & KP_F_CONTENDER)
                 ? P.claim[KP_IDX(P, s[q], (long long)P.R * P.n_sub_per, 13)]
                 : 0u;
#pragma unroll
    for (int q = 0; q < KP_ACC_KPL; ++q) {
      const int key = t0 + 32 * q + (int)lane;
      const bool valid = (f[q] & KP_F_VALID) != 0;
      n_valid += valid ? 1u : 0u;
      const bool win = (f[q] & KP_F_CONTENDER) && c[q] == (uint32_t)key;
      const bool acc = valid && (win || (f[q] & KP_F_BERN));
      const uint32_t m = __ballot_sync(FULL, acc);
      if (acc)
        P.acc_key[KP_IDX(P, a + n_acc + __popc(m & lt), P.t_e, 14)] =
            (uint32_t)key | (win ? 0x80000000u : 0u);
      n_acc += __popc(m);
      if (LOG && key < b && key < P.log.capacity)
        P.log.flags[key] =
            (uint8_t)(f[q] | (win ? KP_F_WINNER : 0u) | (acc ? KP_F_ACCEPTED : 0u));
    }
  }
  // warp counts -> offsets in key order (warps own ascending ranges)
  const int w = (int)(threadIdx.x >> 5);
  if (lane == 0) sh.scan.warp[w] = n_acc;
  __syncthreads();
  int off = 0, block_acc = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    const int cq = sh.scan.warp[q];
    off += q < w ? cq : 0;
    block_acc += cq;
  }
  if (lane == 0) {
    sh.acc_a[w] = a;
    sh.acc_n[w] = n_acc;
    sh.acc_off[w] = off;
  }
  if (threadIdx.x == 0) sh.acc_tot = block_acc;
  unsigned long long bv, dummy;
  block_sum2((unsigned long long)n_valid, 0, sh.red, &bv, &dummy);
  if (threadIdx.x == 0) {
    if (T.b == 0) P.ctl->work_next = 0;  // the expand phase is over
    P.blk_a[KP_IDX(P, T.b, KP_MAX_GRID, 15)] = (uint32_t)block_acc;
    if (bv) atomicAdd(&P.ctl->it_valid, (uint32_t)bv);
  }
}

// Pairwise sum of buf[0..n), n a power of two, by one warp (bottom-up
// tree, the same tree as recursive halving); result in buf[0].
__device__ __forceinline__ void warp_pairwise(double* buf, int n) {
  const int lane = (int)(threadIdx.x & 31u);
  for (int stride = 1; stride < n; stride <<= 1) {
    __syncwarp();
    for (int i = lane * 2 * stride; i < n; i += 64 * stride)
      buf[i] = __dadd_rn(buf[i], buf[i + stride]);
  }
  __syncwarp();
}

// The same tree for n <= 32 KP_TREE_PER_LANE, in registers: lane l loads
// the m = max(n / 32, 1) values l m .. l m + m - 1 through load(i), adds
// the tree's levels of stride below m in place, and the levels of stride m,
// 2m, ... across lanes by shuffles (left operand the lower index, as in
// the shared-memory tree).  Every lane gets the sum.  No shared memory and
// no warp barrier per level.
constexpr int KP_TREE_PER_LANE = 8;

template <class L>
__device__ __forceinline__ double warp_tree_sum(int n, L load) {
  const int lane = (int)(threadIdx.x & 31u);
  const int m = n >= 32 ? n >> 5 : 1;
  double v[KP_TREE_PER_LANE];
#pragma unroll
  for (int q = 0; q < KP_TREE_PER_LANE; ++q) {
    const int i = lane * m + q;
    v[q] = q < m && i < n ? load(i) : 0.0;
  }
#pragma unroll
  for (int st = 1; st < KP_TREE_PER_LANE; st <<= 1)
#pragma unroll
    for (int q = 0; q + st < KP_TREE_PER_LANE; q += 2 * st)
      if (st < m) v[q] = __dadd_rn(v[q], v[q + st]);
  double sum = v[0];
  const int lanes = n / m;
  for (int d = 1; d < lanes; d <<= 1) {
    const double o = __shfl_down_sync(0xffffffffu, sum, d);
    if ((lane & (2 * d - 1)) == 0) sum = __dadd_rn(sum, o);
  }
  return __shfl_sync(0xffffffffu, sum, 0);
}

// Phase S (warp 0): Eq. 3-4 for this block's region chunk and its pairwise
// partial sum (published before the grid barrier that ends the phase).
// Every operation is an explicitly rounded IEEE double operation in the
// order
// FreeVol = ((delta + nv) vol) / ((delta + nv) + ni),
// f4 = (FreeVol FreeVol)(FreeVol FreeVol),
// Score = f4 / ((1 + Cov)(1 + (nv + ni)(nv + ni))).
__device__ __forceinline__ void phase_scores(const KParams& P, const Team& T, int nch, double* sd) {
  if (T.b >= nch) return;
  const int lane = (int)(threadIdx.x & 31u);
  const int ch = P.R_pad / nch;
  const int r0 = T.b * ch;
  for (int i = lane; i < ch; i += 32) {
    const int r = r0 + i;
    double sc = 0.0;
    if (r < P.R && P.avail[r]) {
      const double nv = (double)P.n_valid[r], ni = (double)P.n_invalid[r];
      const double dn = __dadd_rn(P.delta, nv);
      const double vol = P.region_vol ? P.region_vol[r] : P.vol;
      const double fv = __ddiv_rn(__dmul_rn(dn, vol), __dadd_rn(dn, ni));
      const double f2 = __dmul_rn(fv, fv);
      const double f4 = __dmul_rn(f2, f2);
      const double na = __dadd_rn(nv, ni);
      const double den =
          __dmul_rn(__dadd_rn(1.0, (double)P.cov[r]), __dadd_rn(1.0, __dmul_rn(na, na)));
      sc = __ddiv_rn(f4, den);
    }
    if (r < P.R) P.score[r] = sc;
    sd[i] = sc;
  }
  double part;
  if (ch <= 32 * KP_TREE_PER_LANE) {
    __syncwarp();
    part = warp_tree_sum(ch, [&](int i) { return sd[i]; });
  } else {
    warp_pairwise(sd, ch);
    part = sd[0];
  }
  if (lane == 0) P.chunk_sum[KP_IDX(P, T.b, KP_MAX_GRID, 16)] = part;
  __syncwarp();
}

// Phase T (warp 0 of the node-set phase): the sum of Eq. 5 from the chunks'
// partial sums (every chunk's warp reduces them itself, in the same
// pairwise tree, so all get the same value), then P_accept and the integer
// threshold of this block's region chunk.
__device__ __forceinline__ void phase_thresholds(const KParams& P, const Team& T, int nch,
                                                 double* sd) {
  if (T.b >= nch) return;
  const int lane = (int)(threadIdx.x & 31u);
  double sum;
  if (nch <= 32 * KP_TREE_PER_LANE) {
    sum = warp_tree_sum(nch, [&](int i) { return __ldcg(P.chunk_sum + i); });
  } else {
    for (int i = lane; i < nch; i += 32) sd[i] = __ldcg(P.chunk_sum + i);
    warp_pairwise(sd, nch);
    sum = sd[0];
  }
  if (T.b == 0 && lane == 0) P.ctl->score_sum = sum;
  const int ch = P.R_pad / nch;
  const int r0 = T.b * ch;
  for (int i = (int)(threadIdx.x & 31u); i < ch; i += 32) {
    const int r = r0 + i;
    if (r >= P.R) break;
    uint64_t thr = 1ull << 32;  // P_accept = 1 outside R_avail
    if (P.avail[r]) {
      double p;
      if (sum > 0.0) {
        p = __dadd_rn(__ddiv_rn(P.score[r], sum), P.eps);
        if (p > 1.0) p = 1.0;
      } else {
        p = P.eps < 1.0 ? P.eps : 1.0;
      }
      if (p < 1.0) thr = (uint64_t)floor(__dmul_rn(p, 4294967296.0));
    }
    P.thr[r] = thr;
  }
}

// Materialises this block's accepted samples as the nodes id0 .. id0 +
// acc_tot - 1 (id0 = t_old + the accepted samples of the blocks before it:
// node ids follow the sample keys).  Every accepted sample takes the end
// state the expand phase kept for it, its parent, control and duration
// from its key (the same draw), and its region and sub-region; visited and
// the goal test (closed ball on position; the smallest new goal node wins)
// follow.  Thread j of the block takes the block's samples j, j +
// blockDim.x, ...; consecutive threads write consecutive nodes.  With the
// sample log on, the sample is also re-derived from its key (the same
// integrator steps, explicitly rounded, so the same numbers) and must match
// the kept and the logged state bit for bit.
template <int SYS, bool LOG>
__device__ __forceinline__ void materialise(const KParams& P, uint32_t it, int id0, int lam,
                                            const LoopShared& sh, const unsigned char* sblob) {
  using Sys = System<SYS>;
  constexpr int D = Sys::D, N = Sys::N;
  for (int j = (int)threadIdx.x; j < sh.acc_tot; j += (int)blockDim.x) {
    int w = 0;
#pragma unroll
    for (int q = 0; q < KP_WARPS; ++q)
      if (j >= sh.acc_off[q] && j < sh.acc_off[q] + sh.acc_n[q]) w = q;
    const uint32_t e = P.acc_key[KP_IDX(P, sh.acc_a[w] + (j - sh.acc_off[w]), P.t_e, 17)];
    const int key = KP_IDX(P, (int)(e & 0x7fffffffu), P.t_e, 18);
    const int id = KP_IDX(P, id0 + j, P.t_e, 19);
    float x[D], u[N];
    int k;
    uint32_t wacc, wr[4];
    const int v = draw_controls<SYS>(P, it, key, lam, u, &k, &wacc, wr);
    {
      const float4* row = reinterpret_cast<const float4*>(P.xs + (size_t)key * kp_xs_stride(D));
#pragma unroll
      for (int q = 0; q < (D + 3) / 4; ++q) {
        const float4 c = row[q];
        if (4 * q < D) x[4 * q] = c.x;
        if (4 * q + 1 < D) x[4 * q + 1] = c.y;
        if (4 * q + 2 < D) x[4 * q + 2] = c.z;
        if (4 * q + 3 < D) x[4 * q + 3] = c.w;
      }
    }
    int r, s;
    bin_state<SYS>(x, P, &r, &s, sblob);
    r = KP_IDX(P, r, P.R, 20);
    s = KP_IDX(P, s, (long long)P.R * P.n_sub_per, 21);
#pragma unroll
    for (int d = 0; d < D; ++d) P.st[(size_t)d * P.t_e + id] = x[d];
#pragma unroll
    for (int d = 0; d < N; ++d) P.ctrl[(size_t)d * P.t_e + id] = u[d];
    P.steps[id] = (uint8_t)k;
    P.parent[id] = v;
    P.region[id] = r;
    P.node_sub[id] = s;
    P.in_ve[id] = 1;
    P.visited[s] = 1;
    const float dx = __fsub_rn(x[0], P.goal_c[0]), dy = __fsub_rn(x[1], P.goal_c[1]),
                dz = __fsub_rn(x[2], P.goal_c[2]);
    const bool goal = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) <= P.goal_r2;
    if (goal) atomicMin(&P.ctl->goal_node, id);
    if (P.hv_cap > 0 && (e & 0x80000000u)) {
      // training pair: the parent's features and this sample's draw
      const uint32_t h = atomicAdd(P.hv_count, 1u);
      if (h < (uint32_t)P.hv_cap) {
        const __nv_bfloat16* fr =
            reinterpret_cast<const __nv_bfloat16*>(P.feat) + (size_t)(key / lam) * 32;
        for (int c = 0; c < 32; ++c) P.hv_feat[(size_t)h * 32 + c] = __bfloat162float(fr[c]);
#pragma unroll
        for (int d = 0; d < 3; ++d)
          P.hv_target[(size_t)h * 4 + d] = 2.0f * (u[d] - P.u_lo[d]) / P.u_scale[d] - 1.0f;
        P.hv_target[(size_t)h * 4 + 3] =
            P.k_span > 1 ? 2.0f * (float)(k - P.k_min) / (float)(P.k_span - 1) - 1.0f : 0.0f;
      }
    }
    if (LOG && key < P.log.capacity) {
      if (goal) P.log.flags[key] |= (uint8_t)KP_F_GOAL;
      float y[D];
#pragma unroll
      for (int d = 0; d < D; ++d) y[d] = P.st[(size_t)d * P.t_e + v];
      for (int st = 0; st < k; ++st) Sys::step(y, u, P.dt, P);
      bool same = P.log.region[key] == r && P.log.sub[key] == s;
#pragma unroll
      for (int d = 0; d < D; ++d)
        same = same && __float_as_uint(P.log.state[12 * (size_t)key + d]) == __float_as_uint(x[d]) &&
               __float_as_uint(y[d]) == __float_as_uint(x[d]);
      if (!same) raise_error(P.ctl, KP_DEV_ERR_REPLAY, 40);
    }
  }
}

// Phase N: Algorithm 4 node sets, one draw per old node (counter: it, v, 0,
// purpose 2) against the threshold of its region; new nodes are in V_E.
// Publishes the block chunk's V_E count; returns in *n_new the number of
// accepted samples of the pass (the new nodes).
// Order inside the phase: warp 0 of every region-chunk block first writes
// its chunk's thresholds (phase T) and counts itself done; every block then
// appends its own accepted samples (ids from t_old, in key order), which
// needs no threshold; then it waits (bounded) until every chunk is done and
// makes the node-set draws.  New nodes are counted as V_E members without
// reading their sets.
template <int SYS, bool LOG>
__device__ __forceinline__ void phase_nodesets(const KParams& P, const Team& T, uint32_t it,
                                               int t_old, int lam, LoopShared& sh, int* n_new,
                                               const unsigned char* sblob, double* sd) {
  const int nch = P.nch;
  if (threadIdx.x < 32 && T.b < nch) {
    phase_thresholds(P, T, nch, sd);
    __threadfence();
    __syncwarp();
    if (threadIdx.x == 0) atomicAdd(&P.ctl->t_done, 1u);
  }
  unsigned long long acc_before, acc_total;
  block_prefix(T, P.blk_a, sh, &acc_before, &acc_total);
  *n_new = (int)acc_total;
  const int t_new = t_old + (int)acc_total;
  materialise<SYS, LOG>(P, it, t_old + (int)acc_before, lam, sh, sblob);
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (ld_acquire(&P.ctl->t_done) < (uint32_t)nch) {
      if ((++spins & 63u) == 0) {
        if (*((volatile int*)&P.ctl->err) != 0) break;
        if (global_ns() - t0 > P.wait_ns) {
          raise_error(P.ctl, KP_DEV_ERR_TIMEOUT, 25);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  int v0, v1;
  chunk_of(T, t_new, &v0, &v1);
  // old nodes of the chunk: four tiles at a time, their region and
  // threshold loads issued together
  const int o1 = v1 < t_old ? v1 : t_old;
  const int stride = (int)blockDim.x;
  int c = 0;
  for (int t0 = v0; t0 < o1; t0 += 4 * stride) {
    int vq[4], rq[4];
    uint64_t tq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      vq[q] = t0 + q * stride + (int)threadIdx.x;
      rq[q] = vq[q] < o1 ? KP_IDX(P, __ldcg(P.region + KP_IDX(P, vq[q], P.t_e, 22)), P.R, 23) : 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) tq[q] = vq[q] < o1 ? __ldcg(P.thr + rq[q]) : 0ull;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (vq[q] < o1) {
        const uint4 w =
            philox4x32_10(make_uint4(it, (uint32_t)vq[q], 0u, 2u), P.seed_lo, P.seed_hi);
        const int e = (uint64_t)w.x < tq[q] ? 1 : 0;
        P.in_ve[vq[q]] = (uint8_t)e;
        c += e;
      }
    }
  }
  // new nodes are V_E members (their flags are set by the blocks that
  // appended them, so they are counted, not read)
  const int new0 = v0 > t_old ? v0 : t_old;
  const int tot = block_sum(c, sh) + (v1 > new0 ? v1 - new0 : 0);
  if (threadIdx.x == 0) P.blk_b[KP_IDX(P, T.b, KP_MAX_GRID, 24)] = (uint32_t)tot;
}

// The loop of one query (Algorithm 1 body, repeated) run by a team of
// blocks, with the query's obstacle blob already in shared memory.  Stops
// when a goal node is appended, Eq. 6 gives lambda = 0, or the pass or time
// budget is spent.  Returns false when a bounded wait expired.
template <int SYS, bool LOG>
__device__ __forceinline__ bool run_loop(const KParams& P, const Team& T, unsigned char* smem,
                                         LoopShared& sh, int max_iters, uint64_t max_ns) {
  double* sd = reinterpret_cast<double*>(smem + (size_t)P.blob_bytes);
  KCtl* ctl = P.ctl;
  const uint64_t t_start = global_ns();
  if (T.b == 0 && threadIdx.x == 0) {
    ctl->it_valid = 0;
    ctl->stop = 0;
    ctl->n_run = 0;
    ctl->work_next = 0;
    ctl->t_done = 0;
  }
  // the loop state, read once per block
  if (threadIdx.x == 0) {
    sh.bcast[0] = ctl->n_nodes;
    sh.bcast[1] = ctl->iteration;
  }
  __syncthreads();
  int n_tree = sh.bcast[0];
  uint32_t it = (uint32_t)sh.bcast[1];
  const int nch = P.nch;

  // V_E list from the stored node sets
  count_ve(P, T, n_tree, sh);
  if (!team_sync(T, ctl, P.wait_ns, 10)) return false;
  int n_ve = write_ve(P, T, n_tree, sh);
  if (!team_sync(T, ctl, P.wait_ns, 11)) return false;
  int lam = eq6_lambda(P.t_e, n_tree, n_ve, P.lambda_max);
  if (n_ve > 0 && lam == 0) {
    if (T.b == 0 && threadIdx.x == 0) {
      ctl->state = KP_DEV_FULL;
      ctl->n_ve = n_ve;
    }
    return true;
  }

  int run = 0;
  // block 0 stamps the device clock between phases and barriers
  const bool timer = T.b == 0 && threadIdx.x == 0;
  uint64_t t_mark = timer ? global_ns() : 0;
  int32_t* phase_ns = sh.phase_ns;
  int32_t prev_wait = 0;
  auto stamp = [&](int ph) {
    if (timer) {
      const uint64_t now = global_ns();
      phase_ns[ph] = (int32_t)(now - t_mark);
      t_mark = now;
    }
  };
  unsigned char* mtile = smem + P.blob_bytes + P.sd_bytes;
  for (;;) {
    if (P.features_on) {
      phase_features(P, T, n_ve, mtile);
      stamp(3);
      if (!team_sync(T, ctl, P.wait_ns, 19)) return false;
      stamp(6);
    } else if (timer) {
      phase_ns[3] = phase_ns[6] = 0;
    }
    const int S = n_ve > 0 ? n_ve * lam : 0;
    phase_expand<SYS, LOG>(P, T, smem, it, lam, S, sh);
    stamp(0);
    if (!team_sync(T, ctl, P.wait_ns, 20)) return false;
    stamp(1);
    phase_accept<LOG>(P, T, S, nch, sd, sh);
    stamp(2);
    if (!team_sync(T, ctl, P.wait_ns, 21)) return false;
    stamp(4);
    if (timer) phase_ns[5] = phase_ns[7] = 0;
    const int t_old = n_tree;
    int n_acc;
    phase_nodesets<SYS, LOG>(P, T, it, t_old, lam, sh, &n_acc, smem, sd);
    n_tree = t_old + n_acc;
    stamp(8);
    if (!team_sync(T, ctl, P.wait_ns, 23)) return false;
    stamp(9);
    const int ve_prev = n_ve, lam_prev = lam;
    n_ve = write_ve(P, T, n_tree, sh);
    lam = eq6_lambda(P.t_e, n_tree, n_ve, P.lambda_max);
    ++run;
    if (T.b == 0 && threadIdx.x == 0) {
      const int goal = *((volatile int*)&ctl->goal_node);
      const bool solved = goal != KP_NO_GOAL;
      const bool full = n_ve > 0 && lam == 0;
      if (run <= P.stats_cap && P.stats) {
        KStats s;
        s.iteration = (int)it;
        s.n_ve = ve_prev;
        s.lambda = lam_prev;
        s.n_samples = S;
        s.n_valid = (int)*((volatile uint32_t*)&ctl->it_valid);
        s.n_accepted = n_acc;
        s.n_nodes = n_tree;
        s.goal_node = solved ? goal : -1;
        phase_ns[10] = (int32_t)(global_ns() - t_mark);
        phase_ns[11] = prev_wait;
        for (int q = 0; q < 12; ++q) s.phase_ns[q] = phase_ns[q];
        P.stats[run - 1] = s;
      }
      ctl->it_valid = 0;
      ctl->t_done = 0;  // every block is past its threshold wait
      ctl->tot_samples += (unsigned long long)S;
      const bool out_of_time = max_ns > 0 && global_ns() - t_start >= max_ns;
      ctl->state = solved ? KP_DEV_SOLVED : (full ? KP_DEV_FULL : KP_DEV_RUNNING);
      ctl->stop = (solved || full || run >= max_iters || out_of_time) ? 1 : 0;
    }
    ++it;
    const uint64_t t_l = timer ? global_ns() : 0;
    int stop;
    if (!team_sync(T, ctl, P.wait_ns, 24, &ctl->stop, &stop)) return false;
    if (timer) {
      t_mark = global_ns();
      prev_wait = (int32_t)(t_mark - t_l);  // reported with the next pass
    }
    if (stop) break;
  }
  if (T.b == 0 && threadIdx.x == 0) {
    ctl->n_nodes = n_tree;
    ctl->n_ve = n_ve;
    ctl->iteration = (int)it;
    ctl->n_run = run;
  }
  return true;
}

// n bytes at p set to the 16-byte pattern v, by 16-byte stores (every table
// slice of the arena starts on 256 bytes and is padded to a multiple of
// 256, so the last store stays inside the slice).
__device__ __forceinline__ void fill_slice(void* p, size_t n, uint4 v, size_t tid, size_t nth) {
  uint4* q = reinterpret_cast<uint4*>(p);
  const size_t n16 = (n + 15) / 16;
  for (size_t i = tid; i < n16; i += nth) q[i] = v;
}

template <int SYS>
__device__ void init_root(const KParams& P, const RootState& root, bool box_free);

// Whether the root's position lies in no obstacle box (closed boxes, the
// test the hull check makes with a hull of one point), by the whole block:
// thread t tests boxes t, t + blockDim.x, ...  Every thread of the block
// calls it and gets the answer.
__device__ __forceinline__ bool root_box_free(const KParams& P, const RootState& root) {
  const float4* gb = reinterpret_cast<const float4*>(P.boxes);
  const float px = root.x[0], py = root.x[1], pz = root.x[2];
  bool hit = false;
  for (int b = (int)threadIdx.x; b < P.n_boxes_pad; b += (int)blockDim.x) {
    const float4 bl = gb[2 * b], bh = gb[2 * b + 1];
    hit |= (px <= bh.x) & (bl.x <= px) & (py <= bh.y) & (bl.y <= py) & (pz <= bh.z) &
           (bl.z <= pz);
  }
  return __syncthreads_or(hit) == 0;
}

// The region and sub-region tables of Algorithm 1's initialisation, cleared
// by the whole team: visited 0, claims 2^32 - 1, counters 0, R_avail empty,
// P_accept = 1 as the threshold 2^32.
__device__ __forceinline__ void clear_tables(const KParams& P, size_t tid, size_t nth) {
  const size_t R = (size_t)P.R, n_sub = R * (size_t)P.n_sub_per;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  fill_slice(P.visited, n_sub, zero, tid, nth);
  fill_slice(P.claim, n_sub * 4, make_uint4(~0u, ~0u, ~0u, ~0u), tid, nth);
  fill_slice(P.n_valid, R * 4, zero, tid, nth);
  fill_slice(P.n_invalid, R * 4, zero, tid, nth);
  fill_slice(P.cov, R * 4, zero, tid, nth);
  fill_slice(P.avail, R, zero, tid, nth);
  fill_slice(P.thr, R * 8, make_uint4(0u, 1u, 0u, 1u), tid, nth);  // 2^32 each
}

// Algorithm 1's initialisation inside the loop launch: the team clears the
// tables, then block 0 writes the root (which also clears the control
// block's error word, so neither barrier here reads it).
template <int SYS>
__device__ __forceinline__ bool reset_in_launch(const KParams& P, const Team& T,
                                                const RootState& root) {
  clear_tables(P, (size_t)T.b * blockDim.x + threadIdx.x, (size_t)T.nb * blockDim.x);
  const bool box_free = T.b == 0 ? root_box_free(P, root) : false;
  if (!team_sync(T, P.ctl, P.wait_ns, 50, nullptr, nullptr, false)) return false;
  if (T.b == 0 && threadIdx.x == 0) init_root<SYS>(P, root, box_free);
  return team_sync(T, P.ctl, P.wait_ns, 51, nullptr, nullptr, false);
}

// Root-to-goal chain into P.traj rows (state 12, control 4, steps), root
// first; ctl->n_edges its length, -1 without a goal node (rows are written
// for at most KP_TRAJ_ROWS edges).  Run by every thread of one block:
// thread 0 walks the chain once from the goal and keeps the node ids in
// ids[0 .. cap), then the block writes the rows in parallel; a chain longer
// than cap is written by thread 0 on a second walk.
template <int SYS>
__device__ void extract_chain_block(const KParams& P, int* ids, int cap) {
  constexpr int D = System<SYS>::D, N = System<SYS>::N;
  KCtl* ctl = P.ctl;
  __shared__ int s_len;
  if (threadIdx.x == 0) {
    const int g = ctl->goal_node;
    int len = -1;
    if (g != KP_NO_GOAL && g >= 0 && g < P.t_e) {
      len = 0;
      for (int v = g; v > 0 && len <= P.t_e; v = P.parent[v]) {
        if (len < cap) ids[len] = v;
        ++len;
      }
    }
    ctl->n_edges = len;
    s_len = len;
  }
  __syncthreads();
  const int len = s_len;
  if (len <= 0 || len > KP_TRAJ_ROWS) return;
  auto write_row = [&](int row, int v) {
    float* out = P.traj + (size_t)row * 17;
#pragma unroll
    for (int i = 0; i < 12; ++i) out[i] = i < D ? P.st[(size_t)i * P.t_e + v] : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) out[12 + i] = i < N ? P.ctrl[(size_t)i * P.t_e + v] : 0.0f;
    out[16] = (float)P.steps[v];
  };
  if (len <= cap) {
    for (int e = (int)threadIdx.x; e < len; e += (int)blockDim.x) write_row(len - 1 - e, ids[e]);
  } else if (threadIdx.x == 0) {
    int row = len - 1;
    for (int v = ctl->goal_node; v > 0 && row >= 0; v = P.parent[v], --row) write_row(row, v);
  }
}

#ifndef KP_MIN_BLOCKS
#define KP_MIN_BLOCKS 1
#endif
// Single-query launch: the whole grid is one team.  mode: KP_LOOP_RESET
// runs Algorithm 1's initialisation from 'root' first, KP_LOOP_EXTRACT
// writes the root-to-goal chain after the passes (block 0, the ids kept in
// the dynamic shared memory the passes no longer use).
template <int SYS, bool LOG>
__global__ void __launch_bounds__(KP_BLOCK, KP_MIN_BLOCKS)
    kp_loop_kernel(KParams P, int max_iters, uint64_t max_ns, RootState root, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LoopShared sh;
  KCtl* ctl = P.ctl;
  const Team T{(int)blockIdx.x, (int)gridDim.x, &ctl->bar};
  if ((mode & KP_LOOP_RESET) && !reset_in_launch<SYS>(P, T, root)) return;
  if (ctl->state == KP_DEV_RUNNING) {
    if (!stage_boxes(P, reinterpret_cast<float4*>(smem), sh)) return;
    if (!run_loop<SYS, LOG>(P, T, smem, sh, max_iters, max_ns)) return;
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->n_run = 0;
  }
  if ((mode & KP_LOOP_EXTRACT) && blockIdx.x == 0) {
    __syncthreads();
    int cap = (int)(((size_t)P.blob_bytes + (size_t)P.sd_bytes) / 4);
    if (P.extract_cap > 0 && P.extract_cap < cap) cap = P.extract_cap;
    extract_chain_block<SYS>(P, reinterpret_cast<int*>(smem), cap);
  }
}

// Root of a query (thread 0): x_init checked (state box; box_free: no
// obstacle box contains it, root_box_free) and binned; tree, decomposition
// and control block set to Algorithm 1, initialisation.  Thresholds and
// cleared tables are the caller's.
template <int SYS>
__device__ void init_root(const KParams& P, const RootState& root, bool box_free) {
  using Sys = System<SYS>;
  constexpr int D = Sys::D;
  KCtl* ctl = P.ctl;
  float x[D];
  for (int i = 0; i < D; ++i) x[i] = root.x[i];
  bool ok = in_state_box<D>(x, P) && box_free;
  ctl->n_run = 0;
  ctl->stop = 0;
  ctl->it_valid = 0;
  ctl->err = 0;
  ctl->err_where = 0;
  ctl->iteration = 0;
  ctl->n_edges = 0;
  ctl->tot_samples = 0;
  ctl->tot_steps = 0;
  ctl->tot_hull = 0;
  ctl->tot_box_tests = 0;
  ctl->tot_batches = 0;
  ctl->tot_refills = 0;
  ctl->work_next = 0;
  if (!ok) {
    ctl->state = KP_DEV_BAD_ROOT;
    ctl->n_nodes = 0;
    ctl->n_ve = 0;
    ctl->goal_node = KP_NO_GOAL;
    return;
  }
  int r, s;
  bin_state<SYS>(x, P, &r, &s);
  for (int i = 0; i < D; ++i) P.st[(size_t)i * P.t_e] = x[i];
  for (int i = 0; i < Sys::N; ++i) P.ctrl[(size_t)i * P.t_e] = 0.0f;
  P.parent[0] = -1;
  P.steps[0] = 0;
  P.region[0] = r;
  P.node_sub[0] = s;
  P.in_ve[0] = 1;
  P.visited[s] = 1;
  P.cov[r] = 1;
  P.avail[r] = 1;
  ctl->n_nodes = 1;
  ctl->n_ve = 1;
  const float dx = x[0] - P.goal_c[0], dy = x[1] - P.goal_c[1], dz = x[2] - P.goal_c[2];
  const bool in_goal = dx * dx + dy * dy + dz * dz <= P.goal_r2;
  ctl->goal_node = in_goal ? 0 : KP_NO_GOAL;
  ctl->state = in_goal ? KP_DEV_SOLVED : KP_DEV_RUNNING;
}

// Algorithm 1, initialisation, as a launch of its own (kp_reset and the
// no-allocation entry): every block clears its share of the tables
// (clear_tables); the last block to finish (a counter taken after a fence)
// writes the root, so the root's table entries come after every clear.
template <int SYS>
__global__ void kp_reset_kernel(KParams P, RootState root) {
  clear_tables(P, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&P.ctl->reset_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  const bool box_free = root_box_free(P, root);
  if (threadIdx.x != 0) return;
  __threadfence();
  P.ctl->reset_done = 0;
  P.ctl->bar = 0;
  init_root<SYS>(P, root, box_free);
}

}  // namespace kp
