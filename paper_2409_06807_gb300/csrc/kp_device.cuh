// kp_device.cuh -- device-side building blocks of the GB300 Kino-PAX planner:
// launch parameters, the device control block, the Philox4x32-10 stream, the
// bounded grid barrier, block scans and the three systems' integrators.
#pragma once

#include <cstdint>

#include "kp_layout.h"

namespace kp {

// ---------------------------------------------------------------------------
// time and bounded waits
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Records the first error of a launch (0 -> code).
__device__ __forceinline__ void raise_error(KCtl* ctl, int code, int where) {
  if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_where = where;
}

// Array indices of the loop kernel.  In the bounds-checked build (KP_CHECK
// defined) an index outside [0, n) records KP_DEV_ERR_BOUNDS with its site
// and 0 is used in its place, so that no access leaves its array, nothing
// traps, and every block stops at its next barrier; the host reports the
// site.  Otherwise the index is used as it is.
#ifdef KP_CHECK
__device__ __forceinline__ long long kp_checked(KCtl* ctl, long long i, long long n, int site) {
  if (i >= 0 && i < n) return i;
  raise_error(ctl, KP_DEV_ERR_BOUNDS, site);
  return 0;
}
#define KP_IDX(P, i, n, site) ((int)kp_checked((P).ctl, (long long)(i), (long long)(n), (site)))
#else
#define KP_IDX(P, i, n, site) (i)
#endif

// A team of blocks that plans one query: block index within the team, team
// size, and the team's barrier word.  The single-query launch is one team
// of the whole grid; the server launch splits its grid into teams.
struct Team {
  int b, nb;
  uint32_t* bar;
};

// Barrier of a team of co-resident blocks (cooperative launch) on one word
// whose top bit is the phase.  Every block but the team's block 0 adds 1,
// block 0 adds 2^31 - (nb - 1): the arrivals sum to 2^31, so the top bit
// flips with the last arrival and the low 31 bits come back to 0, with no
// reset and no second word.  A block waits until the top bit differs from
// the one its own arrival saw.  The low bits start at 0 (the reset and
// import paths write the word) and stay below 2^31 while any arrival is
// out, so the bit cannot flip early.  Ordering: each arrival is a fence then
// a relaxed add, so the adds form one release sequence; the wait's acquire
// load that sees the flip synchronises with every block's fence, and the
// closing __syncthreads carries that to the block's other threads (a fence
// after the wait measured slower and adds nothing).  Every wait is bounded by 'limit_ns'
// of device time; on expiry the block records KP_ERR_TIMEOUT and all blocks
// leave at their next barrier (the word is then left mid-phase: a launch
// that timed out poisons its context).  Returns false when the launch must
// stop.  With 'watch' given, thread 0 also reads that word after the
// barrier and the block gets its value in *watched (one load per block
// instead of one per thread on a word every block reads).  With check_err
// false the wait ignores the control block's error word (the barriers
// around a launch's own initialisation, which clears that word).
__device__ __forceinline__ bool team_sync(const Team& T, KCtl* ctl, uint64_t limit_ns, int where,
                                          const int* watch = nullptr, int* watched = nullptr,
                                          bool check_err = true) {
  __shared__ int s_ok, s_watch;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t add = T.b == 0 ? 0x80000000u - (uint32_t)(T.nb - 1) : 1u;
    __threadfence();
    const uint32_t seen = atomicAdd(T.bar, add) & 0x80000000u;
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while ((ld_acquire(T.bar) & 0x80000000u) == seen) {
      if ((++spins & 63u) == 0) {
        if (check_err && *((volatile int*)&ctl->err) != 0) { ok = 0; break; }
        if (global_ns() - t0 > limit_ns) {
          raise_error(ctl, KP_DEV_ERR_TIMEOUT, where);
          ok = 0;
          break;
        }
      }
    }
    if (ok && check_err && *((volatile int*)&ctl->err) != 0) ok = 0;
    s_ok = ok;
    if (watch) s_watch = *((volatile const int*)watch);
  }
  __syncthreads();
  if (watch) *watched = s_watch;
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// block-level scans over one flag per thread (blockDim.x multiple of 32)
// ---------------------------------------------------------------------------

struct ScanSmem {
  int warp[33];
};

// Exclusive prefix sum of one int per thread in thread order; total in
// *total.  Must be called by every thread of the block.
__device__ __forceinline__ int block_exclusive_scan(int v, ScanSmem& sm, int* total) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((int)lane >= o) x += y;
  }
  if (lane == 31) sm.warp[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) {
      const int c = sm.warp[i];
      sm.warp[i] = acc;
      acc += c;
    }
    sm.warp[32] = acc;
  }
  __syncthreads();
  const int r = sm.warp[w] + x - v;
  *total = sm.warp[32];
  __syncthreads();
  return r;
}

// Block sum of two per-thread values.
__device__ __forceinline__ void block_sum2(unsigned long long a, unsigned long long b,
                                           unsigned long long* s /*[64]*/,
                                           unsigned long long* ra, unsigned long long* rb) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    s[w] = a;
    s[32 + w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long x = 0, y = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      x += s[i];
      y += s[32 + i];
    }
    s[0] = x;
    s[32] = y;
  }
  __syncthreads();
  *ra = s[0];
  *rb = s[32];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 bijection,
// the key advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 24 high bits of a word as a float in [0, 1), exact.  Each 12-bit half is
// made a float by placing it in the mantissa of 2^23 and subtracting 2^23
// (FP32 pipe, no conversion instruction); hi * 2^12 + lo < 2^24 is exact.
__device__ __forceinline__ float unit24(uint32_t w) {
  const float hi = __fsub_rn(__uint_as_float(0x4B000000u | (w >> 20)), 8388608.0f);
  const float lo = __fsub_rn(__uint_as_float(0x4B000000u | ((w >> 8) & 0xFFFu)), 8388608.0f);
  return __fmul_rn(__fmaf_rn(hi, 4096.0f, lo), 5.9604644775390625e-08f);
}

// ---------------------------------------------------------------------------
// sine and cosine for the integrators
// ---------------------------------------------------------------------------

// Cody & Waite (1980) argument reduction: r = x - k 2pi with k = rint(x /
// 2pi), 2pi split into C1 = fl32(2pi) and C2 = 2pi - C1 so that k C1 is
// exact for |k| < 2^11 (|x| below ~1.2e4 rad); then the hardware sin/cos
// approximations on r in [-pi, pi] (absolute error below 1e-6).
// k is rounded to the nearest integer (ties to even) by adding 1.5 * 2^23
// to x / 2pi in the same fused multiply-add (one rounding) and subtracting
// it again: exact for |x / 2pi| < 2^22, and kept on the FP32 pipe instead
// of the slower conversion unit.
__device__ __forceinline__ void sincos_reduced(float x, float* s, float* c) {
  const float k = __fsub_rn(__fmaf_rn(x, 0.159154943091895336f, 12582912.0f), 12582912.0f);
  float r = __fmaf_rn(-k, 6.28318548202514648f, x);
  r = __fmaf_rn(-k, -1.74845560007448838e-07f, r);
  __sincosf(r, s, c);
}

// ---------------------------------------------------------------------------
// systems (Sec. II, Eq. 1-2), FP32 in registers
//
// Every product and sum is written with an explicitly rounded operation
// (__fmul_rn, __fadd_rn, __fmaf_rn), which the compiler neither fuses nor
// splits: the integrators give the same bits wherever they are inlined, so
// a sample re-derived from its key (the sample log's replay check of every
// appended sample) equals the sample the expand phase checked and binned.
// ---------------------------------------------------------------------------

template <int SYS>
struct System;

// 6D double integrator: p' = v, v' = u; explicit Euler.
template <>
struct System<KP_SYS_DI> {
  static constexpr int D = 6, N = 3;
  // finished lanes a warp waits for before it finalises and refills them
  // (measured on the GB300: cheap steps favour large refill groups; for
  // Euler steps the whole warp, 32)
  static constexpr int REFILL_MIN = 32;
  // smallest first key batch of a warp (keys a warp starts a pass with
  // when the pass is small; measured on the GB300: spreading a small pass
  // over more warps helps the RK4 systems, not the Euler one)
  static constexpr int FIRST_BATCH_MIN = 32;
  // later key batches are the keys left over GUIDED_DIV x the warps (at
  // most KP_KEY_BATCH): larger divisors hand out smaller batches towards
  // the end of a pass (measured: 4 helps the quadrotor's long samples)
  static constexpr int GUIDED_DIV = 2;
  __device__ __forceinline__ static void step(float* x, const float* u, float h,
                                              const KParams&) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float p = __fmaf_rn(h, x[3 + i], x[i]);
      const float v = __fmaf_rn(h, u[i], x[3 + i]);
      x[i] = p;
      x[3 + i] = v;
    }
  }
  __device__ __forceinline__ static float speed(const float* x) {
    return sqrtf(__fmaf_rn(x[5], x[5], __fmaf_rn(x[4], x[4], __fmul_rn(x[3], x[3]))));
  }
};

// One classic RK4 step x <- x + h/6 (k1 + 2 k2 + 2 k3 + k4), stage points
// x + h/2 k1, x + h/2 k2, x + h k3; h6 = h / 6, rounded as an FP32 division
// (KParams::dt_sixth).  The combination is accumulated as each
// stage is evaluated, in the fixed order ((k1 + 2 k2) + 2 k3) + k4, so only
// one stage derivative is live at a time (the register budget of the loop
// kernel holds no four of them for the 12D system).  F(t, k) evaluates the
// field at t into k.
template <int D, class F>
__device__ __forceinline__ void rk4_step(float* x, float h, float h6, F field) {
  float acc[D], k[D], t[D];
  const float hh = __fmul_rn(0.5f, h);
  field(x, k);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    acc[i] = k[i];
    t[i] = __fmaf_rn(hh, k[i], x[i]);
  }
  field(t, k);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    acc[i] = __fmaf_rn(2.0f, k[i], acc[i]);
    t[i] = __fmaf_rn(hh, k[i], x[i]);
  }
  field(t, k);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    acc[i] = __fmaf_rn(2.0f, k[i], acc[i]);
    t[i] = __fmaf_rn(h, k[i], x[i]);
  }
  field(t, k);
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = __fmaf_rn(h6, __fadd_rn(acc[i], k[i]), x[i]);
}

// 6D Dubins airplane (Chitsaz & LaValle 2007); classic RK4.
template <>
struct System<KP_SYS_DUBINS> {
  static constexpr int D = 6, N = 3;
  static constexpr int REFILL_MIN = 16;
  static constexpr int FIRST_BATCH_MIN = 16;
  static constexpr int GUIDED_DIV = 2;
  __device__ __forceinline__ static void f(const float* x, const float* u, float* dx) {
    float sp, cp, st, ct;
    sincos_reduced(x[3], &sp, &cp);
    sincos_reduced(x[4], &st, &ct);
    dx[0] = __fmul_rn(__fmul_rn(x[5], cp), ct);
    dx[1] = __fmul_rn(__fmul_rn(x[5], sp), ct);
    dx[2] = __fmul_rn(x[5], st);
    dx[3] = u[0];
    dx[4] = u[1];
    dx[5] = u[2];
  }
  __device__ __forceinline__ static void step(float* x, const float* u, float h,
                                              const KParams& P) {
    rk4_step<6>(x, h, P.dt_sixth, [&](const float* y, float* dy) { f(y, u, dy); });
  }
  __device__ __forceinline__ static float speed(const float* x) { return fabsf(x[5]); }
};

// 12D quadrotor, Newton-Euler, plus configuration; classic RK4.
// x = (p, phi theta psi, v_world, omega_body); u = rotor thrusts T1..T4.
template <>
struct System<KP_SYS_QUAD> {
  static constexpr int D = 12, N = 4;
  static constexpr int REFILL_MIN = 12;
  static constexpr int FIRST_BATCH_MIN = 16;
  static constexpr int GUIDED_DIV = 4;
  __device__ __forceinline__ static void f(const float* x, const float* u, const KParams& P,
                                           float* dx) {
    // phys: m g l c Ixx Iyy Izz; recip: 1/m 1/Ixx 1/Iyy 1/Izz
    const float g = P.phys[1], l = P.phys[2], c = P.phys[3];
    const float Ix = P.phys[4], Iy = P.phys[5], Iz = P.phys[6];
    float sphi, cphi, sth, cth, sps, cps;
    sincos_reduced(x[3], &sphi, &cphi);
    sincos_reduced(x[4], &sth, &cth);
    sincos_reduced(x[5], &sps, &cps);
    const float sec = __frcp_rn(cth);
    const float tth = __fmul_rn(sth, sec);
    const float p = x[9], q = x[10], r = x[11];
    dx[0] = x[6];
    dx[1] = x[7];
    dx[2] = x[8];
    // Euler-angle rates W(phi, theta) omega
    dx[3] = __fmaf_rn(__fmul_rn(cphi, tth), r, __fmaf_rn(__fmul_rn(sphi, tth), q, p));
    dx[4] = __fmaf_rn(-sphi, r, __fmul_rn(cphi, q));
    dx[5] = __fmul_rn(__fmaf_rn(cphi, r, __fmul_rn(sphi, q)), sec);
    // world acceleration R(phi, theta, psi) (0, 0, sum T) / m - g e3
    const float thrust = __fadd_rn(__fadd_rn(__fadd_rn(u[0], u[1]), u[2]), u[3]);
    const float a = __fmul_rn(thrust, P.recip[0]);
    const float cs = __fmul_rn(cphi, sth);
    dx[6] = __fmul_rn(a, __fmaf_rn(cs, cps, __fmul_rn(sphi, sps)));
    dx[7] = __fmul_rn(a, __fmaf_rn(cs, sps, -__fmul_rn(sphi, cps)));
    dx[8] = __fmaf_rn(a, __fmul_rn(cphi, cth), -g);
    // body torques and I omega' = tau - omega x (I omega)
    const float tx = __fmul_rn(l, __fsub_rn(u[1], u[3]));
    const float ty = __fmul_rn(l, __fsub_rn(u[2], u[0]));
    const float tz = __fmul_rn(c, __fsub_rn(__fadd_rn(__fsub_rn(u[0], u[1]), u[2]), u[3]));
    const float Lx = __fmul_rn(Ix, p), Ly = __fmul_rn(Iy, q), Lz = __fmul_rn(Iz, r);
    dx[9] = __fmul_rn(__fsub_rn(tx, __fmaf_rn(q, Lz, -__fmul_rn(r, Ly))), P.recip[1]);
    dx[10] = __fmul_rn(__fsub_rn(ty, __fmaf_rn(r, Lx, -__fmul_rn(p, Lz))), P.recip[2]);
    dx[11] = __fmul_rn(__fsub_rn(tz, __fmaf_rn(p, Ly, -__fmul_rn(q, Lx))), P.recip[3]);
  }
  __device__ __forceinline__ static void step(float* x, const float* u, float h,
                                              const KParams& P) {
    rk4_step<12>(x, h, P.dt_sixth, [&](const float* y, float* dy) { f(y, u, P, dy); });
  }
  __device__ __forceinline__ static float speed(const float* x) {
    return sqrtf(__fmaf_rn(x[8], x[8], __fmaf_rn(x[7], x[7], __fmul_rn(x[6], x[6]))));
  }
};

// ---------------------------------------------------------------------------
// decomposition (Sec. III): fine cell per axis, then region and sub-region
// ---------------------------------------------------------------------------

__device__ __forceinline__ int fine_cell(float t, int n) {
  // NaN and negatives go to cell 0, the far side is clamped to n - 1
  return t >= 0.0f ? (t < (float)n ? (int)t : n - 1) : 0;
}

// Region and sub-region under the kd-tree decomposition: descend from the
// root (below a plane goes left, to node + 1), then the sub-grid cell of the
// leaf's own box.  The tree is read from the staged blob in shared memory
// when it was staged (sblob given and kd_smem_off >= 0), else from global
// memory.  It is built on the host with depth at most KP_FSO_MAX_DEPTH and
// every child index above its parent's, so the walk ends; the bound only
// guards it.
__device__ __forceinline__ void bin_fso(const float* x, const KParams& P, int* region, int* sub,
                                        const unsigned char* sblob) {
  const bool staged = sblob != nullptr && P.kd_smem_off >= 0;
  const int32_t* codes =
      staged ? reinterpret_cast<const int32_t*>(sblob + P.kd_smem_off) : P.kd_node;
  const float* splits = staged ? reinterpret_cast<const float*>(codes + P.kd_n) : P.kd_split;
  // codes are read unsigned: the tag sits in the top two bits
  int node = 0;
  uint32_t code = (uint32_t)codes[0];
  for (int depth = 0; (code >> 30) != 3u && depth < KP_FSO_MAX_DEPTH; ++depth) {
    const uint32_t a = code >> 30;
    const float xa = a == 0u ? x[0] : (a == 1u ? x[1] : x[2]);
    node = xa < splits[node] ? node + 1 : (int)(code & 0x3fffffffu);
    code = (uint32_t)codes[node];
  }
  const int r = (code >> 30) == 3u ? (int)(code & 0x3fffffffu) : 0;
  const float4 lo = __ldg(P.leaf_box + 2 * r);
  const float4 sc = __ldg(P.leaf_box + 2 * r + 1);
  const int fx = fine_cell(__fmul_rn(__fsub_rn(x[0], lo.x), sc.x), P.sub[0]);
  const int fy = fine_cell(__fmul_rn(__fsub_rn(x[1], lo.y), sc.y), P.sub[1]);
  const int fz = fine_cell(__fmul_rn(__fsub_rn(x[2], lo.z), sc.z), P.sub[2]);
  *region = r;
  *sub = r * P.n_sub_per + fx + P.sub[0] * (fy + P.sub[1] * fz);
}

template <int SYS>
__device__ __forceinline__ void bin_state(const float* x, const KParams& P, int* region, int* sub,
                                          const unsigned char* sblob = nullptr) {
  if (P.fso) {
    bin_fso(x, P, region, sub, sblob);
    return;
  }
  int cell[3], fine[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // the floor of fine_cell on the FP32 pipe (as the broad phase's cells)
    const float t = __fmul_rn(__fsub_rn(x[a], P.ws_lo[a]), P.fine_scale[a]);
    const float v = __fadd_rd(fminf(fmaxf(t, 0.0f), P.n_fine_last[a]), 8388608.0f);
    const int f = __float_as_int(v) - 0x4B000000;
    cell[a] = P.sub_shift[a] >= 0 ? f >> P.sub_shift[a] : f / P.sub[a];
    fine[a] = f - cell[a] * P.sub[a];
  }
  int sb = 0;
  if (P.speed_bins > 1)
    sb = fine_cell(__fmul_rn(System<SYS>::speed(x), P.speed_scale), P.speed_bins);
  // further state dimensions (a grid over the state space), slowest
  int e = 0, stride = 1;
#pragma unroll
  for (int dd = 3; dd < System<SYS>::D; ++dd) {
    const int n = P.state_grid[dd];
    if (n > 1) {
      float t;
      if (P.state_wrap[dd]) {
        const float pi = 3.14159265358979324f;
        const float turns = floorf(__fmul_rn(__fadd_rn(x[dd], pi), 0.159154943091895336f));
        const float y = __fsub_rn(x[dd], __fmul_rn(turns, 6.28318530717958648f));
        t = __fmul_rn(__fadd_rn(y, pi), P.state_scale[dd]);
      } else {
        t = __fmul_rn(__fsub_rn(x[dd], P.x_lo[dd]), P.state_scale[dd]);
      }
      e += stride * fine_cell(t, n);
      stride *= n;
    }
  }
  const int nsb = P.speed_bins > 1 ? P.speed_bins : 1;
  const int r =
      cell[0] + P.grid[0] * (cell[1] + P.grid[1] * (cell[2] + P.grid[2] * (sb + nsb * e)));
  const int k = fine[0] + P.sub[0] * (fine[1] + P.sub[1] * fine[2]);
  *region = r;
  *sub = r * P.n_sub_per + k;
}

// ---------------------------------------------------------------------------
// validity (Sec. II valid set): state box and segment hull vs closed boxes
// ---------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ bool in_state_box(const float* x, const KParams& P) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < D; ++i) ok &= (P.x_lo[i] <= x[i]) & (x[i] <= P.x_hi[i]);
  return ok;
}

// Closed-box overlap of the hull [l, h] with box (bl, bh), on the FP32 add
// pipe: the boxes meet iff all six differences bh - l and h - bl are >= 0,
// i.e. iff none has its sign bit set.  Exact for finite or infinite inputs
// without negative zeros (the caller canonicalises the hull with + 0.0f;
// the host does the same for the boxes): a - b is +0 when a == b and
// negative (never -0) when a < b, because the difference of two floats
// never rounds to zero.
__device__ __forceinline__ bool box_meets_hull(float4 bl, float4 bh, float lx, float ly,
                                               float lz, float hx, float hy, float hz) {
  const uint32_t s = __float_as_uint(bh.x - lx) | __float_as_uint(hx - bl.x) |
                     __float_as_uint(bh.y - ly) | __float_as_uint(hy - bl.y) |
                     __float_as_uint(bh.z - lz) | __float_as_uint(hz - bl.z);
  return (int32_t)s >= 0;
}

// Broad-phase cell of a coordinate already in cell units (the host build
// uses the same FP32 arithmetic), clamped to [0, g - 1] (NaN to 0); last =
// g - 1 as a float.  The floor is taken on the FP32 pipe: adding 2^23 with
// rounding down leaves floor(t) in the low mantissa bits (exact for t in
// [0, 2^23)); the cell comes back both as an int and as a float.
__device__ __forceinline__ int bp_cell_of(float t, float last, float* ft) {
  const float v = __fadd_rd(fminf(fmaxf(t, 0.0f), last), 8388608.0f);
  *ft = __fsub_rn(v, 8388608.0f);
  return __float_as_int(v) - 0x4B000000;
}

// A byte as a float, on the FP32 pipe (exact).
__device__ __forceinline__ float byte_as_float(uint32_t q) {
  return __fsub_rn(__int_as_float(0x4B000000 | q), 8388608.0f);
}

// Exact coarse-then-fine collision test of a step hull (the paper's coarse
// phase, Sec. III-B).  First the clearance of the cell holding the hull's
// low corner: a hull inside that cell grown by its clearance on every side
// meets no box (the clearance is a lower bound on the L-infinity gap, per
// axis in cell units, from the cell to every box; the host subtracts a
// margin far above the FP32 rounding of the cell coordinates).  Otherwise
// only the boxes listed in the uniform-grid cells the hull touches are
// tested: a box meeting the hull shares a point with it, that point's cell
// lies in both cell ranges (the cell map is monotone), so the box is in
// one of the visited lists.  Either way the verdict equals testing every
// box.  'tests' counts the box tests made.
__device__ __forceinline__ bool hull_hits_grid(const KParams& P, const float4* __restrict__ sbox,
                                               const uint16_t* __restrict__ sstart,
                                               const uint16_t* __restrict__ sids,
                                               const uint8_t* __restrict__ sclear, float lx,
                                               float ly, float lz, float hx, float hy, float hz,
                                               uint32_t* tests) {
  const int gx = P.bp_g[0], gy = P.bp_g[1], gz = P.bp_g[2];
  const float tlx = __fmul_rn(__fsub_rn(lx, P.ws_lo[0]), P.bp_scale[0]);
  const float thx = __fmul_rn(__fsub_rn(hx, P.ws_lo[0]), P.bp_scale[0]);
  const float tly = __fmul_rn(__fsub_rn(ly, P.ws_lo[1]), P.bp_scale[1]);
  const float thy = __fmul_rn(__fsub_rn(hy, P.ws_lo[1]), P.bp_scale[1]);
  const float tlz = __fmul_rn(__fsub_rn(lz, P.ws_lo[2]), P.bp_scale[2]);
  const float thz = __fmul_rn(__fsub_rn(hz, P.ws_lo[2]), P.bp_scale[2]);
  float fx, fy, fz, dummy;
  const int x0 = bp_cell_of(tlx, P.bp_last[0], &fx), x1 = bp_cell_of(thx, P.bp_last[0], &dummy);
  const int y0 = bp_cell_of(tly, P.bp_last[1], &fy), y1 = bp_cell_of(thy, P.bp_last[1], &dummy);
  const int z0 = bp_cell_of(tlz, P.bp_last[2], &fz), z1 = bp_cell_of(thz, P.bp_last[2], &dummy);
  if (sclear != nullptr) {
    const float r =
        __fmul_rn(byte_as_float(sclear[KP_IDX(P, x0 + gx * (y0 + gy * z0), gx * gy * gz, 60)]),
                  0.0625f);
    if (r > 0.0f && tlx >= fx - r && thx <= fx + 1.0f + r && tly >= fy - r &&
        thy <= fy + 1.0f + r && tlz >= fz - r && thz <= fz + 1.0f + r)
      return false;
  }
  uint32_t n = 0;
  bool hit = false;
  for (int cz = z0; cz <= z1 && !hit; ++cz)
    for (int cy = y0; cy <= y1 && !hit; ++cy)
      for (int cx = x0; cx <= x1 && !hit; ++cx) {
        const int c = KP_IDX(P, cx + gx * (cy + gy * cz), gx * gy * gz, 61);
        const int e = sstart[c + 1];
        for (int q = sstart[c]; q < e; ++q) {
          const int b = KP_IDX(P, sids[KP_IDX(P, q, P.bp_n_ids, 62)], P.n_boxes_pad, 63);
          ++n;
          if (box_meets_hull(sbox[2 * b], sbox[2 * b + 1], lx, ly, lz, hx, hy, hz)) {
            hit = true;
            break;
          }
        }
      }
  *tests += n;
  return hit;
}

}  // namespace kp
