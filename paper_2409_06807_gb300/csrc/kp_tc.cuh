// kp_tc.cuh -- BF16 GEMM on the fifth-generation tensor cores (tcgen05) for
// the learned proposal's training: C (M x N) = A (M x K) * B (N x K)^T with
// both operands K-major (row-major, K contiguous) in global memory, FP32
// accumulation in tensor memory.
//
// One CTA of 128 threads computes a 128 x 128 tile of C:
//   warp 0, lane 0  : producer -- TMA tiled loads (128B swizzle) of 128 x 64
//                     tiles of A and B into a ring of STAGES shared-memory
//                     stages, completing on the stage's "full" mbarrier;
//   warp 1, lane 0  : issues tcgen05.mma (M 128, N 128, K 16 each, four per
//                     64-wide k tile) into the CTA's TMEM accumulator and
//                     commits each stage back to the producer ("empty");
//   all four warps  : epilogue -- each warp reads its 32 TMEM lanes (rows)
//                     with tcgen05.ld and applies the epilogue.
// Split-K over blockIdx.z accumulates with FP32 atomics (EPI_ATOMIC_F32).
//
// Every wait is bounded by a device-time limit; on expiry the CTA records a
// nonzero site in *err, skips its stores, and still frees its TMEM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

namespace kp {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TILE_A_BYTES = BM * BK * 2;  // 16 KB
constexpr int TILE_B_BYTES = BN * BK * 2;  // 16 KB
constexpr int STAGE_BYTES = TILE_A_BYTES + TILE_B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + room to align to 1 KB
constexpr uint32_t TMEM_COLS = 128;

enum { EPI_BIAS_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_ATOMIC_F32 = 2 };

struct TcArgs {
  int M, N, K;               // C is M x N, contraction length K
  int kt_per_split;          // 64-wide k tiles per blockIdx.z
  const float* bias;         // EPI_BIAS_RELU_BF16: bias[n]
  const __nv_bfloat16* mask; // EPI_MASK_BF16: C kept where mask[m * ldc + n] > 0
  __nv_bfloat16* cb;         // BF16 output, row stride ldc
  __nv_bfloat16* cbt;        // optional BF16 transposed output [n][m], row stride ldt
  float* cf;                 // EPI_ATOMIC_F32 output, row stride ldc
  int ldc, ldt;
  int* err;
  unsigned long long wait_ns;
};

// Instruction descriptor of tcgen05.mma kind::f16: D F32, A and B BF16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart
// (stride byte offset), leading byte offset unused for this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (16 B; ignored)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Waits (bounded) for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 63u) == 63u && now_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives on the mbarrier once every tcgen05 operation this thread issued
// before has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// 32 consecutive 32-bit columns of the calling thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int EPI>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  uint8_t* tiles = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kt_all = (a.K + BK - 1) / BK;
  const int kt0 = blockIdx.z * a.kt_per_split;
  const int kt1 = kt0 + a.kt_per_split < kt_all ? kt0 + a.kt_per_split : kt_all;
  const int nk = kt1 - kt0;  // >= 1: the host sizes the split so

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(saddr(&full[s]), 1);
      mbar_init(saddr(&empty[s]), 1);
    }
    mbar_init(saddr(&done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(&tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(saddr(&empty[s]), (uint32_t)((i / STAGES) - 1) & 1u, a.wait_ns)) {
        s_fail = 1;
        break;
      }
      const uint32_t dA = saddr(tiles + s * STAGE_BYTES);
      mbar_expect_tx(saddr(&full[s]), STAGE_BYTES);
      tma_load_2d(dA, &ta, (kt0 + i) * BK, m0, saddr(&full[s]));
      tma_load_2d(dA + TILE_A_BYTES, &tb, (kt0 + i) * BK, n0, saddr(&full[s]));
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(BM, BN);
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(saddr(&full[s]), (uint32_t)(i / STAGES) & 1u, a.wait_ns)) {
        s_fail = 2;
        break;
      }
      fence_after();
      const uint32_t sA = saddr(tiles + s * STAGE_BYTES), sB = sA + TILE_A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        mma_bf16(tmem, sdesc_sw128(sA + kk * 32), sdesc_sw128(sB + kk * 32), idesc,
                 (i | kk) != 0 ? 1u : 0u);
      mma_commit(saddr(&empty[s]));
    }
    mma_commit(saddr(&done));
  }
  __syncwarp();

  // epilogue: thread (warp, lane) owns row m0 + 32 warp + lane
  if (!mbar_wait(saddr(&done), 0, a.wait_ns)) s_fail = 3;
  fence_after();
  const int row = m0 + warp * 32 + lane;
  const bool live = *((volatile int*)&s_fail) == 0 && row < a.M;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t r[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    if (!live) continue;
    const int nb = n0 + c0;
    const bool full32 = nb + 32 <= a.N;
    if (EPI == EPI_ATOMIC_F32) {
      float* dst = a.cf + (size_t)row * a.ldc + nb;
      if (full32 && (((uintptr_t)dst & 15u) == 0)) {
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + j),
                       "f"(__uint_as_float(r[j])), "f"(__uint_as_float(r[j + 1])),
                       "f"(__uint_as_float(r[j + 2])), "f"(__uint_as_float(r[j + 3]))
                       : "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (nb + j < a.N) atomicAdd(dst + j, __uint_as_float(r[j]));
      }
    } else {
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
      if (EPI == EPI_BIAS_RELU_BF16) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + (nb + j < a.N ? a.bias[nb + j] : 0.0f), 0.0f);
      }
      __nv_bfloat16* dst = a.cb + (size_t)row * a.ldc + nb;
      const bool vec = full32 && (((uintptr_t)dst & 15u) == 0) && (a.ldc % 8) == 0;
      if (vec) {
        if (EPI == EPI_MASK_BF16) {
          const uint4* mk = reinterpret_cast<const uint4*>(a.mask + (size_t)row * a.ldc + nb);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 u = mk[q];
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
              const uint16_t bits = (uint16_t)(w[h >> 1] >> (16 * (h & 1)));
              // a BF16 value is > 0 when its sign bit is clear, it is nonzero
              // and it is not a NaN (exponent all ones, mantissa nonzero)
              if (!((bits & 0x8000u) == 0 && bits != 0 && bits <= 0x7F80u)) v[8 * q + h] = 0.0f;
            }
          }
        }
        uint4* out = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 pr = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
            w[h] = *reinterpret_cast<const uint32_t*>(&pr);
          }
          out[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (nb + j >= a.N) break;
          if (EPI == EPI_MASK_BF16 &&
              !(__bfloat162float(a.mask[(size_t)row * a.ldc + nb + j]) > 0.0f))
            v[j] = 0.0f;
          dst[j] = __float2bfloat16_rn(v[j]);
        }
      }
      if (a.cbt) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (nb + j < a.N) a.cbt[(size_t)(nb + j) * a.ldt + row] = __float2bfloat16_rn(v[j]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(a.err, 100 + s_fail);
}

}  // namespace tc
}  // namespace kp
