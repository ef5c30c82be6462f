// kp_mlp.cuh -- the learned control proposal's network on the tensor cores:
// BF16 operands, FP32 accumulation (mma.sync m16n8k16), shared by the
// standalone inference/training kernels and the planner's loop kernel.
//
// Network: 32 inputs (24 node features, zero padded) -> 256 ReLU -> 256
// ReLU -> 8 outputs; heads: mean = tanh(out[0..3]), log_std = clamp(out[4..7],
// -4, 1).  Weights row-major [out][in] in BF16, biases FP32.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace kp {

constexpr int MLP_IN = 32, MLP_H = 256, MLP_OUT = 8, MLP_NQ = 4;
constexpr int MLP_TILE = 32;           // rows per block tile (standalone kernels)
constexpr int MLP_LOOP_TILE = 32;      // rows per block tile inside the planner loop
constexpr int MLP_XS = MLP_IN + 8;     // padded smem row (bf16) of the input tile
constexpr int MLP_HS = MLP_H + 8;      // padded smem row (bf16) of a hidden tile
constexpr float MLP_LOGSTD_MIN = -4.0f, MLP_LOGSTD_MAX = 1.0f;
// shared memory of one loop tile: input rows + hidden rows (bf16)
constexpr int MLP_LOOP_TILE_SMEM = MLP_LOOP_TILE * MLP_XS * 2 + MLP_LOOP_TILE * MLP_HS * 2;

struct MlpWeights {
  const __nv_bfloat16* W1;  // [256][32]
  const float* b1;
  const __nv_bfloat16* W2;  // [256][256]
  const float* b2;
  const __nv_bfloat16* W3;  // [8][256]
  const float* b3;
};

// D = A (16x16, row) * B (16x8, col) + D, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// A fragment (rows m0.., k0..) from a row-major bf16 tile with row stride ld.
// Register j holds elements (g + 8*(j&1), 2t + 8*(j>>1)) and the next column,
// g = lane / 4, t = lane % 4.
__device__ __forceinline__ void frag_a(const __nv_bfloat16* s, int ld, int m0, int k0,
                                       uint32_t* a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = ld_u32(s + (m0 + g) * ld + k0 + 2 * t);
  a[1] = ld_u32(s + (m0 + g + 8) * ld + k0 + 2 * t);
  a[2] = ld_u32(s + (m0 + g) * ld + k0 + 2 * t + 8);
  a[3] = ld_u32(s + (m0 + g + 8) * ld + k0 + 2 * t + 8);
}

// B fragment (k0.., columns n0..) from weights W[n][k] (row stride ld):
// register j holds (k = 2t + 8j and k + 1, n = g).
__device__ __forceinline__ void frag_b(const __nv_bfloat16* W, int ld, int n0, int k0,
                                       uint32_t* b) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  b[0] = ld_u32(W + (n0 + g) * ld + k0 + 2 * t);
  b[1] = ld_u32(W + (n0 + g) * ld + k0 + 2 * t + 8);
}

// Fragment order of a hidden layer's weights W[n][k] (N = 256 outputs, K
// inputs): for the warp owning columns 32w.. and k-step s, each lane keeps
// its B fragments of the four 8-column blocks as eight consecutive 32-bit
// words (block ni, register h), so that a lane fetches them with two 16-byte
// loads.  Returns the bf16 index of W[n][k] in that order.
__host__ __device__ __forceinline__ int frag_index_hidden(int n, int k, int K) {
  const int w = n >> 5, ni = (n & 31) >> 3, g = n & 7;
  const int s = k >> 4, kk = k & 15, h = kk >> 3, t = (kk & 7) >> 1, e = kk & 1;
  return (((w * (K >> 4) + s) * 32 + g * 4 + t) * 16) + ni * 4 + h * 2 + e;
}

// Fragment order of the output layer W3[8][256]: warp w uses k-steps 2w and
// 2w+1; a lane's four words for them are consecutive (one 16-byte load).
__host__ __device__ __forceinline__ int frag_index_out(int n, int k) {
  const int s = k >> 4, kk = k & 15, h = kk >> 3, t = (kk & 7) >> 1, e = kk & 1;
  return (((s >> 1) * 32 + n * 4 + t) * 8) + (s & 1) * 4 + h * 2 + e;
}

// B fragments of the four 8-column blocks of this warp at k-step s, from a
// hidden layer's weights in fragment order.
__device__ __forceinline__ void frag_b4_ordered(const __nv_bfloat16* Wf, int K, int s,
                                                uint32_t b[4][2]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint4* q = reinterpret_cast<const uint4*>(Wf) + (((warp * (K >> 4) + s) * 32 + lane) * 2);
  const uint4 u0 = __ldg(q), u1 = __ldg(q + 1);
  b[0][0] = u0.x; b[0][1] = u0.y; b[1][0] = u0.z; b[1][1] = u0.w;
  b[2][0] = u1.x; b[2][1] = u1.y; b[3][0] = u1.z; b[3][1] = u1.w;
}

// One dense ReLU layer on a tile of 16*MI rows: out = relu(in * W^T + b),
// every warp producing 32 output columns.  'in' is a bf16 smem tile (row
// stride ld_in, K columns).  Results stay in registers (acc) until the
// caller stores them.
template <int K, int MI, bool ORDERED = false>
__device__ __forceinline__ void layer_relu(const __nv_bfloat16* in, int ld_in,
                                           const __nv_bfloat16* W, const float* bias,
                                           float acc[MI][4][4]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = lane & 3;
  const int n_base = warp * 32;
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const float b0 = bias[n_base + ni * 8 + 2 * t], b1 = bias[n_base + ni * 8 + 2 * t + 1];
      acc[mi][ni][0] = b0;
      acc[mi][ni][1] = b1;
      acc[mi][ni][2] = b0;
      acc[mi][ni][3] = b1;
    }
#pragma unroll 4
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[MI][4], b[4][2];
    if (ORDERED) {
      frag_b4_ordered(W, K, k0 >> 4, b);
    } else {
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) frag_b(W, K, n_base + ni * 8, k0, b[ni]);
    }
#pragma unroll
    for (int mi = 0; mi < MI; ++mi) frag_a(in, ld_in, mi * 16, k0, a[mi]);
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], a[mi], b[ni]);
  }
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mi][ni][q] = fmaxf(acc[mi][ni][q], 0.0f);
}

// Writes a layer's register results as bf16 into a smem tile (and, when
// given, into global rows row0.. of a [rows][256] bf16 array).
template <int MI>
__device__ __forceinline__ void store_hidden(const float acc[MI][4][4], __nv_bfloat16* s,
                                             __nv_bfloat16* g, int row0, int rows_valid) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = mi * 16 + gi + 8 * h;
        const int c = warp * 32 + ni * 8 + 2 * t;
        const uint32_t v = pack_bf16(acc[mi][ni][2 * h], acc[mi][ni][2 * h + 1]);
        *reinterpret_cast<uint32_t*>(s + r * MLP_HS + c) = v;
        if (g && r < rows_valid) *reinterpret_cast<uint32_t*>(g + (size_t)(row0 + r) * MLP_H + c) = v;
      }
}

// Forward pass of one tile of 16*MI rows.  sX holds the bf16 inputs (row
// stride MLP_XS), sH is scratch (16*MI x MLP_HS bf16).  Writes the 8 raw
// outputs of valid rows to raw[(row0 + r) * 8 ..] and, when g_h1/g_h2 are
// given, the hidden activations (training).  Every thread of the block
// (256) must call it.
//
// The output layer (K = 256, 8 columns) is split over K: warp w multiplies
// the 16-row blocks by k-steps 2w and 2w+1 and leaves its partial sums in
// shared memory (over sH, once every warp has read h2); the partials are
// then added in warp order.  Two dependent products per warp instead of
// sixteen keep the tile's latency short.
template <int MI, bool ORDERED = false>
__device__ __forceinline__ void mlp_tile_forward(const MlpWeights& w, const __nv_bfloat16* sX,
                                                 __nv_bfloat16* sH, float* raw, int row0,
                                                 int rows_valid, __nv_bfloat16* g_h1,
                                                 __nv_bfloat16* g_h2) {
  float acc[MI][4][4];
  layer_relu<MLP_IN, MI, ORDERED>(sX, MLP_XS, w.W1, w.b1, acc);
  store_hidden<MI>(acc, sH, g_h1, row0, rows_valid);
  __syncthreads();
  layer_relu<MLP_H, MI, ORDERED>(sH, MLP_HS, w.W2, w.b2, acc);
  __syncthreads();  // every warp has read h1
  store_hidden<MI>(acc, sH, g_h2, row0, rows_valid);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane >> 2, t = lane & 3;
  float d[MI][4];
  uint32_t b[2][2];
  if (ORDERED) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(w.W3) + warp * 32 + lane);
    b[0][0] = u.x; b[0][1] = u.y; b[1][0] = u.z; b[1][1] = u.w;
  } else {
    frag_b(w.W3, MLP_H, 0, warp * 32, b[0]);
    frag_b(w.W3, MLP_H, 0, warp * 32 + 16, b[1]);
  }
#pragma unroll
  for (int mi = 0; mi < MI; ++mi) {
    d[mi][0] = d[mi][1] = d[mi][2] = d[mi][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t a[4];
      frag_a(sH, MLP_HS, mi * 16, warp * 32 + ks * 16, a);
      mma_bf16_16816(d[mi], a, b[ks]);
    }
  }
  __syncthreads();  // every warp has read h2: sH now holds the partials
  float* part = reinterpret_cast<float*>(sH);  // [8 warps][16*MI rows][8]
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = mi * 16 + gi + 8 * h;
      part[(warp * 16 * MI + r) * MLP_OUT + 2 * t] = d[mi][2 * h];
      part[(warp * 16 * MI + r) * MLP_OUT + 2 * t + 1] = d[mi][2 * h + 1];
    }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * MI * MLP_OUT; e += blockDim.x) {
    const int r = e / MLP_OUT, c = e % MLP_OUT;
    float s = w.b3[c];
#pragma unroll
    for (int q = 0; q < 8; ++q) s += part[(q * 16 * MI + r) * MLP_OUT + c];
    if (r < rows_valid) raw[(size_t)(row0 + r) * MLP_OUT + c] = s;
  }
  __syncthreads();
}

// Heads of one output row: mean = tanh, log_std clamped.
__device__ __forceinline__ void mlp_heads(const float* raw, float* mean, float* log_std) {
#pragma unroll
  for (int i = 0; i < MLP_NQ; ++i) {
    mean[i] = tanhf(raw[i]);
    log_std[i] = fminf(fmaxf(raw[MLP_NQ + i], MLP_LOGSTD_MIN), MLP_LOGSTD_MAX);
  }
}

}  // namespace kp
