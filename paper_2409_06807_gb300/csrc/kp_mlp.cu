// kp_mlp.cu -- the learned proposal's network: inference and training
// kernels and the kp_mlp_* entry points of include/kp.h.  Inference runs
// 32-row tiles on mma.sync (the same tile code the planner's loop uses);
// every training GEMM of the backward pass runs on the tcgen05 tensor cores
// (kp_tc.cuh: TMA-staged BF16 operands, FP32 accumulation in tensor memory);
// FP32 master weights and Adam moments.
// Like the planner, the network context allocates no device memory: it
// lives in a caller-owned arena.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "../../include/kp.h"
#include "kp_mlp.cuh"
#include "kp_tc.cuh"

namespace kp {

using bf16 = __nv_bfloat16;

// flat parameter vector (FP32), row-major: W1 b1 W2 b2 W3 b3
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H,
              OFF_B3 = OFF_W3 + MLP_OUT * MLP_H, N_PARAMS = OFF_B3 + MLP_OUT;
constexpr int N_WEIGHTS_BF16 = MLP_H * MLP_IN + MLP_H * MLP_H + MLP_OUT * MLP_H;

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

// One 32-row tile per block: inputs x [M][32] FP32 (rounded to BF16).  Writes
// the raw outputs, and when given the BF16 inputs and hidden activations
// (training) or the heads (inference: mean, log_std per row).
__global__ void __launch_bounds__(256) kp_mlp_forward_kernel(MlpWeights w, const float* x, int M,
                                                             float* raw, float* heads,
                                                             bf16* xb, bf16* h1, bf16* h2,
                                                             bf16* xbt, int ldt) {
  __shared__ __align__(16) bf16 sX[MLP_TILE * MLP_XS];
  __shared__ __align__(16) bf16 sH[MLP_TILE * MLP_HS];
  const int row0 = blockIdx.x * MLP_TILE;
  const int rows = M - row0 < MLP_TILE ? M - row0 : MLP_TILE;
  for (int e = threadIdx.x; e < MLP_TILE * MLP_IN; e += blockDim.x) {
    const int r = e / MLP_IN, c = e % MLP_IN;
    const bf16 v = __float2bfloat16_rn(r < rows ? x[(size_t)(row0 + r) * MLP_IN + c] : 0.0f);
    sX[r * MLP_XS + c] = v;
    if (xb && r < rows) xb[(size_t)(row0 + r) * MLP_IN + c] = v;
    if (xbt && r < rows) xbt[(size_t)c * ldt + row0 + r] = v;
  }
  __syncthreads();
  mlp_tile_forward<MLP_TILE / 16>(w, sX, sH, raw, row0, rows, h1, h2);
  if (heads && threadIdx.x < rows) {
    const int r = row0 + threadIdx.x;
    float mean[MLP_NQ], ls[MLP_NQ];
    mlp_heads(raw + (size_t)r * MLP_OUT, mean, ls);
    for (int i = 0; i < MLP_NQ; ++i) {
      heads[(size_t)r * MLP_OUT + i] = mean[i];
      heads[(size_t)r * MLP_OUT + MLP_NQ + i] = ls[i];
    }
  }
}

// ---------------------------------------------------------------------------
// loss and backward
// ---------------------------------------------------------------------------

// Gaussian negative log-likelihood per row and its gradient with respect to
// the raw outputs (mean through tanh, log_std through the clamp), scaled by
// 1/M.  loss accumulates the batch mean.
__global__ void kp_mlp_head_loss_kernel(const float* raw, const float* t, int M, float* d_raw,
                                        bf16* d_raw_b, float* loss, bf16* d_rawt, int ldt,
                                        float* g_b3) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  float col[MLP_OUT];
#pragma unroll
  for (int i = 0; i < MLP_OUT; ++i) col[i] = 0.0f;
  if (m < M) {
    const float inv_m = 1.0f / (float)M;
    for (int i = 0; i < MLP_NQ; ++i) {
      const float mu = tanhf(raw[(size_t)m * MLP_OUT + i]);
      const float lr = raw[(size_t)m * MLP_OUT + MLP_NQ + i];
      const bool clamped = lr < MLP_LOGSTD_MIN || lr > MLP_LOGSTD_MAX;
      const float ls = fminf(fmaxf(lr, MLP_LOGSTD_MIN), MLP_LOGSTD_MAX);
      const float is = expf(-ls);
      const float z = (t[(size_t)m * MLP_NQ + i] - mu) * is;
      l += ls + 0.5f * z * z;
      const float dm = -z * is * (1.0f - mu * mu) * inv_m;
      const float ds = clamped ? 0.0f : (1.0f - z * z) * inv_m;
      d_raw[(size_t)m * MLP_OUT + i] = dm;
      d_raw[(size_t)m * MLP_OUT + MLP_NQ + i] = ds;
      d_raw_b[(size_t)m * MLP_OUT + i] = __float2bfloat16_rn(dm);
      d_raw_b[(size_t)m * MLP_OUT + MLP_NQ + i] = __float2bfloat16_rn(ds);
      d_rawt[(size_t)i * ldt + m] = __float2bfloat16_rn(dm);
      d_rawt[(size_t)(MLP_NQ + i) * ldt + m] = __float2bfloat16_rn(ds);
      col[i] = dm;
      col[MLP_NQ + i] = ds;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
#pragma unroll
    for (int i = 0; i < MLP_OUT; ++i) col[i] += __shfl_xor_sync(0xffffffffu, col[i], o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (l != 0.0f) atomicAdd(loss, l / (float)M);
#pragma unroll
    for (int i = 0; i < MLP_OUT; ++i)
      if (col[i] != 0.0f) atomicAdd(g_b3 + i, col[i]);
  }
}

// g[r] += sum over the first M columns of row r of a [R][ld] BF16 matrix:
// block (r, c) sums columns [1024 c, 1024 c + 1024) of row r.
__global__ void kp_mlp_rowsum_kernel(const bf16* a, int R, int M, int ld, float* g) {
  __shared__ float red[8];
  const int r = blockIdx.x;
  float s = 0.0f;
  for (int m = blockIdx.y * 1024 + threadIdx.x; m < M && m < (int)(blockIdx.y + 1) * 1024;
       m += blockDim.x)
    s += __bfloat162float(a[(size_t)r * ld + m]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    atomicAdd(g + r, tot);
  }
}

// dh2[m][k] = (sum_n d_raw[m][n] W3[n][k]) where h2[m][k] > 0, else 0, and
// its transpose dh2t[k][m].  A block takes 32 rows; thread k keeps its
// column of W3 and its 32 results, so the row-major store is coalesced and
// the transposed one is four 16-byte stores per thread.
__global__ void __launch_bounds__(256) kp_mlp_dh2_kernel(const float* d_raw, const bf16* W3,
                                                         const bf16* h2, int M, bf16* dh2,
                                                         bf16* dh2t, int ldt) {
  __shared__ float sd[32][MLP_OUT];
  const int m0 = blockIdx.x * 32, k = threadIdx.x;
  for (int e = threadIdx.x; e < 32 * MLP_OUT; e += blockDim.x) {
    const int r = e / MLP_OUT, c = e % MLP_OUT;
    sd[r][c] = m0 + r < M ? d_raw[(size_t)(m0 + r) * MLP_OUT + c] : 0.0f;
  }
  float w3[MLP_OUT];
#pragma unroll
  for (int n = 0; n < MLP_OUT; ++n) w3[n] = __bfloat162float(W3[n * MLP_H + k]);
  __syncthreads();
  float v[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int n = 0; n < MLP_OUT; ++n) s = fmaf(sd[r][n], w3[n], s);
    const int m = m0 + r;
    v[r] = (m < M && __bfloat162float(h2[(size_t)m * MLP_H + k]) > 0.0f) ? s : 0.0f;
    if (m < M) dh2[(size_t)m * MLP_H + k] = __float2bfloat16_rn(v[r]);
  }
  bf16* dst = dh2t + (size_t)k * ldt + m0;
  if (m0 + 32 <= M) {
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
    for (int r = 0; r < 32; ++r)
      if (m0 + r < M) dst[r] = __float2bfloat16_rn(v[r]);
  }
}

// [M][cols] BF16 -> [cols][ldt] (32 x 32 tiles through shared memory; cols a
// multiple of 32).
__global__ void kp_mlp_transpose_kernel(const bf16* a, int M, int cols, bf16* at, int ldt) {
  __shared__ bf16 tile[32][34];
  const int m0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8)
    tile[r][tx] = m0 + r < M ? a[(size_t)(m0 + r) * cols + c0 + tx] : __float2bfloat16_rn(0.0f);
  __syncthreads();
  for (int r = ty; r < 32; r += 8)
    if (m0 + tx < M) at[(size_t)(c0 + r) * ldt + m0 + tx] = tile[tx][r];
}

// ---------------------------------------------------------------------------
// Adam on the FP32 master vector; refreshes the BF16 weight copies
// ---------------------------------------------------------------------------

// Parameter i rounded to BF16 into the row-major weight copy (training
// kernels) and into the fragment-order copy (the planner's loop kernel).
__device__ __forceinline__ void store_weight(int i, float pi, bf16* wb, bf16* wf, bf16* w2t) {
  const bf16 b = __float2bfloat16_rn(pi);
  if (i < OFF_B1) {
    wb[i] = b;
    wf[frag_index_hidden(i / MLP_IN, i % MLP_IN, MLP_IN)] = b;
  } else if (i >= OFF_W2 && i < OFF_B2) {
    const int j = i - OFF_W2;
    wb[MLP_H * MLP_IN + j] = b;
    wf[MLP_H * MLP_IN + frag_index_hidden(j / MLP_H, j % MLP_H, MLP_H)] = b;
    w2t[(j % MLP_H) * MLP_H + j / MLP_H] = b;
  } else if (i >= OFF_W3 && i < OFF_B3) {
    const int j = i - OFF_W3;
    wb[MLP_H * MLP_IN + MLP_H * MLP_H + j] = b;
    wf[MLP_H * MLP_IN + MLP_H * MLP_H + frag_index_out(j / MLP_H, j % MLP_H)] = b;
  }
}

__device__ __forceinline__ void adam_update(int i, float* p, const float* g, float* m, float* v,
                                            float lr, float beta1, float beta2, float eps,
                                            float c1, float c2, bf16* wb, bf16* wf, bf16* w2t) {
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  store_weight(i, pi, wb, wf, w2t);
}

__global__ void kp_mlp_adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr,
                                   float beta1, float beta2, float eps, float c1, float c2,
                                   bf16* wb, bf16* wf, bf16* w2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  adam_update(i, p, g, m, v, lr, beta1, beta2, eps, c1, c2, wb, wf, w2t);
}

// ---- device-driven epoch (one CUDA graph launch per mini-batch) -------------

struct EpochCtl {
  const float* x;        // [rows][32] features
  const float* t;        // [rows][4] targets
  const int32_t* perm;   // row order of the epoch
  int batch;             // index of the next mini-batch
  int step;              // Adam steps taken before the next one
  float lr;
  float loss_sum;        // sum of the mini-batch losses of the epoch
};

// Rows perm[batch * B + r] of x and t into the fixed batch buffers.
__global__ void kp_mlp_gather_kernel(const EpochCtl* ec, int B, float* xg, float* tg) {
  const size_t base = (size_t)ec->batch * B;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * (MLP_IN + MLP_NQ);
       e += gridDim.x * blockDim.x) {
    const int r = e / (MLP_IN + MLP_NQ), c = e % (MLP_IN + MLP_NQ);
    const size_t src = (size_t)ec->perm[base + r];
    if (c < MLP_IN)
      xg[(size_t)r * MLP_IN + c] = ec->x[src * MLP_IN + c];
    else
      tg[(size_t)r * MLP_NQ + c - MLP_IN] = ec->t[src * MLP_NQ + c - MLP_IN];
  }
}

// Adam with the step count and learning rate read from the epoch control.
__global__ void kp_mlp_adam_dev_kernel(float* p, const float* g, float* m, float* v, int n,
                                       const EpochCtl* ec, bf16* wb, bf16* wf, bf16* w2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float beta1 = 0.9f, beta2 = 0.999f;
  const float step = (float)(ec->step + 1);
  const float c1 = 1.0f - powf(beta1, step), c2 = 1.0f - powf(beta2, step);
  adam_update(i, p, g, m, v, ec->lr, beta1, beta2, 1e-8f, c1, c2, wb, wf, w2t);
}

__global__ void kp_mlp_epoch_tail_kernel(EpochCtl* ec, const float* loss) {
  ec->loss_sum += *loss;
  ec->step += 1;
  ec->batch += 1;
}

__global__ void kp_mlp_round_kernel(const float* p, bf16* wb, bf16* wf, bf16* w2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N_PARAMS) return;
  store_weight(i, p[i], wb, wf, w2t);
}

}  // namespace kp

using namespace kp;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct kp_mlp {
  char* arena;
  size_t bytes;
  cudaStream_t stream;
  int max_batch;
  int step;
  float *p, *m, *v, *g;
  bf16* wb;  // W1 | W2 | W3 in BF16, row-major
  bf16* wf;  // the same in fragment order (planner loop)
  bf16* w2t; // W2 transposed ([in][out], tensor-core backward)
  bf16 *dh2t, *h1t, *h2t, *dh1t;  // [256][ldt] transposed activations
  bf16 *xbt, *drawt;               // [32][ldt], [8][ldt]
  int ldt;
  int* err;  // nonzero: a tensor-core kernel's bounded wait expired
  float *xg, *tg;          // gathered mini-batch (device-driven epoch)
  EpochCtl* ec;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t gstream = nullptr;  // the graph's own stream (capture needs a
  cudaEvent_t gev = nullptr;       // non-default stream), ordered by an event
  float *raw, *d_raw, *loss;
  bf16 *xb, *h1, *h2, *d_raw_b, *dh2, *dh1;
};

namespace {

struct MlpLayout {
  size_t p, m, v, g, wb, wf, w2t, dh2t, h1t, h2t, dh1t, xbt, drawt, err, xg, tg, ec, loss, raw, d_raw, xb, h1, h2, d_raw_b, dh2, dh1, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// row stride of the transposed activations: batch rounded up to 64
int ld_t(int B) { return (B + 63) / 64 * 64; }

MlpLayout mlp_layout(int B) {
  MlpLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = a256(off + bytes);
    return o;
  };
  L.p = take((size_t)N_PARAMS * 4);
  L.m = take((size_t)N_PARAMS * 4);
  L.v = take((size_t)N_PARAMS * 4);
  L.g = take((size_t)N_PARAMS * 4);
  L.wb = take((size_t)N_WEIGHTS_BF16 * 2);
  L.wf = take((size_t)N_WEIGHTS_BF16 * 2);
  L.w2t = take((size_t)MLP_H * MLP_H * 2);
  L.dh2t = take((size_t)MLP_H * ld_t(B) * 2);
  L.h1t = take((size_t)MLP_H * ld_t(B) * 2);
  L.h2t = take((size_t)MLP_H * ld_t(B) * 2);
  L.dh1t = take((size_t)MLP_H * ld_t(B) * 2);
  L.xbt = take((size_t)MLP_IN * ld_t(B) * 2);
  L.drawt = take((size_t)MLP_OUT * ld_t(B) * 2);
  L.err = take(16);
  L.xg = take((size_t)B * MLP_IN * 4);
  L.tg = take((size_t)B * MLP_NQ * 4);
  L.ec = take(sizeof(EpochCtl));
  L.loss = take(16);
  L.raw = take((size_t)B * MLP_OUT * 4);
  L.d_raw = take((size_t)B * MLP_OUT * 4);
  L.xb = take((size_t)B * MLP_IN * 2);
  L.h1 = take((size_t)B * MLP_H * 2);
  L.h2 = take((size_t)B * MLP_H * 2);
  L.d_raw_b = take((size_t)B * MLP_OUT * 2);
  L.dh2 = take((size_t)B * MLP_H * 2);
  L.dh1 = take((size_t)B * MLP_H * 2);
  L.total = off;
  return L;
}

MlpWeights weights_of(const kp_mlp* n) {
  MlpWeights w;
  w.W1 = n->wb;
  w.b1 = n->p + OFF_B1;
  w.W2 = n->wb + MLP_H * MLP_IN;
  w.b2 = n->p + OFF_B2;
  w.W3 = n->wb + MLP_H * MLP_IN + MLP_H * MLP_H;
  w.b3 = n->p + OFF_B3;
  return w;
}

#define MLP_CUDA(call)                            \
  do {                                            \
    if ((call) != cudaSuccess) {                  \
      cudaGetLastError();                         \
      return KP_ERR_CUDA;                         \
    }                                             \
  } while (0)


// Forward with stored activations, loss and the full gradient into n->g.
// ---- tensor-core GEMM launches ----------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows][cols] (row stride ld
// elements, a multiple of 8; base 16-byte aligned) read in 64-column x
// 128-row boxes with the 128-byte swizzle; reads outside [rows][cols] give 0.
bool tile_map(CUtensorMap* m, const bf16* base, int rows, int cols, int ld) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || ((uintptr_t)base & 15u) || (ld % 8) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T on the tensor cores: A [M][K] (row stride lda), B [N][K] (row
// stride ldb), both BF16 and K-major.  EPI_ATOMIC_F32 splits K over up to
// 'max_split' CTAs per tile.
template <int EPI>
kp_status tc_gemm(const kp_mlp* n, const bf16* A, int lda, const bf16* B, int ldb, int M, int N,
                  int K, tc::TcArgs args, int max_split) {
  CUtensorMap ta, tb;
  if (!tile_map(&ta, A, M, K, lda) || !tile_map(&tb, B, N, K, ldb)) return KP_ERR_CUDA;
  const int kt_all = (K + tc::BK - 1) / tc::BK;
  int split = EPI == tc::EPI_ATOMIC_F32 ? (max_split < kt_all ? max_split : kt_all) : 1;
  const int per = (kt_all + split - 1) / split;
  split = (kt_all + per - 1) / per;  // no empty split
  args.M = M;
  args.N = N;
  args.K = K;
  args.kt_per_split = per;
  args.err = n->err;
  args.wait_ns = 2000000000ull;
  dim3 grid((N + tc::BN - 1) / tc::BN, (M + tc::BM - 1) / tc::BM, split);
  tc::tc_gemm_kernel<EPI><<<grid, 128, tc::SMEM_BYTES, n->stream>>>(ta, tb, args);
  MLP_CUDA(cudaGetLastError());
  return KP_OK;
}

// KP_ERR_TIMEOUT once a tensor-core kernel's bounded wait has expired (the
// word is sticky until the parameters are set again).  Stream synchronised.
// Raises the dynamic shared memory limit of the tensor-core GEMM kernels
// (done once, outside any stream capture).
kp_status tc_configure() {
  static bool done = false;
  if (!done) {
    MLP_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<tc::EPI_ATOMIC_F32>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    MLP_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<tc::EPI_MASK_BF16>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    MLP_CUDA(cudaFuncSetAttribute(tc::tc_gemm_kernel<tc::EPI_BIAS_RELU_BF16>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
    done = true;
  }
  return KP_OK;
}

kp_status device_error(const kp_mlp* n) {
  int e = 0;
  MLP_CUDA(cudaMemcpy(&e, n->err, 4, cudaMemcpyDeviceToHost));
  return e ? KP_ERR_TIMEOUT : KP_OK;
}

kp_status forward_backward(kp_mlp* n, const float* x, const float* t, int M) {
  MlpWeights w = weights_of(n);
  {
    const kp_status s0 = tc_configure();
    if (s0 != KP_OK) return s0;
  }
  MLP_CUDA(cudaMemsetAsync(n->g, 0, (size_t)N_PARAMS * 4, n->stream));
  MLP_CUDA(cudaMemsetAsync(n->loss, 0, 4, n->stream));
  kp_mlp_forward_kernel<<<(M + MLP_TILE - 1) / MLP_TILE, 256, 0, n->stream>>>(
      w, x, M, n->raw, nullptr, n->xb, n->h1, n->h2, n->xbt, n->ldt);
  MLP_CUDA(cudaGetLastError());
  kp_mlp_head_loss_kernel<<<(M + 255) / 256, 256, 0, n->stream>>>(
      n->raw, t, M, n->d_raw, n->d_raw_b, n->loss, n->drawt, n->ldt, n->g + OFF_B3);
  MLP_CUDA(cudaGetLastError());
  const dim3 tgrid_h((M + 31) / 32, MLP_H / 32);
  kp_mlp_transpose_kernel<<<tgrid_h, 256, 0, n->stream>>>(n->h2, M, MLP_H, n->h2t, n->ldt);
  MLP_CUDA(cudaGetLastError());
  kp_mlp_transpose_kernel<<<tgrid_h, 256, 0, n->stream>>>(n->h1, M, MLP_H, n->h1t, n->ldt);
  MLP_CUDA(cudaGetLastError());
  kp_status s;
  {
    // output layer: dW3 [8][256] = d_raw^T h2
    tc::TcArgs a{};
    a.cf = n->g + OFF_W3;
    a.ldc = MLP_H;
    s = tc_gemm<tc::EPI_ATOMIC_F32>(n, n->drawt, n->ldt, n->h2t, n->ldt, MLP_OUT, MLP_H, M, a, 16);
    if (s != KP_OK) return s;
  }
  // second layer: dh2 = d_raw W3 masked by h2 > 0 (and its transpose)
  kp_mlp_dh2_kernel<<<(M + 31) / 32, MLP_H, 0, n->stream>>>(n->d_raw, w.W3, n->h2, M, n->dh2,
                                                            n->dh2t, n->ldt);
  MLP_CUDA(cudaGetLastError());
  {
    // dW2 [out][in] = dh2^T h1
    tc::TcArgs a{};
    a.cf = n->g + OFF_W2;
    a.ldc = MLP_H;
    s = tc_gemm<tc::EPI_ATOMIC_F32>(n, n->dh2t, n->ldt, n->h1t, n->ldt, MLP_H, MLP_H, M, a, 8);
    if (s != KP_OK) return s;
  }
  kp_mlp_rowsum_kernel<<<dim3(MLP_H, (M + 1023) / 1024), 256, 0, n->stream>>>(n->dh2t, MLP_H, M, n->ldt,
                                                                n->g + OFF_B2);
  MLP_CUDA(cudaGetLastError());
  {
    // first layer: dh1 = (dh2 W2) masked by h1 > 0, and its transpose
    tc::TcArgs a{};
    a.mask = n->h1;
    a.cb = n->dh1;
    a.cbt = n->dh1t;
    a.ldc = MLP_H;
    a.ldt = n->ldt;
    s = tc_gemm<tc::EPI_MASK_BF16>(n, n->dh2, MLP_H, n->w2t, MLP_H, M, MLP_H, MLP_H, a, 1);
    if (s != KP_OK) return s;
  }
  {
    // dW1 [256][32] = dh1^T x
    tc::TcArgs a{};
    a.cf = n->g + OFF_W1;
    a.ldc = MLP_IN;
    s = tc_gemm<tc::EPI_ATOMIC_F32>(n, n->dh1t, n->ldt, n->xbt, n->ldt, MLP_H, MLP_IN, M, a, 8);
    if (s != KP_OK) return s;
  }
  kp_mlp_rowsum_kernel<<<dim3(MLP_H, (M + 1023) / 1024), 256, 0, n->stream>>>(n->dh1t, MLP_H, M, n->ldt,
                                                                n->g + OFF_B1);
  MLP_CUDA(cudaGetLastError());
  return KP_OK;
}

}  // namespace

extern "C" {

size_t kp_mlp_required_bytes(int32_t max_batch) {
  if (max_batch < 1 || max_batch > (1 << 24)) return 0;
  return mlp_layout(max_batch).total;
}

kp_status kp_mlp_create(void* dev_arena, size_t arena_bytes, int32_t max_batch,
                        const float* host_params, void* cuda_stream, kp_mlp** out) {
  if (!out || !dev_arena || ((uintptr_t)dev_arena & 255u) || !host_params) return KP_ERR_ARG;
  *out = nullptr;
  if (max_batch < 1 || max_batch > (1 << 24)) return KP_ERR_ARG;
  const MlpLayout L = mlp_layout(max_batch);
  if (arena_bytes < L.total) return KP_ERR_OOM;
  kp_mlp* n = new (std::nothrow) kp_mlp();
  if (!n) return KP_ERR_OOM;
  n->arena = static_cast<char*>(dev_arena);
  n->bytes = arena_bytes;
  n->stream = static_cast<cudaStream_t>(cuda_stream);
  n->max_batch = max_batch;
  char* A = n->arena;
  n->p = reinterpret_cast<float*>(A + L.p);
  n->m = reinterpret_cast<float*>(A + L.m);
  n->v = reinterpret_cast<float*>(A + L.v);
  n->g = reinterpret_cast<float*>(A + L.g);
  n->wb = reinterpret_cast<bf16*>(A + L.wb);
  n->wf = reinterpret_cast<bf16*>(A + L.wf);
  n->w2t = reinterpret_cast<bf16*>(A + L.w2t);
  n->dh2t = reinterpret_cast<bf16*>(A + L.dh2t);
  n->h1t = reinterpret_cast<bf16*>(A + L.h1t);
  n->h2t = reinterpret_cast<bf16*>(A + L.h2t);
  n->dh1t = reinterpret_cast<bf16*>(A + L.dh1t);
  n->xbt = reinterpret_cast<bf16*>(A + L.xbt);
  n->drawt = reinterpret_cast<bf16*>(A + L.drawt);
  n->ldt = ld_t(max_batch);
  n->err = reinterpret_cast<int*>(A + L.err);
  n->xg = reinterpret_cast<float*>(A + L.xg);
  n->tg = reinterpret_cast<float*>(A + L.tg);
  n->ec = reinterpret_cast<EpochCtl*>(A + L.ec);
  n->loss = reinterpret_cast<float*>(A + L.loss);
  n->raw = reinterpret_cast<float*>(A + L.raw);
  n->d_raw = reinterpret_cast<float*>(A + L.d_raw);
  n->xb = reinterpret_cast<bf16*>(A + L.xb);
  n->h1 = reinterpret_cast<bf16*>(A + L.h1);
  n->h2 = reinterpret_cast<bf16*>(A + L.h2);
  n->d_raw_b = reinterpret_cast<bf16*>(A + L.d_raw_b);
  n->dh2 = reinterpret_cast<bf16*>(A + L.dh2);
  n->dh1 = reinterpret_cast<bf16*>(A + L.dh1);
  kp_status s = kp_mlp_set_params(n, host_params);
  if (s != KP_OK) {
    delete n;
    return s;
  }
  *out = n;
  return KP_OK;
}

kp_status kp_mlp_set_params(kp_mlp* n, const float* host_params) {
  if (!n || !host_params) return KP_ERR_ARG;
  for (int i = 0; i < N_PARAMS; ++i)
    if (!std::isfinite(host_params[i])) return KP_ERR_ARG;
  MLP_CUDA(cudaMemcpyAsync(n->p, host_params, (size_t)N_PARAMS * 4, cudaMemcpyHostToDevice,
                           n->stream));
  MLP_CUDA(cudaMemsetAsync(n->m, 0, (size_t)N_PARAMS * 4, n->stream));
  MLP_CUDA(cudaMemsetAsync(n->v, 0, (size_t)N_PARAMS * 4, n->stream));
  MLP_CUDA(cudaMemsetAsync(n->err, 0, 16, n->stream));
  kp_mlp_round_kernel<<<(N_PARAMS + 255) / 256, 256, 0, n->stream>>>(n->p, n->wb, n->wf, n->w2t);
  MLP_CUDA(cudaGetLastError());
  MLP_CUDA(cudaStreamSynchronize(n->stream));
  n->step = 0;
  return KP_OK;
}

kp_status kp_mlp_get_params(kp_mlp* n, float* host_params) {
  if (!n || !host_params) return KP_ERR_ARG;
  MLP_CUDA(cudaMemcpyAsync(host_params, n->p, (size_t)N_PARAMS * 4, cudaMemcpyDeviceToHost,
                           n->stream));
  MLP_CUDA(cudaStreamSynchronize(n->stream));
  return KP_OK;
}

int32_t kp_mlp_num_params(void) { return N_PARAMS; }

kp_status kp_mlp_forward(kp_mlp* n, const float* dev_x, int32_t M, float* dev_out) {
  if (!n || !dev_x || !dev_out || M < 0 || M > n->max_batch) return KP_ERR_ARG;
  if (M == 0) return KP_OK;
  kp_mlp_forward_kernel<<<(M + MLP_TILE - 1) / MLP_TILE, 256, 0, n->stream>>>(
      weights_of(n), dev_x, M, n->raw, dev_out, nullptr, nullptr, nullptr, nullptr, 0);
  MLP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status kp_mlp_gradients(kp_mlp* n, const float* dev_x, const float* dev_t, int32_t M,
                           float* host_grad, float* host_loss) {
  if (!n || !dev_x || !dev_t || M < 1 || M > n->max_batch) return KP_ERR_ARG;
  kp_status s = forward_backward(n, dev_x, dev_t, M);
  if (s != KP_OK) return s;
  if (host_grad)
    MLP_CUDA(cudaMemcpyAsync(host_grad, n->g, (size_t)N_PARAMS * 4, cudaMemcpyDeviceToHost,
                             n->stream));
  if (host_loss)
    MLP_CUDA(cudaMemcpyAsync(host_loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
  MLP_CUDA(cudaStreamSynchronize(n->stream));
  return device_error(n);
}

kp_status kp_mlp_train_step(kp_mlp* n, const float* dev_x, const float* dev_t, int32_t M,
                            float lr, float* host_loss) {
  if (!n || !dev_x || !dev_t || M < 1 || M > n->max_batch || !(lr > 0.0f)) return KP_ERR_ARG;
  kp_status s = forward_backward(n, dev_x, dev_t, M);
  if (s != KP_OK) return s;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)n->step), c2 = 1.0f - powf(b2, (float)n->step);
  kp_mlp_adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, n->stream>>>(n->p, n->g, n->m, n->v,
                                                                    N_PARAMS, lr, b1, b2, 1e-8f,
                                                                    c1, c2, n->wb, n->wf,
                                                                    n->w2t);
  MLP_CUDA(cudaGetLastError());
  if (host_loss) {
    MLP_CUDA(cudaMemcpyAsync(host_loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
    MLP_CUDA(cudaStreamSynchronize(n->stream));
    return device_error(n);
  }
  return KP_OK;
}

kp_status kp_mlp_train_epoch(kp_mlp* n, const float* dev_x, const float* dev_t,
                             const int32_t* dev_perm, int64_t rows, float lr, float* host_loss) {
  if (!n || !dev_x || !dev_t || !dev_perm || rows < 0 || !(lr > 0.0f)) return KP_ERR_ARG;
  const int B = n->max_batch;
  const int64_t nb = rows / B;
  if (host_loss) *host_loss = 0.0f;
  if (nb == 0) return KP_OK;
  if (nb > (1 << 30)) return KP_ERR_ARG;
  if (!n->gstream) {
    MLP_CUDA(cudaStreamCreateWithFlags(&n->gstream, cudaStreamNonBlocking));
    MLP_CUDA(cudaEventCreateWithFlags(&n->gev, cudaEventDisableTiming));
  }
  // the epoch runs after the work already queued on the caller's stream
  MLP_CUDA(cudaEventRecord(n->gev, n->stream));
  MLP_CUDA(cudaStreamWaitEvent(n->gstream, n->gev, 0));
  EpochCtl h{dev_x, dev_t, dev_perm, 0, n->step, lr, 0.0f};
  MLP_CUDA(cudaMemcpyAsync(n->ec, &h, sizeof(EpochCtl), cudaMemcpyHostToDevice, n->gstream));
  if (!n->graph_exec) {
    // one mini-batch step: gather, forward, backward (tensor-core GEMMs), Adam
    kp_status s = tc_configure();
    if (s != KP_OK) return s;
    cudaStream_t user = n->stream;
    n->stream = n->gstream;
    if (cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      n->stream = user;
      cudaGetLastError();
      return KP_ERR_CUDA;
    }
    kp_mlp_gather_kernel<<<(B * (MLP_IN + MLP_NQ) + 255) / 256, 256, 0, n->stream>>>(n->ec, B, n->xg,
                                                                                   n->tg);
    s = forward_backward(n, n->xg, n->tg, B);
    kp_mlp_adam_dev_kernel<<<(N_PARAMS + 255) / 256, 256, 0, n->stream>>>(
        n->p, n->g, n->m, n->v, N_PARAMS, n->ec, n->wb, n->wf, n->w2t);
    kp_mlp_epoch_tail_kernel<<<1, 1, 0, n->stream>>>(n->ec, n->loss);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(n->stream, &g);
    n->stream = user;
    if (s != KP_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s != KP_OK ? s : KP_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&n->graph_exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      n->graph_exec = nullptr;
      cudaGetLastError();
      return KP_ERR_CUDA;
    }
    n->graph = g;
  }
  for (int64_t b = 0; b < nb; ++b) MLP_CUDA(cudaGraphLaunch(n->graph_exec, n->gstream));
  n->step += (int)nb;
  EpochCtl out{};
  MLP_CUDA(cudaMemcpyAsync(&out, n->ec, sizeof(EpochCtl), cudaMemcpyDeviceToHost, n->gstream));
  MLP_CUDA(cudaStreamSynchronize(n->gstream));
  if (host_loss) *host_loss = out.loss_sum / (float)nb;
  return device_error(n);
}

void kp_mlp_destroy(kp_mlp* n) {
  if (!n) return;
  if (n->graph_exec) cudaGraphExecDestroy(n->graph_exec);
  if (n->graph) cudaGraphDestroy(n->graph);
  if (n->gev) cudaEventDestroy(n->gev);
  if (n->gstream) cudaStreamDestroy(n->gstream);
  delete n;
}

}  // extern "C"

namespace kp {
// Device pointers of the network's weights for the planner's loop kernel:
// BF16 weights in fragment order (frag_index_hidden / frag_index_out), FP32
// biases.
void mlp_device_weights(const kp_mlp* n, const void** W1, const float** b1, const void** W2,
                        const float** b2, const void** W3, const float** b3) {
  MlpWeights w = weights_of(n);
  w.W1 = n->wf;
  w.W2 = n->wf + MLP_H * MLP_IN;
  w.W3 = n->wf + MLP_H * MLP_IN + MLP_H * MLP_H;
  *W1 = w.W1;
  *b1 = w.b1;
  *W2 = w.W2;
  *b2 = w.b2;
  *W3 = w.W3;
  *b3 = w.b3;
}
}  // namespace kp
