// kp_mlp.cu -- the learned proposal's network: inference and training
// kernels (BF16 tensor-core products, FP32 accumulation, FP32 master
// weights and Adam moments) and the kp_mlp_* entry points of include/kp.h.
// Like the planner, the network context allocates no device memory: it
// lives in a caller-owned arena.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "../../include/kp.h"
#include "kp_mlp.cuh"

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
                                                             bf16* xb, bf16* h1, bf16* h2) {
  __shared__ __align__(16) bf16 sX[MLP_TILE * MLP_XS];
  __shared__ __align__(16) bf16 sH[MLP_TILE * MLP_HS];
  const int row0 = blockIdx.x * MLP_TILE;
  const int rows = M - row0 < MLP_TILE ? M - row0 : MLP_TILE;
  for (int e = threadIdx.x; e < MLP_TILE * MLP_IN; e += blockDim.x) {
    const int r = e / MLP_IN, c = e % MLP_IN;
    const bf16 v = __float2bfloat16_rn(r < rows ? x[(size_t)(row0 + r) * MLP_IN + c] : 0.0f);
    sX[r * MLP_XS + c] = v;
    if (xb && r < rows) xb[(size_t)(row0 + r) * MLP_IN + c] = v;
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
                                        bf16* d_raw_b, float* loss) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
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
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l / (float)M);
}

// dh2[m][k] = (sum_n d_raw[m][n] W3[n][k]) where h2[m][k] > 0, else 0.
__global__ void kp_mlp_dh2_kernel(const float* d_raw, const bf16* W3, const bf16* h2, int M,
                                  bf16* dh2) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)M * MLP_H) return;
  const int m = (int)(e / MLP_H), k = (int)(e % MLP_H);
  float s = 0.0f;
#pragma unroll
  for (int n = 0; n < MLP_OUT; ++n)
    s = fmaf(d_raw[(size_t)m * MLP_OUT + n], __bfloat162float(W3[n * MLP_H + k]), s);
  dh2[e] = __float2bfloat16_rn(__bfloat162float(h2[e]) > 0.0f ? s : 0.0f);
}

// Column sums of a [M][N] matrix (FP32 or BF16) added to g[0..N).
template <typename T>
__global__ void kp_mlp_colsum_kernel(const T* a, int M, int N, float* g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int per = (M + gridDim.y - 1) / gridDim.y;
  const int m0 = blockIdx.y * per, m1 = m0 + per < M ? m0 + per : M;
  float s = 0.0f;
  for (int m = m0; m < m1; ++m) s += (float)a[(size_t)m * N + n];
  if (m1 > m0) atomicAdd(g + n, s);
}

// C[M x N] (+)= sum_r A(m, r) B(r, n) on BF16 tensor cores, FP32 accumulate.
//   A(m, r) = A[m * lda + r]  (A_COL false)  or A[r * lda + m]  (A_COL true)
//   B(r, n) = B[n * ldb + r]  (B_RN false)   or B[r * ldb + n]  (B_RN true)
// EPI 0: atomically add to Cf[m * ldc + n] (split over r by gridDim.z);
// EPI 1: Cb[m * ldc + n] = bf16(C) where mask[m * ldc + n] > 0, else 0.
// Tiles of 64 x 64 x 32 are staged in shared memory with the reduction
// index contiguous; 4 warps each compute 32 x 32.
constexpr int GT = 64, GR = 32, GS = GR + 8;
template <bool A_COL, bool B_RN, int EPI>
__global__ void __launch_bounds__(128) kp_mlp_gemm_kernel(const bf16* A, int lda, const bf16* B,
                                                          int ldb, int M, int N, int R, float* Cf,
                                                          bf16* Cb, int ldc, const bf16* mask) {
  __shared__ __align__(16) bf16 As[GT * GS];
  __shared__ __align__(16) bf16 Bs[GT * GS];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int per = (R + gridDim.z - 1) / gridDim.z;
  const int rs = blockIdx.z * per, re = rs + per < R ? rs + per : R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4] = {};
  const bf16 zero = __float2bfloat16_rn(0.0f);
  for (int r0 = rs; r0 < re; r0 += GR) {
    for (int e = threadIdx.x; e < GT * GR; e += blockDim.x) {
      int m, r;
      if (A_COL) { r = e / GT; m = e % GT; } else { m = e / GR; r = e % GR; }
      const int gm = m0 + m, gr = r0 + r;
      bf16 v = zero;
      if (gm < M && gr < re) v = A_COL ? A[(size_t)gr * lda + gm] : A[(size_t)gm * lda + gr];
      As[m * GS + r] = v;
    }
    for (int e = threadIdx.x; e < GT * GR; e += blockDim.x) {
      int n, r;
      if (B_RN) { r = e / GT; n = e % GT; } else { n = e / GR; r = e % GR; }
      const int gn = n0 + n, gr = r0 + r;
      bf16 v = zero;
      if (gn < N && gr < re) v = B_RN ? B[(size_t)gr * ldb + gn] : B[(size_t)gn * ldb + gr];
      Bs[n * GS + r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k0 = 0; k0 < GR; k0 += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) frag_a(As, GS, wm + mi * 16, k0, a[mi]);
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) frag_b(Bs, GS, wn + ni * 8, k0, b[ni]);
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mi * 16 + g + 8 * (q >> 1);
        const int n = n0 + wn + ni * 8 + 2 * t + (q & 1);
        if (m >= M || n >= N) continue;
        const size_t o = (size_t)m * ldc + n;
        if (EPI == 0) {
          atomicAdd(Cf + o, acc[mi][ni][q]);
        } else {
          Cb[o] = __float2bfloat16_rn(__bfloat162float(mask[o]) > 0.0f ? acc[mi][ni][q] : 0.0f);
        }
      }
}

// Adam on the FP32 master vector; refreshes the BF16 weight copies.
// Parameter i rounded to BF16 into the row-major weight copy (training
// kernels) and into the fragment-order copy (the planner's loop kernel).
__device__ __forceinline__ void store_weight(int i, float pi, bf16* wb, bf16* wf) {
  const bf16 b = __float2bfloat16_rn(pi);
  if (i < OFF_B1) {
    wb[i] = b;
    wf[frag_index_hidden(i / MLP_IN, i % MLP_IN, MLP_IN)] = b;
  } else if (i >= OFF_W2 && i < OFF_B2) {
    const int j = i - OFF_W2;
    wb[MLP_H * MLP_IN + j] = b;
    wf[MLP_H * MLP_IN + frag_index_hidden(j / MLP_H, j % MLP_H, MLP_H)] = b;
  } else if (i >= OFF_W3 && i < OFF_B3) {
    const int j = i - OFF_W3;
    wb[MLP_H * MLP_IN + MLP_H * MLP_H + j] = b;
    wf[MLP_H * MLP_IN + MLP_H * MLP_H + frag_index_out(j / MLP_H, j % MLP_H)] = b;
  }
}

__global__ void kp_mlp_adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr,
                                   float beta1, float beta2, float eps, float c1, float c2,
                                   bf16* wb, bf16* wf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  store_weight(i, pi, wb, wf);
}

__global__ void kp_mlp_round_kernel(const float* p, bf16* wb, bf16* wf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N_PARAMS) return;
  store_weight(i, p[i], wb, wf);
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
  float *raw, *d_raw, *loss;
  bf16 *xb, *h1, *h2, *d_raw_b, *dh2, *dh1;
};

namespace {

struct MlpLayout {
  size_t p, m, v, g, wb, wf, loss, raw, d_raw, xb, h1, h2, d_raw_b, dh2, dh1, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

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

template <bool AC, bool BR, int EPI>
kp_status gemm(const kp_mlp* n, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int R,
               float* Cf, bf16* Cb, int ldc, const bf16* mask, int split) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, split);
  kp_mlp_gemm_kernel<AC, BR, EPI><<<grid, 128, 0, n->stream>>>(A, lda, B, ldb, M, N, R, Cf, Cb,
                                                               ldc, mask);
  MLP_CUDA(cudaGetLastError());
  return KP_OK;
}

// Forward with stored activations, loss and the full gradient into n->g.
kp_status forward_backward(kp_mlp* n, const float* x, const float* t, int M) {
  MlpWeights w = weights_of(n);
  MLP_CUDA(cudaMemsetAsync(n->g, 0, (size_t)N_PARAMS * 4, n->stream));
  MLP_CUDA(cudaMemsetAsync(n->loss, 0, 4, n->stream));
  kp_mlp_forward_kernel<<<(M + MLP_TILE - 1) / MLP_TILE, 256, 0, n->stream>>>(
      w, x, M, n->raw, nullptr, n->xb, n->h1, n->h2);
  MLP_CUDA(cudaGetLastError());
  kp_mlp_head_loss_kernel<<<(M + 255) / 256, 256, 0, n->stream>>>(n->raw, t, M, n->d_raw,
                                                                  n->d_raw_b, n->loss);
  MLP_CUDA(cudaGetLastError());
  const int split = (M + 255) / 256 < 64 ? (M + 255) / 256 : 64;
  // output layer: dW3 = d_raw^T h2, db3 = column sums of d_raw
  kp_status s = gemm<true, true, 0>(n, n->d_raw_b, MLP_OUT, n->h2, MLP_H, MLP_OUT, MLP_H, M,
                                    n->g + OFF_W3, nullptr, MLP_H, nullptr, split);
  if (s != KP_OK) return s;
  kp_mlp_colsum_kernel<float><<<dim3(1, 32), 256, 0, n->stream>>>(n->d_raw, M, MLP_OUT,
                                                                   n->g + OFF_B3);
  MLP_CUDA(cudaGetLastError());
  // second layer: dh2 = d_raw W3 masked by h2 > 0; dW2 = dh2^T h1; db2
  kp_mlp_dh2_kernel<<<(int)(((size_t)M * MLP_H + 255) / 256), 256, 0, n->stream>>>(
      n->d_raw, w.W3, n->h2, M, n->dh2);
  MLP_CUDA(cudaGetLastError());
  s = gemm<true, true, 0>(n, n->dh2, MLP_H, n->h1, MLP_H, MLP_H, MLP_H, M, n->g + OFF_W2, nullptr,
                          MLP_H, nullptr, split);
  if (s != KP_OK) return s;
  kp_mlp_colsum_kernel<bf16><<<dim3(1, 64), 256, 0, n->stream>>>(n->dh2, M, MLP_H, n->g + OFF_B2);
  MLP_CUDA(cudaGetLastError());
  // first layer: dh1 = dh2 W2 masked by h1 > 0; dW1 = dh1^T x; db1
  s = gemm<false, true, 1>(n, n->dh2, MLP_H, w.W2, MLP_H, M, MLP_H, MLP_H, nullptr, n->dh1, MLP_H,
                           n->h1, 1);
  if (s != KP_OK) return s;
  s = gemm<true, true, 0>(n, n->dh1, MLP_H, n->xb, MLP_IN, MLP_H, MLP_IN, M, n->g + OFF_W1,
                          nullptr, MLP_IN, nullptr, split);
  if (s != KP_OK) return s;
  kp_mlp_colsum_kernel<bf16><<<dim3(1, 64), 256, 0, n->stream>>>(n->dh1, M, MLP_H, n->g + OFF_B1);
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
  kp_mlp_round_kernel<<<(N_PARAMS + 255) / 256, 256, 0, n->stream>>>(n->p, n->wb, n->wf);
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
      weights_of(n), dev_x, M, n->raw, dev_out, nullptr, nullptr, nullptr);
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
  return KP_OK;
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
                                                                    c1, c2, n->wb, n->wf);
  MLP_CUDA(cudaGetLastError());
  if (host_loss) {
    MLP_CUDA(cudaMemcpyAsync(host_loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
    MLP_CUDA(cudaStreamSynchronize(n->stream));
  }
  return KP_OK;
}

void kp_mlp_destroy(kp_mlp* n) { delete n; }

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
