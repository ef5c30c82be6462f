// kp_launch.cuh -- host launchers of one system's kernels.  Included once by
// each kp_sys_*.cu with KP_SYS set, so the three systems compile in
// parallel translation units.
#pragma once

#include <cuda_runtime.h>

#include "kp_loop.cuh"

#define KP_CAT2(a, b) a##b
#define KP_CAT(a, b) KP_CAT2(a, b)

namespace kp {

cudaError_t KP_CAT(loop_occupancy_, KP_SYS_NAME)(bool log, size_t smem, int* blocks_per_sm) {
  const void* f = log ? (const void*)kp_loop_kernel<KP_SYS, true>
                      : (const void*)kp_loop_kernel<KP_SYS, false>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, KP_BLOCK, smem);
}

cudaError_t KP_CAT(launch_loop_, KP_SYS_NAME)(const KParams& P, int grid, size_t smem,
                                             int max_iters, uint64_t max_ns, bool log,
                                             cudaStream_t stream, const RootState& root,
                                             int mode) {
  KParams p = P;
  int mi = max_iters;
  uint64_t mn = max_ns;
  RootState rs = root;
  int md = mode;
  void* args[] = {&p, &mi, &mn, &rs, &md};
  const void* f = log ? (const void*)kp_loop_kernel<KP_SYS, true>
                      : (const void*)kp_loop_kernel<KP_SYS, false>;
  return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(KP_BLOCK), args, smem, stream);
}

cudaError_t KP_CAT(launch_reset_, KP_SYS_NAME)(const KParams& P, const RootState& root,
                                              cudaStream_t stream) {
  // about four 16-byte stores of the claim table per thread, at least one
  // thread per region
  const size_t n_sub = (size_t)P.R * (size_t)P.n_sub_per;
  size_t blocks = (n_sub + 4095) / 4096;
  const size_t by_region = ((size_t)P.R + 255) / 256;
  if (blocks < by_region) blocks = by_region;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  kp_reset_kernel<KP_SYS><<<(unsigned)blocks, 256, 0, stream>>>(P, root);
  return cudaGetLastError();
}

}  // namespace kp
