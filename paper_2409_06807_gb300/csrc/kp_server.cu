// kp_server.cu -- many planning queries in one persistent cooperative
// launch.  The grid is split into teams of blocks; each team repeatedly
// claims the next published query from a host-mapped ring, copies the
// query's parameter block into shared memory, resets the query's arena
// slice, runs the Kino-PAX loop on it (run_loop: the same code as the
// single-query launch), extracts the root-to-goal chain and publishes a
// completion record to host-mapped memory.  A query's result depends on its
// inputs alone (not on its team or on co-running queries).  Every wait is
// bounded: a team with no work for idle_ns leaves, and the host launches the
// server again when new work arrives.
#include <cuda_runtime.h>

#include "kp_layout.h"
#define KP_MIN_BLOCKS 2
#include "kp_loop.cuh"

namespace kp {

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Acquire load at system scope: a published count, after which the ring
// entries the host wrote before it are visible.
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Clears the query's tables (team-strided) and writes its root.
template <int SYS>
__device__ __forceinline__ bool reset_query(const KParams& P, const Team& T, const RootState& root,
                                            KCtl* sctl, uint64_t wait_ns) {
  clear_tables(P, (size_t)T.b * blockDim.x + threadIdx.x, (size_t)T.nb * blockDim.x);
  if (!team_sync(T, sctl, wait_ns, 40)) return false;
  if (T.b == 0) {
    const bool box_free = root_box_free(P, root);
    if (threadIdx.x == 0) init_root<SYS>(P, root, box_free);
  }
  return team_sync(T, sctl, wait_ns, 41);
}

template <int SYS>
__device__ __forceinline__ bool run_query(const KParams& P, const Team& T, const KQuery* q,
                                          unsigned char* blob, LoopShared& sh, KCtl* sctl,
                                          uint64_t wait_ns) {
  // the slot was rewritten by the host since it was last read: L2 reads
  RootState root;
  for (int i = 0; i < 12; ++i)
    root.x[i] = __uint_as_float(__ldcg(reinterpret_cast<const unsigned int*>(&q->root.x[i])));
  if (!reset_query<SYS>(P, T, root, sctl, wait_ns)) return false;
  if (P.ctl->state != KP_DEV_RUNNING) return true;  // bad root or root in goal
  if (!stage_boxes(P, reinterpret_cast<float4*>(blob), sh)) return false;
  const int max_iters = (int)__ldcg(reinterpret_cast<const unsigned int*>(&q->max_iters));
  const uint64_t max_ns = __ldcg(reinterpret_cast<const unsigned long long*>(&q->max_ns));
  return run_loop<SYS, false>(P, T, blob, sh, max_iters, max_ns);
}

__global__ void __launch_bounds__(KP_BLOCK, KP_MIN_BLOCKS) kp_server_kernel(KServerArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LoopShared sh;
  const int team = blockIdx.x / A.team_blocks, b = blockIdx.x % A.team_blocks;
  const int n_teams = gridDim.x / A.team_blocks;
  if (team >= n_teams) return;  // blocks past the last full team stay idle
  KServerDev* dev = A.dev;
  KCtl* sctl = &dev->sctl;
  const Team T{b, A.team_blocks, &dev->team_bar[team][0]};
  KParams& P = *reinterpret_cast<KParams*>(smem);
  unsigned char* blob = smem + ((sizeof(KParams) + 127) & ~(size_t)127);
  for (;;) {
    // the team leader claims the next published query, waiting at most idle_ns
    if (b == 0 && threadIdx.x == 0) {
      uint32_t slot = KS_EXIT;
      const uint64_t t0 = global_ns();
      for (;;) {
        if (ld_volatile(&A.host->stop) || *((volatile int*)&sctl->err)) break;
        const uint32_t posted = ld_acquire_sys(&A.host->posted);
        const uint32_t taken = ld_volatile(&dev->taken);
        if (taken < posted) {
          if (atomicCAS(&dev->taken, taken, taken + 1) == taken) {
            slot = ld_volatile(&A.host->ring[taken % KS_RING]);
            break;
          }
          continue;
        }
        if (global_ns() - t0 > A.idle_ns) break;
        __nanosleep(1000);
      }
      dev->team_slot[team] = slot;
    }
    if (!team_sync(T, sctl, A.wait_ns, 42)) {
      if (b == 0 && threadIdx.x == 0) {
        atomicCAS(&A.host->error, 0, KP_DEV_ERR_TIMEOUT | (sctl->err_where << 8));
        __threadfence_system();
      }
      return;
    }
    const uint32_t slot = ld_volatile(&dev->team_slot[team]);
    if (slot == KS_EXIT) return;
    const KQuery* q = A.queries + slot;
    // the query's parameter block into shared memory (L2 reads: the host
    // rewrote the slot since it was last read)
    for (int i = threadIdx.x; i < (int)(sizeof(KParams) / 4); i += blockDim.x)
      reinterpret_cast<uint32_t*>(&P)[i] = __ldcg(reinterpret_cast<const unsigned int*>(&q->P) + i);
    __syncthreads();
    const uint64_t t_start = global_ns();
    bool ok;
    switch (P.sys) {
      case KP_SYS_DI: ok = run_query<KP_SYS_DI>(P, T, q, blob, sh, sctl, A.wait_ns); break;
      case KP_SYS_DUBINS: ok = run_query<KP_SYS_DUBINS>(P, T, q, blob, sh, sctl, A.wait_ns); break;
      default: ok = run_query<KP_SYS_QUAD>(P, T, q, blob, sh, sctl, A.wait_ns);
    }
    if (!ok || !team_sync(T, sctl, A.wait_ns, 43)) {
      if (b == 0 && threadIdx.x == 0) {
        raise_error(sctl, KP_DEV_ERR_TIMEOUT, 44);
        const int where = P.ctl->err ? P.ctl->err_where : sctl->err_where;
        atomicCAS(&A.host->error, 0, KP_DEV_ERR_TIMEOUT | (where << 8));
        __threadfence_system();
      }
      return;
    }
    if (b == 0) {
      // the chain by the team's first block (the ids in the blob's shared
      // memory, which the next query restages after its claim barrier)
      KCtl* ctl = P.ctl;
      if (ctl->state == KP_DEV_SOLVED) {
        int* ids = reinterpret_cast<int*>(blob);
        int cap = (int)(((size_t)P.blob_bytes + (size_t)P.sd_bytes) / 4);
        if (P.extract_cap > 0 && P.extract_cap < cap) cap = P.extract_cap;
        switch (P.sys) {
          case KP_SYS_DI: extract_chain_block<KP_SYS_DI>(P, ids, cap); break;
          case KP_SYS_DUBINS: extract_chain_block<KP_SYS_DUBINS>(P, ids, cap); break;
          default: extract_chain_block<KP_SYS_QUAD>(P, ids, cap);
        }
      } else if (threadIdx.x == 0) {
        ctl->n_edges = -1;
      }
      __syncthreads();
    }
    if (b == 0 && threadIdx.x == 0) {
      KCtl* ctl = P.ctl;
      const uint32_t seq = atomicAdd(&dev->done_seq, 1u);
      KDone* d = &A.host->done[seq % KS_RING];
      d->slot = (int32_t)slot;
      d->state = ctl->state;
      d->err = ctl->err;
      d->n_edges = ctl->n_edges;
      d->iterations = ctl->iteration;
      d->n_nodes = ctl->n_nodes;
      d->goal_node = ctl->goal_node == KP_NO_GOAL ? -1 : ctl->goal_node;
      d->samples = ctl->tot_samples;
      d->t_start_ns = t_start;
      d->t_end_ns = global_ns();
      __threadfence_system();
      *reinterpret_cast<volatile uint32_t*>(&d->seq) = seq + 1;
      __threadfence_system();
    }
  }
}

cudaError_t server_occupancy(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(kp_server_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kp_server_kernel, KP_BLOCK,
                                                       smem);
}

cudaError_t launch_server(const KServerArgs& A, int grid, size_t smem, cudaStream_t stream) {
  KServerArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)kp_server_kernel, dim3(grid), dim3(KP_BLOCK),
                                     args, smem, stream);
}

}  // namespace kp
