// Host-only harness of the planner library's host logic, for CPU tests:
// the broad-phase grid of the step-hull test (shape choice, cell lists),
// the kd-tree of the free-space-obeying decomposition (Sec. IV-B) and the
// query server's device-pool allocator.  It compiles the library's host
// code (kp_api.cu) into this unit and calls those parts directly; no
// device code runs.  The launch entry points kp_api.cu refers to are
// stubbed: they report "not supported" and are never called here.
#include "../../paper_2409_06807_gb300/csrc/kp_api.cu"

namespace kp {
void mlp_device_weights(const kp_mlp*, const void** W1, const float** b1, const void** W2,
                        const float** b2, const void** W3, const float** b3) {
  *W1 = *W2 = *W3 = nullptr;
  *b1 = *b2 = *b3 = nullptr;
}
cudaError_t server_occupancy(size_t, int*) { return cudaErrorNotSupported; }
cudaError_t launch_server(const KServerArgs&, int, size_t, cudaStream_t) { return cudaErrorNotSupported; }
#define KPT_STUB_SYS(name)                                                                       \
  cudaError_t loop_occupancy_##name(bool, size_t, int*) { return cudaErrorNotSupported; }       \
  cudaError_t launch_loop_##name(const KParams&, int, size_t, int, uint64_t, bool, cudaStream_t, \
                                 const RootState&, int) {                                      \
    return cudaErrorNotSupported;                                                              \
  }                                                                                            \
  cudaError_t launch_reset_##name(const KParams&, const RootState&, cudaStream_t) {             \
    return cudaErrorNotSupported;                                                              \
  }
KPT_STUB_SYS(di)
KPT_STUB_SYS(dubins)
KPT_STUB_SYS(quad)
#undef KPT_STUB_SYS
}  // namespace kp

namespace {
// The padded box rows the builders read (lo xyz, 0, hi xyz, 0), as the
// blob's first part.
std::vector<float> padded(const float* boxes, int nb) {
  std::vector<float> fb((size_t)((nb + 7) / 8 * 8) * 8, 0.0f);
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      fb[(size_t)b * 8 + a] = boxes[(size_t)b * 6 + a] + 0.0f;
      fb[(size_t)b * 8 + 4 + a] = boxes[(size_t)b * 6 + 3 + a] + 0.0f;
    }
  return fb;
}

kp_workspace unit_workspace(const float lo[3], const float hi[3], const int sub[3]) {
  kp_workspace ws{};
  for (int a = 0; a < 3; ++a) {
    ws.lo[a] = lo[a];
    ws.hi[a] = hi[a];
    ws.grid[a] = 1;
    ws.sub[a] = sub ? sub[a] : 1;
  }
  ws.speed_bins = 1;
  return ws;
}
}  // namespace

extern "C" {

// Builds the obstacle blob of nb boxes (host rows lo xyz, hi xyz) for the
// workspace [lo, hi] into 'blob' (room for max_bytes).  Writes the grid's
// cells per axis, its scale (cells per unit length), the byte offsets of
// the cell starts and of the box ids, of the cells' clearances (-1 without),
// and returns the blob's size.
int kpt_blob(const float* boxes, int nb, const float* lo, const float* hi, int max_bytes,
             unsigned char* blob, int* g3, float* scale3, int* start_off, int* ids_off,
             int* clear_off) {
  const kp_workspace ws = unit_workspace(lo, hi, nullptr);
  KParams P{};
  const size_t bytes = build_blob(blob, nb > 0 ? boxes : nullptr, nb, ws, P, (size_t)max_bytes);
  for (int a = 0; a < 3; ++a) {
    g3[a] = P.bp_g[a];
    scale3[a] = P.bp_scale[a];
  }
  *start_off = P.bp_start_off;
  *ids_off = P.bp_ids_off;
  *clear_off = P.bp_clear_off;
  return (int)bytes;
}

// The arena's room for the obstacle blob (KP_BLOB_BYTES).
int kpt_blob_bytes(void) { return KP_BLOB_BYTES; }

// Builds the kd-tree over the boxes' faces; writes each leaf's box (lo xyz,
// hi xyz) in depth-first order, up to 'cap' leaves.  Returns the leaf
// count, or -1 past the leaf or depth limit.
int kpt_kd_leaves(const float* boxes, int nb, const float* lo, const float* hi, float* leaves,
                  int cap) {
  const std::vector<float> fb = padded(boxes, nb);
  KdTree T;
  std::vector<int> all((size_t)nb);
  for (int b = 0; b < nb; ++b) all[(size_t)b] = b;
  if (!kd_cell(T, fb.data(), all, lo, hi, 0)) return -1;
  const int n = (int)(T.lo.size() / 3);
  for (int r = 0; r < n && r < cap; ++r)
    for (int a = 0; a < 3; ++a) {
      leaves[(size_t)r * 6 + a] = T.lo[(size_t)r * 3 + a];
      leaves[(size_t)r * 6 + 3 + a] = T.hi[(size_t)r * 3 + a];
    }
  return n;
}

// The query server's device-pool allocator (first fit over a free list of
// 256-byte granules, coalescing on free), on a host-only server object
// whose pool is the range [0, bytes).
void* kpt_pool_new(size_t bytes) {
  kp_server* s = new kp_server();
  s->pool_bytes = bytes;
  s->free_list[0] = bytes & ~(size_t)255;
  return s;
}
int kpt_pool_alloc(void* s, size_t bytes, size_t* off) {
  return pool_alloc(static_cast<kp_server*>(s), bytes, off) ? 1 : 0;
}
void kpt_pool_free(void* s, size_t off, size_t bytes) {
  pool_free(static_cast<kp_server*>(s), off, bytes);
}
// Free blocks in offset order (up to cap); returns their count.
int kpt_pool_blocks(void* s, size_t* offs, size_t* sizes, int cap) {
  int n = 0;
  for (const auto& kv : static_cast<kp_server*>(s)->free_list) {
    if (n < cap) {
      offs[n] = kv.first;
      sizes[n] = kv.second;
    }
    ++n;
  }
  return n;
}
void kpt_pool_delete(void* s) { delete static_cast<kp_server*>(s); }

}  // extern "C"
