// Launchers of the decode kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "decode_warp.cuh"

namespace mcdev {

// Launch set-up shared by the kernel files: raises a kernel's dynamic
// shared-memory limit once per device (prepare) and caches occupancy answers.
void prepare(const void *f);
int occupancy(const void *f, int threads, int smem);
template <class K>
const void *fn(K k) {
  return reinterpret_cast<const void *>(k);
}

uint32_t decode_smem_per_warp(uint32_t max_block_words);
uint32_t cull_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t max_verts,
                            uint32_t per_grab);
uint32_t batch_smem_per_warp(uint32_t max_block_words, uint32_t per_grab);

cudaError_t launch_plain(const BatchArgs &a, uint32_t first, uint32_t count, uint32_t warps,
                         uint32_t max_block_words, bool checked, uint8_t *out_local,
                         uint32_t *out_global, float *out_pos, uint32_t *status, cudaStream_t s);

// vertices: out_pos receives full 8-float vertices (positions + attributes)
cudaError_t launch_batch(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                         uint32_t max_block_words, bool checked, bool vertices,
                         uint8_t *out_local, uint32_t *out_global, float *out_pos,
                         uint32_t *status, uint32_t *scratch, cudaStream_t s);

// order_state (may be NULL): look-back state of the ordered compaction, one
// zeroed 8-byte word per grab
cudaError_t launch_cull(const BatchArgs &a, const float *view_proj, const mc_cone *cones,
                        uint32_t ctas, uint32_t warps, uint32_t per_grab, bool checked,
                        uint32_t *tri_out, uint32_t *tri_count, float *out_pos, uint32_t *status,
                        uint32_t *scratch, uint64_t *order_state, cudaStream_t s);

int max_ctas_per_sm_batch(uint32_t warps, uint32_t max_block_words, uint32_t per_grab,
                          bool vertices = false);
// Two meshlets per warp, 16 lanes each (per_grab >= 2).
cudaError_t launch_batch_pairs(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                               uint32_t max_block_words, bool checked, uint8_t *out_local,
                               uint32_t *out_global, float *out_pos, uint32_t *status,
                               uint32_t *scratch, cudaStream_t s);
int max_ctas_per_sm_batch_pairs(uint32_t warps, uint32_t max_block_words, uint32_t per_grab);
// Multi-view fused cull (1 <= n_views <= 8, per_grab <= 4): view v's
// survivors go to tri_out + v * tri_stride, its count to tri_counts[v].
uint32_t cull_views_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t max_verts,
                                  uint32_t per_grab, uint32_t n_views);
cudaError_t launch_cull_views(const BatchArgs &a, const float *view_projs, uint32_t n_views,
                              const mc_cone *cones, uint32_t ctas, uint32_t warps,
                              uint32_t per_grab, bool checked, uint32_t *tri_out,
                              uint64_t tri_stride, uint32_t *tri_counts, float *out_pos,
                              uint32_t *status, uint32_t *scratch, cudaStream_t s);
int max_ctas_per_sm_cull_views(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                               uint32_t max_verts, uint32_t per_grab, uint32_t n_views);
int max_ctas_per_sm_cull(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                         uint32_t max_verts, uint32_t per_grab);

cudaError_t launch_requests(const BatchArgs &a, const mc_request *reqs, uint32_t n_reqs,
                            uint32_t total_work, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                            bool checked, uint32_t *status, uint32_t *scratch, cudaStream_t s);
int max_ctas_per_sm_requests(uint32_t warps, uint32_t max_block_words);

}  // namespace mcdev
