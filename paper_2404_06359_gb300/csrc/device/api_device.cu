// C ABI of the device side: argument checks, launch shapes, the autotuner,
// CUDA-graph capture and the host-buffer (end-to-end) decode.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "meshlet_codec.h"

using namespace mcdev;

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr uint32_t kScratchBytes = 256;

struct Key {
  int device;
  uint32_t n_meshlets, max_block_words;
  uint64_t payload_bytes;
  bool operator<(const Key &o) const {
    return std::tie(device, n_meshlets, max_block_words, payload_bytes) <
           std::tie(o.device, o.n_meshlets, o.max_block_words, o.payload_bytes);
  }
};
std::mutex g_tune_mu;
std::map<Key, mc_tuning> g_tuned;

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

Key key_of(const mc_device_batch *b) {
  int dev = 0;
  cudaGetDevice(&dev);
  return Key{dev, b->n_meshlets, b->max_block_words, b->payload_bytes};
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

mc_status check_batch(const mc_device_batch *b) {
  if (!b || !b->desc || !b->payload || !b->grids) return MC_ERR_INVALID_ARG;
  if (!aligned(b->desc, 16) || !aligned(b->payload, 16) || !aligned(b->grids, 16))
    return MC_ERR_INVALID_ARG;
  if (b->n_grids == 0 || b->n_grids > 65536) return MC_ERR_INVALID_ARG;
  // largest block: 2 x 8 flag words, 64 reuse words, 768 position words and
  // 1280 attribute words (5 channels x 256 vertices x 32 bits), padded
  if (b->max_block_words == 0 || b->max_block_words > 2 * 8 + 64 + 768 + 1280 + 4)
    return MC_ERR_INVALID_ARG;
  if (b->payload_bytes % 16) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets > (1u << 31)) return MC_ERR_LIMIT;  // headroom of the 32-bit work counter
  if (b->max_verts > 256 || (b->max_verts && b->max_verts < 3)) return MC_ERR_INVALID_ARG;
  if (b->cones && !aligned(b->cones, 16)) return MC_ERR_INVALID_ARG;
  if (b->n_attr > 5 || (b->n_attr && (b->attr_bits < 1 || b->attr_bits > 32)))
    return MC_ERR_INVALID_ARG;
  return MC_OK;
}

BatchArgs args_of(const mc_device_batch *b) {
  BatchArgs a;
  a.desc = b->desc;
  a.payload = b->payload;
  a.grids = b->grids;
  a.n_meshlets = b->n_meshlets;
  a.n_grids = b->n_grids;
  a.payload_bytes = b->payload_bytes;
  a.total_tris = b->total_tris;
  a.total_verts = b->total_verts;
  a.max_block_words = b->max_block_words;
  a.max_tris = (b->max_tris == 0 || b->max_tris > 256) ? 256 : b->max_tris;
  a.max_verts = std::min<uint32_t>(b->max_verts ? b->max_verts : 256, std::min(a.max_tris + 2, 256u));
  a.n_attr = b->n_attr;
  a.attr_bits = b->n_attr ? b->attr_bits : 0;
  a.attr_desc = b->attr_desc;
  a.attr_grids = b->attr_grids;
  a.n_attr_grids = b->n_attr_grids;
  a.wait_cycles = 0;
  return a;
}

mc_status from_cuda(cudaError_t e) { return e == cudaSuccess ? MC_OK : MC_ERR_CUDA; }

// Resolves a launch shape for the persistent batch kernel.
mc_tuning resolve_batch(const mc_device_batch *b, const mc_tuning *t) {
  mc_tuning r{};
  if (t) r = *t;
  if (!t || (!r.warps_per_cta && !r.ctas_per_sm && !r.meshlets_per_grab)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key_of(b));
    if (it != g_tuned.end()) {
      uint32_t checked = r.checked;
      r = it->second;
      r.checked = checked;
    }
  }
  if (!r.warps_per_cta) r.warps_per_cta = 8;
  if (!r.meshlets_per_grab) r.meshlets_per_grab = 2;
  if (r.meshlets_per_grab > 16) r.meshlets_per_grab = 16;
  if (r.lanes_per_meshlet != 16) r.lanes_per_meshlet = 32;
  if (r.lanes_per_meshlet == 16 && r.meshlets_per_grab < 2) r.meshlets_per_grab = 2;
  if (!r.ctas_per_sm) {
    int occ = r.lanes_per_meshlet == 16
                  ? max_ctas_per_sm_batch_pairs(r.warps_per_cta, b->max_block_words, r.meshlets_per_grab)
                  : max_ctas_per_sm_batch(r.warps_per_cta, b->max_block_words, r.meshlets_per_grab);
    r.ctas_per_sm = occ > 0 ? (uint32_t)occ : 1;
  }
  return r;
}

mc_status launch_batch_checked(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                               float *d_pos, uint32_t *d_status, void *d_scratch,
                               const mc_tuning &r, cudaStream_t s, bool vertices = false) {
  if (r.warps_per_cta < 1 || r.warps_per_cta > 32 || r.meshlets_per_grab < 1 ||
      r.meshlets_per_grab > 16)
    return MC_ERR_INVALID_ARG;
  // two meshlets per warp: the decoder of positions only, grabs of >= 2
  const bool pairs = r.lanes_per_meshlet == 16 && !vertices;
  auto occ_of = [&](uint32_t g) {
    return pairs ? max_ctas_per_sm_batch_pairs(r.warps_per_cta, b->max_block_words, g)
                 : max_ctas_per_sm_batch(r.warps_per_cta, b->max_block_words, g, vertices);
  };
  // a grab's buffers live in shared memory: shrink the grab until the
  // requested number of warps fits on an SM
  const uint32_t min_grab = pairs ? 2u : 1u;
  uint32_t grab = std::max(r.meshlets_per_grab, min_grab);
  int occ = occ_of(grab);
  while (occ <= 0 && grab > min_grab) occ = occ_of(--grab);
  if (occ <= 0) return MC_ERR_INVALID_ARG;
  uint32_t per_sm = std::min<uint32_t>(r.ctas_per_sm, (uint32_t)occ);
  uint32_t ctas = per_sm * (uint32_t)sm_count();
  if (ctas == 0) return MC_ERR_CUDA;
  cudaError_t e =
      pairs ? launch_batch_pairs(args_of(b), ctas, r.warps_per_cta, grab, b->max_block_words,
                                 r.checked != 0, d_local, d_global, d_pos, d_status,
                                 static_cast<uint32_t *>(d_scratch), s)
            : launch_batch(args_of(b), ctas, r.warps_per_cta, grab, b->max_block_words,
                           r.checked != 0, vertices, d_local, d_global, d_pos, d_status,
                           static_cast<uint32_t *>(d_scratch), s);
  if (e == cudaSuccess) g_launches++;
  return from_cuda(e);
}

}  // namespace

extern "C" size_t mc_scratch_bytes(void) { return kScratchBytes; }

extern "C" uint64_t mc_launch_count(void) { return g_launches.load(); }

extern "C" mc_status mc_decode_plain(const mc_device_batch *b, uint32_t first, uint32_t count,
                                     uint8_t *d_local, uint32_t *d_global, float *d_pos,
                                     uint32_t *d_status, const mc_tuning *t, void *stream) {
  if (!b) return MC_ERR_INVALID_ARG;
  if (count == 0 && first <= b->n_meshlets) return MC_OK;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_pos || (uint64_t)first + count > b->n_meshlets) return MC_ERR_INVALID_ARG;
  uint32_t warps = (t && t->warps_per_cta) ? t->warps_per_cta : 8;
  if (warps > 32) return MC_ERR_INVALID_ARG;
  if (!aligned(d_local, 16) || !aligned(d_global, 16)) return MC_ERR_INVALID_ARG;
  cudaError_t e = launch_plain(args_of(b), first, count, warps, b->max_block_words,
                               t && t->checked, d_local, d_global, d_pos, d_status,
                               static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) g_launches++;
  return from_cuda(e);
}

// ------------------------------------------------ allocation-free variant
//
// mc_decode_batch needs a small caller-provided device scratch buffer for its
// work-queue counters.  Some callers cannot provide one: hosts that own every
// device allocation and forbid libraries from allocating (engines running a
// fixed memory budget), or code paths where a cudaMalloc would implicitly
// synchronise the device in the middle of a frame.  For them the counters
// live in this file-scope device array instead.  It is created when the
// library's device code is loaded and every GPU that loads the library keeps
// it until the process exits; all calls on a device share it.
namespace {
constexpr size_t kNoAllocScratchBytes = 256;  // the counters need mc_scratch_bytes()
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchBytes / 4];
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the name alone is a host-side stand-in, not a device address).
mc_status noalloc_scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MC_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return MC_ERR_LIMIT;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MC_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return MC_OK;
}
}  // namespace

extern "C" mc_status mc_decode_batch_noalloc(const mc_device_batch *b, uint8_t *d_local,
                                             uint32_t *d_global, float *d_pos, uint32_t *d_status,
                                             const mc_tuning *t, void *stream) {
  if (!b) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0) return MC_OK;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_pos || !aligned(d_local, 16) || !aligned(d_global, 16)) return MC_ERR_INVALID_ARG;
  // the fixed array holds the queue counters; the counters are 32-bit, so the
  // batch must leave headroom for the grabs that run past the last meshlet
  if (mc_scratch_bytes() > kNoAllocScratchBytes || b->n_meshlets > (1u << 31)) return MC_ERR_LIMIT;
  void *scratch = nullptr;
  st = noalloc_scratch_address(&scratch);
  if (st != MC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps whatever the previous call left: start from zero
  if (cudaMemsetAsync(scratch, 0, mc_scratch_bytes(), s) != cudaSuccess) return MC_ERR_CUDA;
  mc_tuning r = resolve_batch(b, t);
  return launch_batch_checked(b, d_local, d_global, d_pos, d_status, scratch, r, s);
}

extern "C" mc_status mc_decode_batch(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                                     float *d_pos, uint32_t *d_status, void *d_scratch,
                                     const mc_tuning *t, void *stream) {
  if (!b) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0) return MC_OK;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_pos || !d_scratch || !aligned(d_scratch, 16) || !aligned(d_local, 16) ||
      !aligned(d_global, 16))
    return MC_ERR_INVALID_ARG;
  mc_tuning r = resolve_batch(b, t);
  return launch_batch_checked(b, d_local, d_global, d_pos, d_status, d_scratch, r,
                              static_cast<cudaStream_t>(stream));
}

extern "C" mc_status mc_decode_batch_vertices(const mc_device_batch *b, uint8_t *d_local,
                                              uint32_t *d_global, float *d_vertex,
                                              uint32_t *d_status, void *d_scratch,
                                              const mc_tuning *t, void *stream) {
  if (!b) return MC_ERR_INVALID_ARG;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (b->n_attr == 0 || !b->attr_desc || !b->attr_grids || b->n_attr_grids == 0 ||
      !aligned(b->attr_desc, 16) || !aligned(b->attr_grids, 16))
    return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0) return MC_OK;
  if (!d_vertex || !aligned(d_vertex, 16) || !d_scratch || !aligned(d_scratch, 16) ||
      !aligned(d_local, 16) || !aligned(d_global, 16))
    return MC_ERR_INVALID_ARG;
  mc_tuning r = resolve_batch(b, t);
  return launch_batch_checked(b, d_local, d_global, d_vertex, d_status, d_scratch, r,
                              static_cast<cudaStream_t>(stream), true);
}

namespace {
constexpr uint32_t kOrderedGrabMax = 3;  // two grabs' survivors fit a warp's buffer

mc_status launch_cull_checked(const mc_device_batch *b, const float *d_vp, uint32_t *d_tri_out,
                              uint32_t *d_tri_count, float *d_pos, uint32_t *d_status,
                              void *d_scratch, const mc_tuning *t, cudaStream_t s,
                              uint64_t *d_order = nullptr) {
  const uint32_t warps = (t && t->warps_per_cta) ? t->warps_per_cta : 4;
  uint32_t per_grab = (t && t->meshlets_per_grab) ? t->meshlets_per_grab : 4;
  if (warps < 1 || warps > 32 || per_grab < 1 || per_grab > 16) return MC_ERR_INVALID_ARG;
  if (d_order) per_grab = std::min<uint32_t>(per_grab, kOrderedGrabMax);
  BatchArgs a = args_of(b);
  a.wait_cycles = t ? t->wait_cycles : 0;
  // a grab's survivors are buffered in shared memory: shrink the grab until
  // the requested number of warps fits on an SM
  uint32_t grab = per_grab;
  int occ = max_ctas_per_sm_cull(warps, b->max_block_words, a.max_tris, a.max_verts, grab);
  while (occ <= 0 && grab > 1)
    occ = max_ctas_per_sm_cull(warps, b->max_block_words, a.max_tris, a.max_verts, --grab);
  if (occ <= 0) return MC_ERR_INVALID_ARG;
  uint32_t per_sm = (t && t->ctas_per_sm) ? std::min<uint32_t>(t->ctas_per_sm, occ) : (uint32_t)occ;
  uint32_t ctas = per_sm * (uint32_t)sm_count();
  if (ctas == 0) return MC_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  if (d_order)  // the look-back state starts at "not published" for every grab
    e = cudaMemsetAsync(d_order, 0, 8ull * ((b->n_meshlets + grab - 1) / grab), s);
  if (e == cudaSuccess)
    e = launch_cull(a, d_vp, b->cones, ctas, warps, grab, t && t->checked, d_tri_out, d_tri_count,
                    d_pos, d_status, static_cast<uint32_t *>(d_scratch), d_order, s);
  if (e == cudaSuccess) g_launches++;
  return from_cuda(e);
}
}  // namespace

extern "C" mc_status mc_decode_cull(const mc_device_batch *b, const float *d_view_proj,
                                    uint32_t *d_tri_out, uint32_t *d_tri_count, float *d_pos,
                                    uint32_t *d_status, void *d_scratch, const mc_tuning *t,
                                    void *stream) {
  if (!b || !d_tri_count) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0)
    return from_cuda(cudaMemsetAsync(d_tri_count, 0, 4, static_cast<cudaStream_t>(stream)));
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_view_proj || !d_tri_out || !d_pos || !d_scratch || !aligned(d_scratch, 16))
    return MC_ERR_INVALID_ARG;
  return launch_cull_checked(b, d_view_proj, d_tri_out, d_tri_count, d_pos, d_status, d_scratch, t,
                             static_cast<cudaStream_t>(stream));
}

namespace {
constexpr uint32_t kViewsGrabMax = 4;  // meshlets per grab of the multi-view cull (8 bits each)

mc_status launch_cull_views_checked(const mc_device_batch *b, const float *d_vps, uint32_t n_views,
                                    uint32_t *d_tri_out, uint64_t tri_stride,
                                    uint32_t *d_tri_counts, float *d_pos, uint32_t *d_status,
                                    void *d_scratch, const mc_tuning *t, cudaStream_t s) {
  const uint32_t warps = (t && t->warps_per_cta) ? t->warps_per_cta : 4;
  uint32_t per_grab = (t && t->meshlets_per_grab) ? t->meshlets_per_grab : kViewsGrabMax;
  if (warps < 1 || warps > 32 || per_grab < 1 || per_grab > 16) return MC_ERR_INVALID_ARG;
  per_grab = std::min(per_grab, kViewsGrabMax);
  const BatchArgs a = args_of(b);
  uint32_t grab = per_grab;
  int occ = max_ctas_per_sm_cull_views(warps, b->max_block_words, a.max_tris, a.max_verts, grab,
                                       n_views);
  while (occ <= 0 && grab > 1)
    occ = max_ctas_per_sm_cull_views(warps, b->max_block_words, a.max_tris, a.max_verts, --grab,
                                     n_views);
  if (occ <= 0) return MC_ERR_INVALID_ARG;
  uint32_t per_sm = (t && t->ctas_per_sm) ? std::min<uint32_t>(t->ctas_per_sm, occ) : (uint32_t)occ;
  uint32_t ctas = per_sm * (uint32_t)sm_count();
  if (ctas == 0) return MC_ERR_CUDA;
  cudaError_t e = launch_cull_views(a, d_vps, n_views, b->cones, ctas, warps, grab,
                                    t && t->checked, d_tri_out, tri_stride, d_tri_counts, d_pos,
                                    d_status, static_cast<uint32_t *>(d_scratch), s);
  if (e == cudaSuccess) g_launches++;
  return from_cuda(e);
}

mc_status check_cull_views(const mc_device_batch *b, const float *d_view_projs, uint32_t n_views,
                           uint32_t *d_tri_out, uint64_t tri_stride, uint32_t *d_tri_counts,
                           float *d_pos, void *d_scratch) {
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_view_projs || !aligned(d_view_projs, 4) || n_views == 0 || !d_tri_out ||
      !aligned(d_tri_out, 4) || !d_tri_counts || !d_pos || !d_scratch || !aligned(d_scratch, 16) ||
      tri_stride < 3 * b->total_tris)
    return MC_ERR_INVALID_ARG;
  return MC_OK;
}
}  // namespace

extern "C" mc_status mc_decode_cull_views(const mc_device_batch *b, const float *d_view_projs,
                                          uint32_t n_views, uint32_t *d_tri_out,
                                          uint64_t tri_stride, uint32_t *d_tri_counts,
                                          float *d_pos, uint32_t *d_status, void *d_scratch,
                                          const mc_tuning *t, void *stream) {
  if (!b || !d_tri_counts || n_views == 0 || n_views > 8) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0)
    return from_cuda(
        cudaMemsetAsync(d_tri_counts, 0, 4ull * n_views, static_cast<cudaStream_t>(stream)));
  mc_status st =
      check_cull_views(b, d_view_projs, n_views, d_tri_out, tri_stride, d_tri_counts, d_pos, d_scratch);
  if (st != MC_OK) return st;
  return launch_cull_views_checked(b, d_view_projs, n_views, d_tri_out, tri_stride, d_tri_counts,
                                   d_pos, d_status, d_scratch, t, static_cast<cudaStream_t>(stream));
}

extern "C" size_t mc_cull_order_bytes(const mc_device_batch *b) {
  return b ? 8ull * b->n_meshlets + 16 : 0;
}

extern "C" mc_status mc_decode_cull_ordered(const mc_device_batch *b, const float *d_view_proj,
                                            uint32_t *d_tri_out, uint32_t *d_tri_count,
                                            float *d_pos, uint32_t *d_status, void *d_scratch,
                                            void *d_order, const mc_tuning *t, void *stream) {
  if (!b || !d_tri_count) return MC_ERR_INVALID_ARG;
  if (b->n_meshlets == 0)
    return from_cuda(cudaMemsetAsync(d_tri_count, 0, 4, static_cast<cudaStream_t>(stream)));
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_view_proj || !d_tri_out || !d_pos || !d_scratch || !aligned(d_scratch, 16) || !d_order ||
      !aligned(d_order, 8))
    return MC_ERR_INVALID_ARG;
  return launch_cull_checked(b, d_view_proj, d_tri_out, d_tri_count, d_pos, d_status, d_scratch, t,
                             static_cast<cudaStream_t>(stream), static_cast<uint64_t *>(d_order));
}

extern "C" mc_status mc_decode_requests(const mc_device_batch *pool, const mc_request *d_reqs,
                                        uint32_t n_reqs, uint32_t total_work, uint32_t *d_status,
                                        void *d_scratch, const mc_tuning *t, void *stream) {
  if (!pool) return MC_ERR_INVALID_ARG;
  if (n_reqs == 0 || total_work == 0) return MC_OK;
  mc_status st = check_batch(pool);
  if (st != MC_OK) return st;
  if (!d_reqs || !aligned(d_reqs, 16) || !d_scratch || !aligned(d_scratch, 16) ||
      total_work > (1u << 31))
    return MC_ERR_INVALID_ARG;
  const uint32_t warps = (t && t->warps_per_cta) ? t->warps_per_cta : 8;
  const uint32_t per_grab = (t && t->meshlets_per_grab) ? t->meshlets_per_grab : 2;
  if (warps > 32 || per_grab > 64) return MC_ERR_INVALID_ARG;
  int occ = max_ctas_per_sm_requests(warps, pool->max_block_words);
  if (occ <= 0) return MC_ERR_INVALID_ARG;
  uint32_t per_sm = (t && t->ctas_per_sm) ? std::min<uint32_t>(t->ctas_per_sm, occ) : (uint32_t)occ;
  // small request batches do not need the whole GPU
  uint32_t ctas = std::min<uint32_t>(per_sm * (uint32_t)sm_count(),
                                     std::max<uint32_t>(1u, (total_work + warps * per_grab - 1) / (warps * per_grab)));
  cudaError_t e = launch_requests(args_of(pool), d_reqs, n_reqs, total_work, ctas, warps, per_grab,
                                  t && t->checked, d_status, static_cast<uint32_t *>(d_scratch),
                                  static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) g_launches++;
  return from_cuda(e);
}

extern "C" mc_status mc_autotune(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                                 float *d_pos, uint32_t *d_status, void *d_scratch, void *stream,
                                 mc_tuning *best, float *best_ms) {
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_pos || !d_scratch) return MC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MC_ERR_CUDA;
  mc_tuning bt{};
  float bms = 1e30f;
  const uint32_t warps_c[] = {4, 8, 16};
  const uint32_t grab_c[] = {1, 2, 4, 8, 16};
  const uint32_t lanes_c[] = {32, 16};
  st = MC_OK;
  for (uint32_t lanes : lanes_c)
  for (uint32_t w : warps_c) {
    for (uint32_t g : grab_c) {
      if (lanes == 16 && g < 2) continue;
      int occ = lanes == 16 ? max_ctas_per_sm_batch_pairs(w, b->max_block_words, g)
                            : max_ctas_per_sm_batch(w, b->max_block_words, g);
      if (occ <= 0) continue;
      for (uint32_t frac = 0; frac < 2; frac++) {
        mc_tuning c{};
        c.warps_per_cta = w;
        c.meshlets_per_grab = g;
        c.lanes_per_meshlet = lanes;
        c.ctas_per_sm = frac == 0 ? (uint32_t)occ : std::max(1u, (uint32_t)occ / 2);
        if (frac == 1 && c.ctas_per_sm == (uint32_t)occ) continue;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 4 && st == MC_OK; rep++) {
          // rewriting the positions evicts the compressed input from L2, as
          // between frames; the first run of a shape also does its one-time
          // launch set-up and is not counted
          if (cudaMemsetAsync(d_pos, 0, 12ull * b->total_verts, s) != cudaSuccess) st = MC_ERR_CUDA;
          cudaEventRecord(e0, s);
          st = launch_batch_checked(b, d_local, d_global, d_pos, d_status, d_scratch, c, s);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) st = MC_ERR_CUDA;
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        if (st != MC_OK) break;
        if (ms_min < bms) {
          bms = ms_min;
          bt = c;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MC_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key_of(b)] = bt;
  }
  if (best) *best = bt;
  if (best_ms) *best_ms = bms;
  return MC_OK;
}

struct mc_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;
};

namespace {
template <class F>
mc_status capture(F &&body, mc_graph **out) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MC_ERR_CUDA;
  mc_graph *g = new mc_graph();
  mc_status st = MC_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = MC_ERR_CUDA;
  uint64_t before = g_launches.load();
  if (st == MC_OK) st = body(cs);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (st == MC_OK && e != cudaSuccess) st = MC_ERR_CUDA;
  if (st == MC_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = MC_ERR_CUDA;
  g->graph = graph;
  g->launches = g_launches.load() - before;
  g_launches.store(before);  // captured, not yet launched
  cudaStreamDestroy(cs);
  if (st != MC_OK) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st;
  }
  *out = g;
  return MC_OK;
}
}  // namespace

extern "C" mc_status mc_graph_capture_batch(const mc_device_batch *b, uint8_t *d_local,
                                            uint32_t *d_global, float *d_pos, uint32_t *d_status,
                                            void *d_scratch, const mc_tuning *t, void *stream,
                                            mc_graph **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_pos || !d_scratch || b->n_meshlets == 0) return MC_ERR_INVALID_ARG;
  (void)stream;
  mc_tuning r = resolve_batch(b, t);  // resolved before capture (no device queries inside)
  return capture(
      [&](cudaStream_t cs) {
        return launch_batch_checked(b, d_local, d_global, d_pos, d_status, d_scratch, r, cs);
      },
      out);
}

extern "C" mc_status mc_graph_capture_cull(const mc_device_batch *b, const float *d_view_projs,
                                           uint32_t n_views, uint32_t *d_tri_out,
                                           uint32_t *d_tri_count, float *d_pos, uint32_t *d_status,
                                           void *d_scratch, const mc_tuning *t, void *stream,
                                           mc_graph **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  mc_status st = check_batch(b);
  if (st != MC_OK) return st;
  if (!d_view_projs || n_views == 0 || !d_tri_out || !d_tri_count || !d_pos || !d_scratch ||
      b->n_meshlets == 0)
    return MC_ERR_INVALID_ARG;
  (void)stream;
  return capture(
      [&](cudaStream_t cs) {
        for (uint32_t i = 0; i < n_views; i++) {
          mc_status s2 = launch_cull_checked(b, d_view_projs + 16 * (size_t)i, d_tri_out,
                                             d_tri_count + i, d_pos, d_status, d_scratch, t, cs);
          if (s2 != MC_OK) return s2;
        }
        return MC_OK;
      },
      out);
}

extern "C" mc_status mc_graph_capture_cull_views(const mc_device_batch *b,
                                                 const float *d_view_projs, uint32_t n_views,
                                                 uint32_t *d_tri_out, uint64_t tri_stride,
                                                 uint32_t *d_tri_counts, float *d_pos,
                                                 uint32_t *d_status, void *d_scratch,
                                                 const mc_tuning *t, void *stream, mc_graph **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!b || b->n_meshlets == 0) return MC_ERR_INVALID_ARG;
  mc_status st =
      check_cull_views(b, d_view_projs, n_views, d_tri_out, tri_stride, d_tri_counts, d_pos, d_scratch);
  if (st != MC_OK) return st;
  (void)stream;
  return capture(
      [&](cudaStream_t cs) {
        for (uint32_t v0 = 0; v0 < n_views; v0 += 8) {
          mc_status s2 = launch_cull_views_checked(b, d_view_projs + 16 * (size_t)v0,
                                                   std::min(8u, n_views - v0), d_tri_out, tri_stride,
                                                   d_tri_counts + v0, d_pos, d_status, d_scratch, t,
                                                   cs);
          if (s2 != MC_OK) return s2;
        }
        return MC_OK;
      },
      out);
}

extern "C" mc_status mc_graph_launch(mc_graph *g, void *stream) {
  if (!g || !g->exec) return MC_ERR_INVALID_ARG;
  cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) g_launches += g->launches;
  return from_cuda(e);
}

extern "C" void mc_graph_free(mc_graph *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

namespace {
// Internal streams of the host-buffer decode (input copies, decode, output
// copies) and their events, created once per device.
constexpr uint32_t kHostChunks = 8;
struct HostPipe {
  std::mutex mu;  // one call enqueues at a time (the events are shared)
  cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
  cudaEvent_t ev[2 * kHostChunks + 3] = {};
  bool ok = false;
};
std::mutex g_pipe_mu;
std::map<int, HostPipe> g_pipes;

HostPipe *host_pipe() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe &p = g_pipes[dev];
  if (!p.ok) {
    bool ok = cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &e : p.ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return nullptr;
    p.ok = true;
  }
  return &p;
}
}  // namespace

extern "C" mc_status mc_decode_batch_host(const mc_blob_view_t *v, mc_desc *d_desc,
                                          uint8_t *d_payload, mc_grid *d_grids, uint8_t *d_local,
                                          uint32_t *d_global, float *d_pos, uint32_t *d_status,
                                          void *d_scratch, uint8_t *h_local, uint32_t *h_global,
                                          float *h_pos, const mc_tuning *t, void *stream) {
  if (!v || !d_desc || !d_payload || !d_grids || !d_pos) return MC_ERR_INVALID_ARG;
  if ((h_local && !d_local) || (h_global && !d_global)) return MC_ERR_INVALID_ARG;
  const uint32_t n = v->n_meshlets;
  if (n == 0) return MC_OK;
  if (!v->desc || !v->payload || !v->grids) return MC_ERR_INVALID_ARG;
  mc_device_batch b{};
  b.desc = d_desc;
  b.payload = d_payload;
  b.grids = d_grids;
  b.n_meshlets = n;
  b.n_grids = v->n_grids;
  b.payload_bytes = v->payload_bytes;
  b.total_tris = v->total_tris;
  b.total_verts = v->total_verts;
  b.max_block_words = v->max_block_words;
  b.max_tris = v->max_tris;
  b.max_verts = v->max_verts;
  mc_status st = check_batch(&b);
  if (st != MC_OK) return st;
  if (!d_scratch || !aligned(d_scratch, 16) || !aligned(d_local, 16) || !aligned(d_global, 16))
    return MC_ERR_INVALID_ARG;
  // chunk boundaries (consecutive meshlets); their payload, triangle and
  // vertex ranges come from the host descriptors, which must be monotonic
  const uint32_t K = std::max<uint32_t>(1u, std::min<uint32_t>(kHostChunks, (n + 8191) / 8192));
  uint32_t cut[kHostChunks + 1];
  uint64_t pay[kHostChunks + 1], tri[kHostChunks + 1], vtx[kHostChunks + 1];
  for (uint32_t i = 0; i <= K; i++) {
    cut[i] = (uint32_t)((uint64_t)n * i / K);
    const bool end = cut[i] == n;
    pay[i] = end ? v->payload_bytes : 16ull * v->desc[cut[i]].payload_off16;
    tri[i] = end ? v->total_tris : v->desc[cut[i]].tri_base;
    vtx[i] = end ? v->total_verts : v->desc[cut[i]].vertex_base;
    if (i > 0 && (pay[i] < pay[i - 1] || tri[i] < tri[i - 1] || vtx[i] < vtx[i - 1]))
      return MC_ERR_CORRUPT;
  }
  if (pay[0] != 0 || tri[0] != 0 || vtx[0] != 0 || pay[K] > v->payload_bytes) return MC_ERR_CORRUPT;
  HostPipe *P = host_pipe();
  if (!P) return MC_ERR_CUDA;
  const mc_tuning r = resolve_batch(&b, t);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(P->mu);
  // chunk i: input copies on P->in, decode on P->comp, output copies on
  // P->out, so chunk i's decode overlaps chunk i+1's input and chunk i-1's
  // output copies; the caller's stream orders the whole call
  cudaEvent_t *ev = P->ev;
  cudaError_t e = cudaEventRecord(ev[0], s);
  for (cudaStream_t q : {P->in, P->comp, P->out})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q, ev[0], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_grids, v->grids, sizeof(mc_grid) * (size_t)v->n_grids,
                        cudaMemcpyHostToDevice, P->in);
  for (uint32_t i = 0; i < K && e == cudaSuccess && st == MC_OK; i++) {
    const uint32_t m_a = cut[i], m_b = cut[i + 1];
    e = cudaMemcpyAsync(d_desc + m_a, v->desc + m_a, sizeof(mc_desc) * (size_t)(m_b - m_a),
                        cudaMemcpyHostToDevice, P->in);
    if (e == cudaSuccess && pay[i + 1] > pay[i])
      e = cudaMemcpyAsync(d_payload + pay[i], v->payload + pay[i], pay[i + 1] - pay[i],
                          cudaMemcpyHostToDevice, P->in);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + i], P->in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->comp, ev[1 + i], 0);
    if (e != cudaSuccess) break;
    mc_device_batch c = b;
    c.desc = d_desc + m_a;
    c.n_meshlets = m_b - m_a;
    c.payload_bytes = pay[i + 1];  // the chunk's blocks end there
    st = launch_batch_checked(&c, d_local, d_global, d_pos, d_status, d_scratch, r, P->comp);
    if (st != MC_OK) break;
    e = cudaEventRecord(ev[1 + kHostChunks + i], P->comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->out, ev[1 + kHostChunks + i], 0);
    if (e == cudaSuccess && h_local)
      e = cudaMemcpyAsync(h_local + 3 * tri[i], d_local + 3 * tri[i], 3 * (tri[i + 1] - tri[i]),
                          cudaMemcpyDeviceToHost, P->out);
    if (e == cudaSuccess && h_global)
      e = cudaMemcpyAsync(h_global + 3 * tri[i], d_global + 3 * tri[i], 12 * (tri[i + 1] - tri[i]),
                          cudaMemcpyDeviceToHost, P->out);
    if (e == cudaSuccess && h_pos)
      e = cudaMemcpyAsync(h_pos + 3 * vtx[i], d_pos + 3 * vtx[i], 12 * (vtx[i + 1] - vtx[i]),
                          cudaMemcpyDeviceToHost, P->out);
  }
  // join the internal streams back into the caller's stream (also on error,
  // so that nothing of this call is left unordered)
  cudaError_t j = cudaEventRecord(ev[2 * kHostChunks + 1], P->comp);
  if (j == cudaSuccess) j = cudaStreamWaitEvent(s, ev[2 * kHostChunks + 1], 0);
  if (j == cudaSuccess) j = cudaEventRecord(ev[2 * kHostChunks + 2], P->out);
  if (j == cudaSuccess) j = cudaStreamWaitEvent(s, ev[2 * kHostChunks + 2], 0);
  cudaEventRecord(ev[0], P->in);
  cudaStreamWaitEvent(s, ev[0], 0);
  if (st != MC_OK) return st;
  if (e == cudaSuccess) e = j;
  return from_cuda(e);
}
