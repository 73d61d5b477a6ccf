// Decode kernels for sm_103a: plain (one warp per meshlet, grid over a
// meshlet range), batched (persistent CTAs pulling meshlets from a device work
// queue) and the serving form over request lists; the launch set-up the
// kernel files share.  The fused cull kernels are in cull.cu.
#include <cuda_runtime.h>

#include "decode_warp.cuh"
#include "grab_loop.cuh"
#include "kernels.h"

namespace mcdev {

// Per-warp shared memory of the single-meshlet kernels: payload words (plus
// over-read slack), then the strip stream.
__host__ __device__ inline uint32_t warp_words(uint32_t max_block_words) {
  return ((max_block_words + 3) & ~3u) + kSlackWords;
}
__host__ __device__ inline uint32_t warp_smem_bytes(uint32_t max_block_words) {
  return 4 * warp_words(max_block_words) + kStreamBytes;
}
uint32_t decode_smem_per_warp(uint32_t max_block_words) { return warp_smem_bytes(max_block_words); }
// Batched kernel: the grab loop's buffers, a 64-byte attribute slot, then the
// strip stream.
uint32_t batch_smem_per_warp(uint32_t max_block_words, uint32_t per_grab) {
  return grab_loop_bytes(max_block_words, per_grab) + 64 + kStreamBytes;
}

template <bool CHECKED>
__device__ __forceinline__ void decode_one(const BatchArgs &a, uint32_t m, uint32_t *sw,
                                           uint8_t *sI, uint32_t lane, uint8_t *out_local,
                                           uint32_t *out_global, float *out_pos,
                                           uint32_t *status) {
  const Desc d = with_attrs(load_desc(a.desc + m), a);
  if (!header_ok(d, a)) {
    if (lane == 0) set_status(status, MC_ERR_CORRUPT);
    return;
  }
  const Grid g = load_grid(a.grids + d.grid);
  stage_payload(d, a.payload, sw, lane);
  __syncwarp();
  if (!decode_dispatch<CHECKED>(d, g, sw, sI, lane, out_local, out_global, out_pos) && lane == 0)
    set_status(status, MC_ERR_CORRUPT);
  __syncwarp();
}

template <bool CHECKED>
__global__ void decode_plain_kernel(BatchArgs a, uint32_t first, uint32_t count,
                                    uint32_t smem_per_warp, uint8_t *out_local,
                                    uint32_t *out_global, float *out_pos, uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint8_t *base = smem + warp * smem_per_warp;
  uint32_t *sw = reinterpret_cast<uint32_t *>(base);
  uint8_t *sI = base + smem_per_warp - kStreamBytes;
  const uint32_t i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= count) return;
  decode_one<CHECKED>(a, first + i, sw, sI, lane, out_local, out_global, out_pos, status);
}

// Persistent batched decode: each warp runs the grab loop and decodes the
// staged meshlets one after another from shared memory.  VTX: out_pos
// receives full 8-float vertices (positions + attribute channels); the
// meshlet's attribute minima and grid are first copied into the warp's
// 64-byte slot in front of the strip stream.
template <bool CHECKED, bool VTX>
__global__ void __launch_bounds__(512) decode_batch_kernel(BatchArgs a, uint32_t per_grab,
                                                           uint32_t smem_per_warp, uint8_t *out_local,
                                                           uint32_t *out_global, float *out_pos,
                                                           uint32_t *status, uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint8_t *base = smem + warp * smem_per_warp;
  uint8_t *sI = base + smem_per_warp - kStreamBytes;
  uint32_t *sa = reinterpret_cast<uint32_t *>(sI - 64);
  grab_loop<2>(a, per_grab, base, lane, scratch + kQueue, status, NoPre{},
            [&](const Desc &d, const uint32_t *sw, uint32_t, uint32_t, uint32_t m) {
              const Grid g = load_grid(a.grids + d.grid);
              if (VTX) {
                bool ok = true;
                if (lane < a.n_attr) {
                  const mc_attr_desc *ad = a.attr_desc + m;
                  const uint32_t gi = __ldg(&ad->grid);
                  ok = gi < a.n_attr_grids;
                  if (ok) {
                    const mc_attr_grid *ag = a.attr_grids + gi;
                    ok = __ldg(&ag->attr_bits) == a.attr_bits;
                    sa[lane] = __ldg(&ad->La[lane]);
                    ok = ok & (sa[lane] <= ~field_max(a.attr_bits));  // La + 2^b - 1 fits 32 bits
                    sa[5 + lane] = __float_as_uint(__ldg(&ag->G[lane]));
                    sa[10 + lane] = __float_as_uint(__ldg(&ag->delta[lane]));
                  }
                }
                if (!__all_sync(kFull, ok)) {
                  if (lane == 0) set_status(status, MC_ERR_CORRUPT);
                  return;
                }
                __syncwarp();
              }
              if (!decode_dispatch<CHECKED, VTX>(d, g, sw, sI, lane, out_local, out_global, out_pos,
                                                 sa, a.n_attr, a.attr_bits) &&
                  lane == 0)
                set_status(status, MC_ERR_CORRUPT);
            });
  // the last CTA to finish leaves the queue reset for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      atomicExch(scratch + kQueue, 0u);
      atomicExch(scratch + kDone, 0u);
    }
  }
}

// Persistent batched decode with two meshlets per warp (16 lanes each):
// the grab loop hands the meshlets of each grab out in pairs and both halves
// decode at once (decode_pair), so the per-meshlet set-up (descriptor,
// header check, grid, output pointers) is paid once per pair.  Per warp:
// the grab loop's buffers, then one strip-stream buffer per half.
uint32_t batch_pairs_smem_per_warp(uint32_t max_block_words, uint32_t per_grab) {
  return grab_loop_bytes(max_block_words, per_grab) + 2 * kStreamBytes;
}

template <bool CHECKED>
__global__ void __launch_bounds__(512) decode_batch_pairs_kernel(BatchArgs a, uint32_t per_grab,
                                                                 uint32_t smem_per_warp,
                                                                 uint8_t *out_local,
                                                                 uint32_t *out_global,
                                                                 float *out_pos, uint32_t *status,
                                                                 uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint8_t *base = smem + warp * smem_per_warp;
  uint8_t *sI = base + smem_per_warp - (2 - (lane >> 4)) * kStreamBytes;  // this half's stream
  grab_loop_pairs(a, per_grab, base, lane, scratch + kQueue, status,
                  [&](const Desc &d, bool live, const uint32_t *sw, uint32_t) {
                    const Grid g = load_grid(a.grids + d.grid);
                    if (!decode_pair_dispatch<CHECKED>(d, live, g, sw, sI, lane, out_local,
                                                       out_global, out_pos) &&
                        (lane & 15u) == 0)
                      set_status(status, MC_ERR_CORRUPT);
                  });
  // the last CTA to finish leaves the queue reset for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      atomicExch(scratch + kQueue, 0u);
      atomicExch(scratch + kDone, 0u);
    }
  }
}

// Continuous-batching decode: persistent warps take `per_grab` work items
// (meshlets of the concatenated request ranges); each item is mapped to its
// request by binary search over work_start, its descriptor is renumbered
// relative to the request's first meshlet, and it decodes into the request's
// buffers.
template <bool CHECKED>
__global__ void __launch_bounds__(512) decode_requests_kernel(BatchArgs a, const mc_request *reqs,
                                                              uint32_t n_reqs, uint32_t total_work,
                                                              uint32_t per_grab, uint32_t *status,
                                                              uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t spw = 4 * (((a.max_block_words + 3) & ~3u) + kSlackWords) + kStreamBytes;
  uint8_t *base = smem + warp * spw;
  uint32_t *sw = reinterpret_cast<uint32_t *>(base);
  uint8_t *sI = base + spw - kStreamBytes;
  for (;;) {
    uint32_t w0 = 0;
    if (lane == 0) w0 = atomicAdd(scratch + kQueue, per_grab);
    w0 = __shfl_sync(kFull, w0, 0);
    if (w0 >= total_work) break;
    const uint32_t w1 = min(total_work, w0 + per_grab);
    // request holding w0: the last with work_start <= w0
    uint32_t lo = 0, hi = n_reqs;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&reqs[mid].work_start) <= w0) lo = mid; else hi = mid;
    }
    uint32_t r = lo;
    for (uint32_t w = w0; w < w1; w++) {
      while (r + 1 < n_reqs && __ldg(&reqs[r + 1].work_start) <= w) r++;
      const mc_request *q = reqs + r;
      const uint32_t item = w - __ldg(&q->work_start);
      if (item >= __ldg(&q->n_meshlets)) {  // work past a request's range: malformed table
        if (lane == 0) set_status(status, MC_ERR_INVALID_ARG);
        continue;
      }
      const uint32_t m = __ldg(&q->first_meshlet) + item;
      if (m >= a.n_meshlets) {
        if (lane == 0) set_status(status, MC_ERR_INVALID_ARG);
        continue;
      }
      Desc d = with_attrs(load_desc(a.desc + m), a);
      d.tbase -= __ldg(&q->tri_base);
      d.vbase -= __ldg(&q->vertex_base);
      BatchArgs ra = a;
      ra.total_tris = __ldg(&q->tri_count);
      ra.total_verts = __ldg(&q->vert_count);
      if (!header_ok(d, ra)) {
        if (lane == 0) set_status(status, MC_ERR_CORRUPT);
        continue;
      }
      uint8_t *ol = reinterpret_cast<uint8_t *>(__ldg(reinterpret_cast<const unsigned long long *>(&q->d_local)));
      uint32_t *og = reinterpret_cast<uint32_t *>(__ldg(reinterpret_cast<const unsigned long long *>(&q->d_global)));
      float *op = reinterpret_cast<float *>(__ldg(reinterpret_cast<const unsigned long long *>(&q->d_pos)));
      if (!op) {
        if (lane == 0) set_status(status, MC_ERR_INVALID_ARG);
        continue;
      }
      const Grid g = load_grid(a.grids + d.grid);
      stage_payload(d, a.payload, sw, lane);
      __syncwarp();
      if (!decode_dispatch<CHECKED>(d, g, sw, sI, lane, ol, og, op) && lane == 0)
        set_status(status, MC_ERR_CORRUPT);
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      atomicExch(scratch + kQueue, 0u);
      atomicExch(scratch + kDone, 0u);
    }
  }
}

// ------------------------------------------------------------- launchers
}  // namespace mcdev

#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>

namespace mcdev {
namespace {
constexpr int kMaxSmem = 227 * 1024;  // opt-in shared memory per CTA on sm_103a

// Per-device, per-kernel launch set-up done once: the dynamic shared-memory
// limit is raised to the maximum on first use (it only permits larger
// launches), and occupancy answers are cached, so a launch costs no driver
// calls beyond the launch itself.
std::mutex g_attr_mu;
std::set<std::pair<int, const void *>> g_attr_done;
std::map<std::tuple<int, const void *, int, int>, int> g_occ;

int device_now() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
}  // namespace

void prepare(const void *f) {
  const int dev = device_now();
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (!g_attr_done.insert({dev, f}).second) return;
  // dynamic limit = the device's opt-in maximum minus the kernel's static
  // shared memory
  int optin = 0;
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      cudaFuncGetAttributes(&fa, f) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin - (int)fa.sharedSizeBytes);
  (void)cudaGetLastError();  // a refused attribute shows up as a launch error instead
}
int occupancy(const void *f, int threads, int smem) {
  if (smem > kMaxSmem - 64) return 0;  // leave room for the kernels' static shared memory
  prepare(f);
  const auto key = std::make_tuple(device_now(), f, threads, smem);
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) n = 0;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  g_occ[key] = n;
  return n;
}

cudaError_t launch_plain(const BatchArgs &a, uint32_t first, uint32_t count, uint32_t warps,
                         uint32_t max_block_words, bool checked, uint8_t *out_local,
                         uint32_t *out_global, float *out_pos, uint32_t *status,
                         cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t spw = warp_smem_bytes(max_block_words);
  const uint32_t smem = spw * warps;
  const uint32_t grid = (count + warps - 1) / warps;
  if (checked) {
    prepare(fn(decode_plain_kernel<true>));
    decode_plain_kernel<true><<<grid, warps * 32, smem, s>>>(a, first, count, spw, out_local,
                                                             out_global, out_pos, status);
  } else {
    prepare(fn(decode_plain_kernel<false>));
    decode_plain_kernel<false><<<grid, warps * 32, smem, s>>>(a, first, count, spw, out_local,
                                                              out_global, out_pos, status);
  }
  return cudaGetLastError();
}

namespace {
template <bool CHECKED, bool VTX>
cudaError_t launch_batch_t(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                           uint32_t spw, uint8_t *out_local, uint32_t *out_global, float *out_pos,
                           uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  prepare(fn(decode_batch_kernel<CHECKED, VTX>));
  decode_batch_kernel<CHECKED, VTX><<<ctas, warps * 32, spw * warps, s>>>(
      a, per_grab, spw, out_local, out_global, out_pos, status, scratch);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_batch_pairs(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                               uint32_t max_block_words, bool checked, uint8_t *out_local,
                               uint32_t *out_global, float *out_pos, uint32_t *status,
                               uint32_t *scratch, cudaStream_t s) {
  const uint32_t spw = batch_pairs_smem_per_warp(max_block_words, per_grab);
  if (checked) {
    prepare(fn(decode_batch_pairs_kernel<true>));
    decode_batch_pairs_kernel<true><<<ctas, warps * 32, spw * warps, s>>>(
        a, per_grab, spw, out_local, out_global, out_pos, status, scratch);
  } else {
    prepare(fn(decode_batch_pairs_kernel<false>));
    decode_batch_pairs_kernel<false><<<ctas, warps * 32, spw * warps, s>>>(
        a, per_grab, spw, out_local, out_global, out_pos, status, scratch);
  }
  return cudaGetLastError();
}

int max_ctas_per_sm_batch_pairs(uint32_t warps, uint32_t max_block_words, uint32_t per_grab) {
  const int smem = (int)(batch_pairs_smem_per_warp(max_block_words, per_grab) * warps);
  prepare(fn(decode_batch_pairs_kernel<true>));
  return occupancy(fn(decode_batch_pairs_kernel<false>), warps * 32, smem);
}

cudaError_t launch_batch(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                         uint32_t max_block_words, bool checked, bool vertices,
                         uint8_t *out_local, uint32_t *out_global, float *out_pos,
                         uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  const uint32_t spw = batch_smem_per_warp(max_block_words, per_grab);
  if (vertices)
    return checked ? launch_batch_t<true, true>(a, ctas, warps, per_grab, spw, out_local, out_global,
                                                out_pos, status, scratch, s)
                   : launch_batch_t<false, true>(a, ctas, warps, per_grab, spw, out_local,
                                                 out_global, out_pos, status, scratch, s);
  return checked ? launch_batch_t<true, false>(a, ctas, warps, per_grab, spw, out_local, out_global,
                                               out_pos, status, scratch, s)
                 : launch_batch_t<false, false>(a, ctas, warps, per_grab, spw, out_local, out_global,
                                                out_pos, status, scratch, s);
}

cudaError_t launch_requests(const BatchArgs &a, const mc_request *reqs, uint32_t n_reqs,
                            uint32_t total_work, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                            bool checked, uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  const uint32_t spw = 4 * (((a.max_block_words + 3) & ~3u) + kSlackWords) + kStreamBytes;
  const uint32_t smem = spw * warps;
  if (checked) {
    prepare(fn(decode_requests_kernel<true>));
    decode_requests_kernel<true><<<ctas, warps * 32, smem, s>>>(a, reqs, n_reqs, total_work, per_grab,
                                                                status, scratch);
  } else {
    prepare(fn(decode_requests_kernel<false>));
    decode_requests_kernel<false><<<ctas, warps * 32, smem, s>>>(a, reqs, n_reqs, total_work, per_grab,
                                                                 status, scratch);
  }
  return cudaGetLastError();
}

// Occupancy of the unchecked builds (the checked ones use the same shared
// memory; their register counts are within the same 64-per-thread class).
int max_ctas_per_sm_requests(uint32_t warps, uint32_t max_block_words) {
  const int smem = (int)((4 * (((max_block_words + 3) & ~3u) + kSlackWords) + kStreamBytes) * warps);
  prepare(fn(decode_requests_kernel<true>));
  return occupancy(fn(decode_requests_kernel<false>), warps * 32, smem);
}

int max_ctas_per_sm_batch(uint32_t warps, uint32_t max_block_words, uint32_t per_grab,
                          bool vertices) {
  const int smem = (int)(batch_smem_per_warp(max_block_words, per_grab) * warps);
  if (vertices) {
    prepare(fn(decode_batch_kernel<true, true>));
    return occupancy(fn(decode_batch_kernel<false, true>), warps * 32, smem);
  }
  prepare(fn(decode_batch_kernel<true, false>));
  return occupancy(fn(decode_batch_kernel<false, false>), warps * 32, smem);
}

}  // namespace mcdev
