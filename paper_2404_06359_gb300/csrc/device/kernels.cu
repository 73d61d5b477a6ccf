// Decode kernels for sm_103a: plain (one warp per meshlet, grid over a
// meshlet range), batched (persistent CTAs pulling meshlets from a device work
// queue) and fused decode + cull + compaction.
#include <cuda_runtime.h>

#include "decode_warp.cuh"
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
// Batched kernel: descriptors of one grab, the grab's payload blocks, stream.
__host__ __device__ inline uint32_t grab_words(uint32_t max_block_words, uint32_t per_grab) {
  return 8 * per_grab + per_grab * ((max_block_words + 3) & ~3u) + kSlackWords;
}
uint32_t decode_smem_per_warp(uint32_t max_block_words) { return warp_smem_bytes(max_block_words); }
uint32_t batch_smem_per_warp(uint32_t max_block_words, uint32_t per_grab) {
  return 4 * grab_words(max_block_words, per_grab) + kStreamBytes;
}

template <bool CHECKED>
__device__ __forceinline__ void decode_one(const BatchArgs &a, uint32_t m, uint32_t *sw,
                                           uint8_t *sI, uint32_t lane, uint8_t *out_local,
                                           uint32_t *out_global, float *out_pos,
                                           uint32_t *status) {
  const Desc d = load_desc(a.desc + m);
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

// Scratch words used by the persistent kernels.
enum { kQueue = 0, kDone = 1, kCount = 2 };

// Persistent batched decode.  Each warp takes `per_grab` (<= 16) consecutive
// meshlets from the work queue; because consecutive meshlets have
// consecutive payload blocks, the warp loads all their descriptors and the
// whole payload range in one pass of 16-byte loads (one memory latency per
// grab), then decodes them one after another from shared memory.  A grab
// whose range does not look contiguous falls back to staging meshlet by
// meshlet.
template <bool CHECKED>
__global__ void __launch_bounds__(512) decode_batch_kernel(BatchArgs a, uint32_t per_grab,
                                                           uint32_t smem_per_warp, uint8_t *out_local,
                                                           uint32_t *out_global, float *out_pos,
                                                           uint32_t *status, uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint8_t *base = smem + warp * smem_per_warp;
  uint32_t *sdesc = reinterpret_cast<uint32_t *>(base);
  uint32_t *spay = sdesc + 8 * per_grab;
  uint8_t *sI = base + smem_per_warp - kStreamBytes;
  const uint32_t cap16 = (per_grab * ((a.max_block_words + 3) & ~3u)) / 4;
  const uint32_t bytes16 = a.payload_bytes / 16 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)(a.payload_bytes / 16);
  const uint4 *gdesc = reinterpret_cast<const uint4 *>(a.desc);
  const uint4 *gpay = reinterpret_cast<const uint4 *>(a.payload);
  for (;;) {
    uint32_t m0 = 0;
    if (lane == 0) m0 = atomicAdd(scratch + kQueue, per_grab);
    m0 = __shfl_sync(kFull, m0, 0);
    if (m0 >= a.n_meshlets) break;
    const uint32_t cnt = min(per_grab, a.n_meshlets - m0);
    uint4 dv = make_uint4(0, 0, 0, 0);
    if (lane < 2 * cnt) dv = __ldg(gdesc + 2ull * m0 + lane);
    uint32_t end16 = bytes16;
    if (m0 + cnt < a.n_meshlets) end16 = __ldg(&a.desc[m0 + cnt].payload_off16);
    if (lane < 2 * cnt) reinterpret_cast<uint4 *>(sdesc)[lane] = dv;
    const uint32_t start16 = __shfl_sync(kFull, dv.x, 0);
    bool grab_staged = end16 >= start16 && end16 - start16 <= cap16 && end16 <= bytes16;
    if (grab_staged) {
      uint4 *dst = reinterpret_cast<uint4 *>(spay);
      for (uint32_t i = lane; i < end16 - start16; i += 32) dst[i] = __ldg(gpay + start16 + i);
    }
    __syncwarp();
    for (uint32_t j = 0; j < cnt; j++) {
      const uint4 *sd = reinterpret_cast<const uint4 *>(sdesc) + 2 * j;
      const Desc d = unpack_desc(sd[0], sd[1]);
      if (!header_ok(d, a)) {
        if (lane == 0) set_status(status, MC_ERR_CORRUPT);
        continue;
      }
      const uint32_t padded16 = ((block_words(d) + 3) & ~3u) / 4;
      const uint32_t *sw;
      if (grab_staged && d.off16 >= start16 && d.off16 - start16 + padded16 <= end16 - start16) {
        sw = spay + 4 * (d.off16 - start16);
      } else {
        grab_staged = false;  // spay is reused meshlet by meshlet from here on
        __syncwarp();
        stage_payload(d, a.payload, spay, lane);
        __syncwarp();
        sw = spay;
      }
      const Grid g = load_grid(a.grids + d.grid);
      if (!decode_dispatch<CHECKED>(d, g, sw, sI, lane, out_local, out_global, out_pos) && lane == 0)
        set_status(status, MC_ERR_CORRUPT);
    }
    __syncwarp();
  }
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
      Desc d = load_desc(a.desc + m);
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

// ---------------------------------------------------------------- culling
__device__ __forceinline__ float clip_row(const float *M, int r, float x, float y, float z) {
  return __fmaf_rn(M[4 * r + 2], z, __fmaf_rn(M[4 * r + 1], y, __fmaf_rn(M[4 * r + 0], x, M[4 * r + 3])));
}

// true when all 8 corners of the meshlet's quantisation box are outside one
// clip plane.  Lanes 0..7 each take one corner and collect the planes it is
// outside of; the warp AND-reduces the plane masks.
__device__ __forceinline__ bool box_outside(const Desc &d, const Grid &g, const float *M,
                                            uint32_t lane) {
  uint32_t mask = 0x3Fu;
  if (lane < 8) {
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint32_t top = d.L[c] + (d.b >= 32 ? 0xFFFFFFFFu : ((1u << d.b) - 1u));
      p[c] = dequant((lane >> c) & 1u ? top : d.L[c], g.G[c], g.D[c]);
    }
    const float w = clip_row(M, 3, p[0], p[1], p[2]);
    mask = 0;
#pragma unroll
    for (int r = 0; r < 3; r++) {
      const float comp = clip_row(M, r, p[0], p[1], p[2]);
      if (__fadd_rn(w, comp) < 0.0f) mask |= 1u << (2 * r);
      if (__fsub_rn(w, comp) < 0.0f) mask |= 2u << (2 * r);
    }
  }
  return __reduce_and_sync(kFull, mask) != 0;
}

// Per-warp shared memory of the culling kernel (bytes, 16-byte aligned parts):
// descriptors of a grab, its payload blocks + slack, the strip stream, clip
// x / y / w per vertex, and the grab's surviving triangles.
struct CullLayout {
  uint32_t desc, pay, stream, clip, surv, bytes;
};
__host__ __device__ inline CullLayout cull_layout(uint32_t max_block_words, uint32_t max_tris,
                                                  uint32_t per_grab) {
  CullLayout l;
  l.desc = 0;
  l.pay = 32 * per_grab;
  l.stream = l.pay + 4 * (per_grab * ((max_block_words + 3) & ~3u) + kSlackWords);
  l.clip = l.stream + kStreamBytes;
  l.surv = l.clip + 3 * 4 * 256;
  l.bytes = l.surv + ((12 * per_grab * max_tris + 15) & ~15u);
  return l;
}
uint32_t cull_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t per_grab) {
  return cull_layout(max_block_words, max_tris, per_grab).bytes;
}

// Decode + cull of one staged meshlet; survivors (global index triples)
// are appended to surv[] from position n_keep.  Returns the new count, or
// 0xFFFFFFFF for a corrupt stream (checked build).
template <bool CHECKED, bool B16, bool W8>
__device__ __forceinline__ uint32_t cull_staged(const Desc &d, const Grid &g, const float *M,
                                                const uint32_t *sw, uint8_t *sI, float *cx,
                                                float *cy, float *cw, uint32_t *surv,
                                                uint32_t n_keep, uint32_t lane, float *out_pos) {
  if (CHECKED && !stream_header_ok(d, sw)) return 0xFFFFFFFFu;
  const uint32_t nw = (d.T + 31) >> 5;
  const uint32_t *pw = sw + 2 * nw + ((d.T + 2 - d.V) * d.w + 31) / 32;
  const bool small = small_coords(d);
  float *op = out_pos + 3ull * d.vbase;
  for (uint32_t v = lane; v < d.V; v += 32) {
    uint32_t q[3];
    vertex_q<B16>(pw, v, d.b, q);
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
      p[c] = small ? dequant_small(d.L[c] + q[c], g.G[c], g.D[c]) : dequant(d.L[c] + q[c], g.G[c], g.D[c]);
    op[3 * v] = p[0];
    op[3 * v + 1] = p[1];
    op[3 * v + 2] = p[2];
    cx[v] = clip_row(M, 0, p[0], p[1], p[2]);
    cy[v] = clip_row(M, 1, p[0], p[1], p[2]);
    cw[v] = clip_row(M, 3, p[0], p[1], p[2]);
  }
  __syncwarp();
  const uint32_t vb = d.vbase;
  const bool ok = walk_triangles<CHECKED, W8>(
      d, sw, sI, lane, [&](uint32_t k, uint32_t x, uint32_t y, uint32_t z, bool live) {
        bool keep = false;
        if (live && x != y && y != z && x != z) {
          const float w0 = cw[x], w1 = cw[y], w2 = cw[z];
          if (w0 <= 0.0f || w1 <= 0.0f || w2 <= 0.0f) {
            keep = true;
          } else {
            const float x0 = cx[x], y0 = cy[x], x1 = cx[y], y1 = cy[y];
            const float x2 = cx[z], y2 = cy[z];
            const float c0 = __fmaf_rn(y1, w2, -__fmul_rn(w1, y2));
            const float c1 = __fmaf_rn(x1, w2, -__fmul_rn(w1, x2));
            const float c2 = __fmaf_rn(x1, y2, -__fmul_rn(y1, x2));
            const float det = __fmaf_rn(w0, c2, __fmaf_rn(-y0, c1, __fmul_rn(x0, c0)));
            keep = det > 0.0f;
          }
        }
        const uint32_t bal = __ballot_sync(kFull, keep);
        if (keep) {
          const uint32_t o = n_keep + __popc(bal & ((1u << lane) - 1u));
          surv[3 * o] = vb + x;
          surv[3 * o + 1] = vb + y;
          surv[3 * o + 2] = vb + z;
        }
        n_keep += __popc(bal);
      });
  return ok ? n_keep : 0xFFFFFFFFu;
}

template <bool CHECKED>
__device__ __forceinline__ uint32_t cull_dispatch(const Desc &d, const Grid &g, const float *M,
                                                  const uint32_t *sw, uint8_t *sI, float *cx,
                                                  float *cy, float *cw, uint32_t *surv,
                                                  uint32_t n_keep, uint32_t lane, float *out_pos) {
  if (d.b == 16) {
    if (d.w == 8) return cull_staged<CHECKED, true, true>(d, g, M, sw, sI, cx, cy, cw, surv, n_keep, lane, out_pos);
    return cull_staged<CHECKED, true, false>(d, g, M, sw, sI, cx, cy, cw, surv, n_keep, lane, out_pos);
  }
  if (d.w == 8) return cull_staged<CHECKED, false, true>(d, g, M, sw, sI, cx, cy, cw, surv, n_keep, lane, out_pos);
  return cull_staged<CHECKED, false, false>(d, g, M, sw, sI, cx, cy, cw, surv, n_keep, lane, out_pos);
}

// Fused decode + cull + compaction.  Persistent warps take `per_grab`
// consecutive meshlets (staged like the batched decoder), drop meshlets whose
// box is outside the frustum before touching their triangles, decode and cull
// the rest, collect the grab's survivors in shared memory and reserve their
// output space with one atomicAdd per grab.
template <bool CHECKED>
__global__ void __launch_bounds__(512) decode_cull_kernel(BatchArgs a, const float *view_proj,
                                                          uint32_t per_grab, uint32_t *tri_out,
                                                          uint32_t *tri_count, float *out_pos,
                                                          uint32_t *status, uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float s_M[16];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const CullLayout L = cull_layout(a.max_block_words, a.max_tris, per_grab);
  uint8_t *base = smem + warp * L.bytes;
  uint32_t *sdesc = reinterpret_cast<uint32_t *>(base + L.desc);
  uint32_t *spay = reinterpret_cast<uint32_t *>(base + L.pay);
  uint8_t *sI = base + L.stream;
  float *cx = reinterpret_cast<float *>(base + L.clip);
  float *cy = cx + 256;
  float *cw = cy + 256;
  uint32_t *surv = reinterpret_cast<uint32_t *>(base + L.surv);
  if (threadIdx.x < 16) s_M[threadIdx.x] = view_proj[threadIdx.x];
  __syncthreads();
  const uint32_t cap16 = (per_grab * ((a.max_block_words + 3) & ~3u)) / 4;
  const uint32_t bytes16 = a.payload_bytes / 16 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)(a.payload_bytes / 16);
  const uint4 *gdesc = reinterpret_cast<const uint4 *>(a.desc);
  const uint4 *gpay = reinterpret_cast<const uint4 *>(a.payload);
  for (;;) {
    uint32_t m0 = 0;
    if (lane == 0) m0 = atomicAdd(scratch + kQueue, per_grab);
    m0 = __shfl_sync(kFull, m0, 0);
    if (m0 >= a.n_meshlets) break;
    const uint32_t cnt = min(per_grab, a.n_meshlets - m0);
    uint4 dv = make_uint4(0, 0, 0, 0);
    if (lane < 2 * cnt) dv = __ldg(gdesc + 2ull * m0 + lane);
    uint32_t end16 = bytes16;
    if (m0 + cnt < a.n_meshlets) end16 = __ldg(&a.desc[m0 + cnt].payload_off16);
    if (lane < 2 * cnt) reinterpret_cast<uint4 *>(sdesc)[lane] = dv;
    const uint32_t start16 = __shfl_sync(kFull, dv.x, 0);
    bool grab_staged = end16 >= start16 && end16 - start16 <= cap16 && end16 <= bytes16;
    if (grab_staged) {
      uint4 *dst = reinterpret_cast<uint4 *>(spay);
      for (uint32_t i = lane; i < end16 - start16; i += 32) dst[i] = __ldg(gpay + start16 + i);
    }
    __syncwarp();
    uint32_t n_keep = 0;
    for (uint32_t j = 0; j < cnt; j++) {
      const uint4 *sd = reinterpret_cast<const uint4 *>(sdesc) + 2 * j;
      const Desc d = unpack_desc(sd[0], sd[1]);
      if (!header_ok(d, a)) {
        if (lane == 0) set_status(status, MC_ERR_CORRUPT);
        continue;
      }
      const Grid g = load_grid(a.grids + d.grid);
      if (box_outside(d, g, s_M, lane)) continue;
      const uint32_t padded16 = ((block_words(d) + 3) & ~3u) / 4;
      const uint32_t *sw;
      if (grab_staged && d.off16 >= start16 && d.off16 - start16 + padded16 <= end16 - start16) {
        sw = spay + 4 * (d.off16 - start16);
      } else {
        grab_staged = false;
        __syncwarp();
        stage_payload(d, a.payload, spay, lane);
        __syncwarp();
        sw = spay;
      }
      const uint32_t r = cull_dispatch<CHECKED>(d, g, s_M, sw, sI, cx, cy, cw, surv, n_keep, lane, out_pos);
      if (r == 0xFFFFFFFFu) {
        if (lane == 0) set_status(status, MC_ERR_CORRUPT);
      } else {
        n_keep = r;
      }
      __syncwarp();
    }
    if (n_keep) {
      uint32_t dst = 0;
      if (lane == 0) dst = atomicAdd(scratch + kCount, n_keep);
      dst = __shfl_sync(kFull, dst, 0);
      uint32_t *o = tri_out + 3ull * dst;
      for (uint32_t i = lane; i < 3 * n_keep; i += 32) o[i] = surv[i];
    }
    __syncwarp();
  }
  // the last CTA publishes the count and resets the scratch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      __threadfence();
      *tri_count = atomicAdd(scratch + kCount, 0u);
      atomicExch(scratch + kCount, 0u);
      atomicExch(scratch + kQueue, 0u);
      atomicExch(scratch + kDone, 0u);
    }
  }
}

// ------------------------------------------------------------- launchers
cudaError_t launch_plain(const BatchArgs &a, uint32_t first, uint32_t count, uint32_t warps,
                         uint32_t max_block_words, bool checked, uint8_t *out_local,
                         uint32_t *out_global, float *out_pos, uint32_t *status,
                         cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t spw = warp_smem_bytes(max_block_words);
  const uint32_t smem = spw * warps;
  const uint32_t grid = (count + warps - 1) / warps;
  if (checked) {
    cudaFuncSetAttribute(decode_plain_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_plain_kernel<true><<<grid, warps * 32, smem, s>>>(a, first, count, spw, out_local,
                                                             out_global, out_pos, status);
  } else {
    cudaFuncSetAttribute(decode_plain_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_plain_kernel<false><<<grid, warps * 32, smem, s>>>(a, first, count, spw, out_local,
                                                              out_global, out_pos, status);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs &a, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                         uint32_t max_block_words, bool checked, uint8_t *out_local,
                         uint32_t *out_global, float *out_pos, uint32_t *status,
                         uint32_t *scratch, cudaStream_t s) {
  const uint32_t spw = batch_smem_per_warp(max_block_words, per_grab);
  const uint32_t smem = spw * warps;
  if (checked) {
    cudaFuncSetAttribute(decode_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_batch_kernel<true><<<ctas, warps * 32, smem, s>>>(a, per_grab, spw, out_local,
                                                             out_global, out_pos, status, scratch);
  } else {
    cudaFuncSetAttribute(decode_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_batch_kernel<false><<<ctas, warps * 32, smem, s>>>(a, per_grab, spw, out_local,
                                                              out_global, out_pos, status, scratch);
  }
  return cudaGetLastError();
}

cudaError_t launch_cull(const BatchArgs &a, const float *view_proj, uint32_t ctas, uint32_t warps,
                        uint32_t per_grab, bool checked, uint32_t *tri_out, uint32_t *tri_count,
                        float *out_pos, uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  const uint32_t smem = cull_smem_per_warp(a.max_block_words, a.max_tris, per_grab) * warps;
  if (checked) {
    cudaFuncSetAttribute(decode_cull_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_cull_kernel<true><<<ctas, warps * 32, smem, s>>>(a, view_proj, per_grab, tri_out, tri_count,
                                                            out_pos, status, scratch);
  } else {
    cudaFuncSetAttribute(decode_cull_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_cull_kernel<false><<<ctas, warps * 32, smem, s>>>(a, view_proj, per_grab, tri_out, tri_count,
                                                             out_pos, status, scratch);
  }
  return cudaGetLastError();
}

cudaError_t launch_requests(const BatchArgs &a, const mc_request *reqs, uint32_t n_reqs,
                            uint32_t total_work, uint32_t ctas, uint32_t warps, uint32_t per_grab,
                            bool checked, uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  const uint32_t spw = 4 * (((a.max_block_words + 3) & ~3u) + kSlackWords) + kStreamBytes;
  const uint32_t smem = spw * warps;
  if (checked) {
    cudaFuncSetAttribute(decode_requests_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_requests_kernel<true><<<ctas, warps * 32, smem, s>>>(a, reqs, n_reqs, total_work, per_grab,
                                                                status, scratch);
  } else {
    cudaFuncSetAttribute(decode_requests_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    decode_requests_kernel<false><<<ctas, warps * 32, smem, s>>>(a, reqs, n_reqs, total_work, per_grab,
                                                                 status, scratch);
  }
  return cudaGetLastError();
}

int max_ctas_per_sm_requests(uint32_t warps, uint32_t max_block_words) {
  int n = 0;
  const int smem = (int)((4 * (((max_block_words + 3) & ~3u) + kSlackWords) + kStreamBytes) * warps);
  cudaFuncSetAttribute(decode_requests_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(decode_requests_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decode_requests_kernel<false>, warps * 32, smem);
  return n;
}

int max_ctas_per_sm_batch(uint32_t warps, uint32_t max_block_words, uint32_t per_grab) {
  int n = 0;
  const int smem = (int)(batch_smem_per_warp(max_block_words, per_grab) * warps);
  if (smem > 227 * 1024) return 0;
  cudaFuncSetAttribute(decode_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(decode_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decode_batch_kernel<false>, warps * 32, smem);
  return n;
}

int max_ctas_per_sm_cull(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                         uint32_t per_grab) {
  int n = 0;
  const int smem = (int)(cull_smem_per_warp(max_block_words, max_tris, per_grab) * warps);
  if (smem > 227 * 1024) return 0;
  cudaFuncSetAttribute(decode_cull_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(decode_cull_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decode_cull_kernel<false>, warps * 32, smem);
  return n;
}


}  // namespace mcdev
