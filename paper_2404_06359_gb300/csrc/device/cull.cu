// Fused decode + cull + compaction, one view per launch, for sm_103a:
// survivors compacted in any order or, ORDERED, in meshlet order.
#include <cuda_runtime.h>

#include "cull_common.cuh"
#include "decode_warp.cuh"
#include "grab_loop.cuh"
#include "kernels.h"

namespace mcdev {

// Meshlet tests of a grab: bit j of the result is set when all 8 corners of
// meshlet j's quantisation box [L, L + 2^b - 1] (dequantised like the
// vertices) are outside one clip plane, or when cones is set, eye_ok and the
// meshlet's normal cone faces away from eye.  Lane 8 i + c takes corner c of
// meshlet 4 p + i in pass p and collects the planes the corner is outside
// of; the eight lanes of a meshlet AND their plane masks; lane 8 i runs the
// cone test.  A descriptor with an out-of-range grid index gets no bit (its
// header check rejects it).
__device__ __forceinline__ uint32_t grab_outside(const BatchArgs &a, uint32_t m0,
                                                 const uint32_t *sdesc, uint32_t cnt,
                                                 const float *M, const mc_cone *cones,
                                                 const float *eye, bool eye_ok, uint32_t lane) {
  uint32_t out = 0;
  const uint32_t corner = lane & 7u;
  for (uint32_t p = 0; 4 * p < cnt; p++) {
    const uint32_t j = 4 * p + (lane >> 3);
    uint32_t mask = 0;
    bool away = false;
    if (j < cnt) {
      const uint32_t *w = sdesc + 8 * j;
      const uint32_t b = (w[4] >> 8) & 0xFFu, grid = w[4] >> 16;
      if (grid < a.n_grids) {
        const Grid g = load_grid(a.grids + grid);
        const uint32_t ext = field_max(b);
        float p3[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const uint32_t L = w[5 + c];
          p3[c] = dequant((corner >> c) & 1u ? L + ext : L, g.G[c], g.D[c]);
        }
        const float cw = clip_row(M, 3, p3[0], p3[1], p3[2]);
#pragma unroll
        for (int r = 0; r < 3; r++) {
          const float comp = clip_row(M, r, p3[0], p3[1], p3[2]);
          mask |= (__fadd_rn(cw, comp) < 0.0f ? 1u : 0u) << (2 * r);
          mask |= (__fsub_rn(cw, comp) < 0.0f ? 2u : 0u) << (2 * r);
        }
      }
      if (cones && eye_ok && corner == 0) away = cone_faces_away(cones + m0 + j, eye);
    }
    mask &= __shfl_xor_sync(kFull, mask, 1);
    mask &= __shfl_xor_sync(kFull, mask, 2);
    mask &= __shfl_xor_sync(kFull, mask, 4);
    const uint32_t bal = __ballot_sync(kFull, (mask != 0 || away) && corner == 0);
    out |= ((bal & 1u) | ((bal >> 7) & 2u) | ((bal >> 14) & 4u) | ((bal >> 21) & 8u)) << (4 * p);
  }
  return out;
}

constexpr uint32_t kSurvSources = 32;  // meshlets one survivor buffer may reference
constexpr uint32_t kSurvMeshlets = 6;  // survivor buffer capacity, in largest meshlets

struct CullLayout {
  uint32_t stream, clip, n_clip, svb, surv, cap, bytes;
};
// Per-warp shared memory of the fused cull: the grab loop's buffers, the
// strip entries, clip-space x, y, w of the meshlet's vertices
// (V <= max_verts entries), the vertex bases of the meshlets the survivor
// buffer references, and the survivor buffer (cap triangles, one word each:
// three local indices and the source slot).
__host__ __device__ inline CullLayout cull_layout(uint32_t max_block_words, uint32_t max_tris,
                                                  uint32_t max_verts, uint32_t per_grab) {
  CullLayout l;
  l.stream = grab_loop_bytes(max_block_words, per_grab);
  l.clip = l.stream + kStreamBytes;
  l.n_clip = (max_verts + 7) & ~7u;
  l.svb = l.clip + 12 * l.n_clip;
  l.surv = l.svb + 4 * kSurvSources;
  l.cap = kSurvMeshlets * max_tris;
  l.bytes = l.surv + ((4 * l.cap + 15) & ~15u);
  return l;
}
uint32_t cull_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t max_verts,
                            uint32_t per_grab) {
  return cull_layout(max_block_words, max_tris, max_verts, per_grab).bytes;
}

// Decode + cull of one staged meshlet; survivors are appended to surv[] from
// position n_keep as x | y << 8 | z << 16 | tag (tag = source slot << 24).
// Returns the new count, or 0xFFFFFFFF for a corrupt stream (checked build).
// Clip x, y of vertex v sit in cxy[v] (float2), clip w in cw[v].
template <bool CHECKED, bool B16, int RM>
__device__ __forceinline__ uint32_t cull_staged(const Desc &d, const Grid &g, const float *M,
                                                const uint32_t *sw, uint8_t *sI, float2 *cxy,
                                                float *cw, uint32_t *surv, uint32_t n_keep,
                                                uint32_t tag, uint32_t lane, float *out_pos) {
  if (CHECKED && !stream_header_ok(d, sw)) return 0xFFFFFFFFu;
  const uint32_t *pw = sw + conn_words(d);
  const bool small = small_coords(d);
  float *op = out_pos + 3ull * (d.vbase + lane);
  const uint32_t vpasses = (d.V + 31) >> 5;
  uint32_t v = lane;
  for (uint32_t i = 0; i < vpasses; i++, v += 32, op += 96) {
    const uint32_t vv = min(v, d.V - 1);  // idle lanes recompute the last vertex
    uint32_t q[3];
    vertex_q<B16>(pw, vv, d.b, q);
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
      p[c] = small ? dequant_small(d.L[c] + q[c], g.G[c], g.D[c]) : dequant(d.L[c] + q[c], g.G[c], g.D[c]);
    stg3_f32_if(op, p[0], p[1], p[2], v < d.V);
    cxy[vv] = make_float2(clip_row(M, 0, p[0], p[1], p[2]), clip_row(M, 1, p[0], p[1], p[2]));
    cw[vv] = clip_row(M, 3, p[0], p[1], p[2]);
  }
  __syncwarp();
  const uint32_t a_surv = smem_addr(surv);
  const bool ok = walk_triangles<CHECKED, RM>(
      d, sw, sI, lane, [&](uint32_t k, uint32_t x, uint32_t y, uint32_t z, bool live) {
        // evaluated on every lane without branches; dead lanes read vertex 0
        const uint32_t xi = live ? x : 0u, yi = live ? y : 0u, zi = live ? z : 0u;
        const float2 p0 = cxy[xi], p1 = cxy[yi], p2 = cxy[zi];
        const float w0 = cw[xi], w1 = cw[yi], w2 = cw[zi];
        const float c0 = __fmaf_rn(p1.y, w2, -__fmul_rn(w1, p2.y));
        const float c1 = __fmaf_rn(p1.x, w2, -__fmul_rn(w1, p2.x));
        const float c2 = __fmaf_rn(p1.x, p2.y, -__fmul_rn(p1.y, p2.x));
        const float det = __fmaf_rn(w0, c2, __fmaf_rn(-p0.y, c1, __fmul_rn(p0.x, c0)));
        const bool behind = (w0 <= 0.0f) | (w1 <= 0.0f) | (w2 <= 0.0f);
        const bool keep = live & (x != y) & (y != z) & (x != z) & (behind | (det > 0.0f));
        const uint32_t bal = __ballot_sync(kFull, keep);
        const uint32_t o = n_keep + __popc(bal & ((1u << lane) - 1u));
        sts_u32_if(a_surv + 4 * o, x | (y << 8) | (z << 16) | tag, keep);
        n_keep += __popc(bal);
      });
  return ok ? n_keep : 0xFFFFFFFFu;
}

template <bool CHECKED>
__device__ __forceinline__ uint32_t cull_dispatch(const Desc &d, const Grid &g, const float *M,
                                                  const uint32_t *sw, uint8_t *sI, float2 *cxy,
                                                  float *cw, uint32_t *surv, uint32_t n_keep,
                                                  uint32_t tag, uint32_t lane, float *out_pos) {
#define MC_CULL(B, R) cull_staged<CHECKED, B, R>(d, g, M, sw, sI, cxy, cw, surv, n_keep, tag, lane, out_pos)
  if (d.b == 16) {
    if (d.w == 8) return MC_CULL(true, kReuseBytes);
    if (d.w == 0) return MC_CULL(true, kPlainGts);
    return MC_CULL(true, kReuseBits);
  }
  if (d.w == 8) return MC_CULL(false, kReuseBytes);
  if (d.w == 0) return MC_CULL(false, kPlainGts);
  return MC_CULL(false, kReuseBits);
#undef MC_CULL
}

// Writes a warp's buffered survivors as global index triples: one atomicAdd
// reserves their output range, word e of which is corner e % 3 of survivor
// e / 3 (coalesced stores).
__device__ __forceinline__ void cull_flush(const uint32_t *surv, const uint32_t *svb, uint32_t n,
                                           uint32_t lane, uint32_t *tri_out, uint32_t *counter) {
  uint32_t dst = 0;
  if (lane == 0) dst = atomicAdd(counter, n);
  dst = __shfl_sync(kFull, dst, 0);
  uint32_t *o = tri_out + 3ull * dst;
  for (uint32_t e = lane; e < 3 * n; e += 32) {
    const uint32_t t = e / 3, c = e - 3 * t;
    const uint32_t p = surv[t];
    o[e] = svb[p >> 24] + ((p >> (8 * c)) & 0xFFu);
  }
  __syncwarp();
}

// Ordered compaction: decoupled look-back over the grabs (each grab is a
// contiguous run of meshlets taken from the queue in order).  When a warp has
// decoded grab g it publishes g's survivor count as an aggregate (grab 0: as
// its inclusive prefix) and goes on to its next grab; after that one it
// resolves g: it sums the values g's predecessors have published back to the
// nearest inclusive prefix (32 at a time, one per lane), then publishes g's
// inclusive prefix.  By then g's predecessors have almost always published,
// so the warp seldom waits.  (Trying to resolve g at once, before the next
// grab, was 4 % slower: the attempt often found a predecessor unpublished.)  A grab's aggregate is published without waiting on
// anything, grabs are handed out in order to running warps and no grab waits
// on a later one, so the chain resolves; every wait is bounded (about a
// second).  State word: bits 62-63 = 0 not yet, 1 aggregate, 2 inclusive
// prefix; bits 0-31 = value.
// The state words carry only their own values (no other data is handed
// between warps through them: each grab writes its own survivors, read only
// after the kernel), so relaxed gpu-scope accesses of the whole 64-bit word
// suffice; release / acquire would make each publication wait for the
// warp's earlier position and survivor stores.
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62;
__device__ __forceinline__ void grab_publish(uint64_t *state, uint32_t g, uint32_t count,
                                             uint32_t lane) {
  if (lane == 0) st_relaxed_u64(state + g, (g == 0 ? kInc : kAgg) | count);
}
// The exclusive prefix of grab g (published as an aggregate before), or
// 0xFFFFFFFF when a wait on an unpublished predecessor gave up after
// wait_cycles clock cycles (0 = kWaitCycles).
__device__ __forceinline__ uint32_t grab_lookback(uint64_t *state, uint32_t g, uint32_t count,
                                                  uint32_t lane, uint32_t wait_cycles) {
  if (g == 0) return 0;
  uint32_t excl = 0;
  int64_t j = (int64_t)g - 1;
  // elapsed cycles in 32 bits (the limit is below 2^32; unsigned differences survive the wrap)
  const uint32_t limit = wait_cycles ? wait_cycles : (uint32_t)kWaitCycles;
  const uint32_t t0 = (uint32_t)clock64();
  for (;;) {
    const int64_t idx = j - (int64_t)lane;
    const uint64_t v = idx >= 0 ? ld_relaxed_u64(state + idx) : kInc;  // before grab 0: prefix 0
    const uint32_t flag = (uint32_t)(v >> 62);
    const uint32_t inc_mask = __ballot_sync(kFull, flag == 2u);
    const uint32_t wait_mask = __ballot_sync(kFull, flag == 0u);
    const uint32_t stop = inc_mask ? (uint32_t)__ffs(inc_mask) - 1u : 31u;  // lanes 0..stop count
    const uint32_t upto = stop == 31u ? kFull : ((2u << stop) - 1u);
    if (wait_mask & upto) {
      if (__any_sync(kFull, (uint32_t)clock64() - t0 > limit)) return 0xFFFFFFFFu;
      continue;
    }
    excl += __reduce_add_sync(kFull, lane <= stop ? (uint32_t)v : 0u);
    if (inc_mask) break;
    j -= 32;
  }
  if (lane == 0) st_relaxed_u64(state + g, kInc | (uint64_t)(excl + count));
  return excl;
}

// Writes a grab's buffered survivors at a known output position (ordered
// compaction); same layout as cull_flush.
__device__ __forceinline__ void cull_write_at(const uint32_t *surv, const uint32_t *svb, uint32_t n,
                                              uint32_t lane, uint32_t *tri_out, uint32_t dst) {
  uint32_t *o = tri_out + 3ull * dst;
  for (uint32_t e = lane; e < 3 * n; e += 32) {
    const uint32_t t = e / 3, c = e - 3 * t;
    const uint32_t p = surv[t];
    o[e] = svb[p >> 24] + ((p >> (8 * c)) & 0xFFu);
  }
  __syncwarp();
}

// Fused decode + cull + compaction.  Persistent warps run the grab loop,
// drop meshlets whose box is outside the frustum before touching their
// triangles, decode and cull the rest and collect survivors in shared memory
// across grabs; a full buffer (or the end of the work) is written out with
// one atomicAdd.  ORDERED: survivors are written in meshlet order, each
// grab's at the position the look-back over order_state gives; the buffer is
// split into two halves (per_grab <= kSurvMeshlets / 2 meshlets each): a
// grab's survivors wait in one half while the next grab is decoded into the
// other; the last grab writes the count.
template <bool CHECKED, int MAX_THREADS, bool ORDERED>
__global__ void __launch_bounds__(MAX_THREADS) decode_cull_kernel(BatchArgs a, const float *view_proj,
                                                          const mc_cone *cones, uint32_t per_grab,
                                                          uint32_t *tri_out, uint32_t *tri_count,
                                                          float *out_pos, uint32_t *status,
                                                          uint32_t *scratch, uint64_t *order_state) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float s_M[16];
  __shared__ float s_eye[4];  // camera position, [3] = 1 when there is one
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const CullLayout L = cull_layout(a.max_block_words, a.max_tris, a.max_verts, per_grab);
  uint8_t *base = smem + warp * L.bytes;
  uint8_t *sI = base + L.stream;
  float2 *cxy = reinterpret_cast<float2 *>(base + L.clip);
  float *cw = reinterpret_cast<float *>(cxy + L.n_clip);
  uint32_t *svb = reinterpret_cast<uint32_t *>(base + L.svb);
  uint32_t *surv = reinterpret_cast<uint32_t *>(base + L.surv);
  uint32_t n_keep = 0, n_src = 0;  // buffered survivors, meshlets they reference
  // ORDERED: half of the buffer per grab; the previous grab (first meshlet
  // pend_m0, pend_n survivors), whose output position is resolved after the
  // current one, sits in the other half
  const uint32_t half_cap = L.cap / 2, half_src = kSurvSources / 2;
  uint32_t half = 0, pend_m0 = 0xFFFFFFFFu, pend_n = 0;
  if (threadIdx.x < 16) s_M[threadIdx.x] = view_proj[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) s_eye[3] = cones && view_eye(s_M, s_eye) ? 1.0f : 0.0f;
  __syncthreads();
  const bool eye_ok = s_eye[3] != 0.0f;
  auto resolve = [&](uint32_t m0, uint32_t n, uint32_t h) {
    const uint32_t excl = grab_lookback(order_state, m0 / per_grab, n, lane, a.wait_cycles);
    if (excl == 0xFFFFFFFFu) {
      if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
      return;
    }
    cull_write_at(surv + h * half_cap, svb + h * half_src, n, lane, tri_out, excl);
    if (lane == 0 && m0 + per_grab >= a.n_meshlets) *tri_count = excl + n;
  };
  grab_loop<ORDERED ? 0 : 1>(a, per_grab, base, lane, scratch + kQueue, status,
                [&](uint32_t m0, const uint32_t *sdesc, uint32_t cnt) {
                  return grab_outside(a, m0, sdesc, cnt, s_M, cones, s_eye, eye_ok, lane);
                },
                [&](const Desc &d, const uint32_t *sw, uint32_t j, uint32_t outside, uint32_t) {
                  if ((outside >> j) & 1u) return;
                  const Grid g = load_grid(a.grids + d.grid);
                  // d.T <= max_tris (header_ok), so the meshlet fits an emptied buffer
                  // (ordered: a whole grab always fits its half)
                  if (!ORDERED && (n_keep + d.T > L.cap || n_src == kSurvSources)) {
                    cull_flush(surv, svb, n_keep, lane, tri_out, scratch + kCount);
                    n_keep = 0;
                    n_src = 0;
                  }
                  uint32_t *hs = ORDERED ? surv + half * half_cap : surv;
                  uint32_t *hb = ORDERED ? svb + half * half_src : svb;
                  if (lane == 0) hb[n_src] = d.vbase;
                  const uint32_t r = cull_dispatch<CHECKED>(d, g, s_M, sw, sI, cxy, cw, hs, n_keep,
                                                            n_src << 24, lane, out_pos);
                  if (r == 0xFFFFFFFFu) {
                    if (lane == 0) set_status(status, MC_ERR_CORRUPT);
                  } else if (r != n_keep) {
                    n_keep = r;
                    n_src++;
                  }
                  __syncwarp();
                },
                [&](uint32_t m0, uint32_t) {
                  if (!ORDERED) return;
                  grab_publish(order_state, m0 / per_grab, n_keep, lane);
                  if (pend_m0 != 0xFFFFFFFFu) resolve(pend_m0, pend_n, half ^ 1u);
                  pend_m0 = m0;  // resolved after the next grab
                  pend_n = n_keep;
                  half ^= 1u;
                  n_keep = 0;
                  n_src = 0;
                });
  if (ORDERED && pend_m0 != 0xFFFFFFFFu) resolve(pend_m0, pend_n, half ^ 1u);
  if (!ORDERED && n_keep) cull_flush(surv, svb, n_keep, lane, tri_out, scratch + kCount);
  // the last CTA publishes the count and resets the scratch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      __threadfence();
      if (!ORDERED) *tri_count = atomicAdd(scratch + kCount, 0u);
      atomicExch(scratch + kCount, 0u);
      atomicExch(scratch + kQueue, 0u);
      atomicExch(scratch + kDone, 0u);
    }
  }
}

// ------------------------------------------------------------- launchers

namespace {
// Small CTAs (up to 4 warps) get a build whose register budget needs no
// spills; larger CTAs the 512-thread build.
template <bool CHECKED, int MAX_THREADS, bool ORDERED>
cudaError_t launch_cull_t(const BatchArgs &a, const float *view_proj, const mc_cone *cones,
                          uint32_t ctas, uint32_t warps, uint32_t per_grab, uint32_t *tri_out,
                          uint32_t *tri_count, float *out_pos, uint32_t *status, uint32_t *scratch,
                          uint64_t *order_state, cudaStream_t s) {
  const uint32_t smem =
      cull_smem_per_warp(a.max_block_words, a.max_tris, a.max_verts, per_grab) * warps;
  prepare(fn(decode_cull_kernel<CHECKED, MAX_THREADS, ORDERED>));
  decode_cull_kernel<CHECKED, MAX_THREADS, ORDERED><<<ctas, warps * 32, smem, s>>>(
      a, view_proj, cones, per_grab, tri_out, tri_count, out_pos, status, scratch, order_state);
  return cudaGetLastError();
}
template <int MAX_THREADS, bool ORDERED>
cudaError_t launch_cull_c(const BatchArgs &a, const float *view_proj, const mc_cone *cones,
                          uint32_t ctas, uint32_t warps, uint32_t per_grab, bool checked,
                          uint32_t *tri_out, uint32_t *tri_count, float *out_pos, uint32_t *status,
                          uint32_t *scratch, uint64_t *order_state, cudaStream_t s) {
  if (checked)
    return launch_cull_t<true, MAX_THREADS, ORDERED>(a, view_proj, cones, ctas, warps, per_grab,
                                                     tri_out, tri_count, out_pos, status, scratch,
                                                     order_state, s);
  return launch_cull_t<false, MAX_THREADS, ORDERED>(a, view_proj, cones, ctas, warps, per_grab,
                                                    tri_out, tri_count, out_pos, status, scratch,
                                                    order_state, s);
}
}  // namespace

cudaError_t launch_cull(const BatchArgs &a, const float *view_proj, const mc_cone *cones,
                        uint32_t ctas, uint32_t warps, uint32_t per_grab, bool checked,
                        uint32_t *tri_out, uint32_t *tri_count, float *out_pos, uint32_t *status,
                        uint32_t *scratch, uint64_t *order_state, cudaStream_t s) {
  if (order_state) {
    if (warps <= 4)
      return launch_cull_c<128, true>(a, view_proj, cones, ctas, warps, per_grab, checked, tri_out,
                                      tri_count, out_pos, status, scratch, order_state, s);
    return launch_cull_c<512, true>(a, view_proj, cones, ctas, warps, per_grab, checked, tri_out,
                                    tri_count, out_pos, status, scratch, order_state, s);
  }
  if (warps <= 4)
    return launch_cull_c<128, false>(a, view_proj, cones, ctas, warps, per_grab, checked, tri_out,
                                     tri_count, out_pos, status, scratch, nullptr, s);
  return launch_cull_c<512, false>(a, view_proj, cones, ctas, warps, per_grab, checked, tri_out,
                                   tri_count, out_pos, status, scratch, nullptr, s);
}

int max_ctas_per_sm_cull(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                         uint32_t max_verts, uint32_t per_grab) {
  const int smem = (int)(cull_smem_per_warp(max_block_words, max_tris, max_verts, per_grab) * warps);
  if (warps > 16) return 0;
  if (warps <= 4) {
    prepare(fn(decode_cull_kernel<true, 128, false>));
    prepare(fn(decode_cull_kernel<true, 128, true>));
    prepare(fn(decode_cull_kernel<false, 128, true>));
    return occupancy(fn(decode_cull_kernel<false, 128, false>), warps * 32, smem);
  }
  prepare(fn(decode_cull_kernel<true, 512, false>));
  prepare(fn(decode_cull_kernel<true, 512, true>));
  prepare(fn(decode_cull_kernel<false, 512, true>));
  return occupancy(fn(decode_cull_kernel<false, 512, false>), warps * 32, smem);
}

}  // namespace mcdev
