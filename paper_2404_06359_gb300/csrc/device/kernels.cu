// Decode kernels for sm_103a: plain (one warp per meshlet, grid over a
// meshlet range), batched (persistent CTAs pulling meshlets from a device work
// queue) and fused decode + cull + compaction.
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

// Scratch words used by the persistent kernels.
enum { kQueue = 0, kDone = 1, kCount = 2, kViewCount = 8 };  // kViewCount..+7: per-view counts
constexpr uint32_t kMaxViews = 8;

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
  grab_loop(a, per_grab, base, lane, scratch + kQueue, status, NoPre{},
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

// ---------------------------------------------------------------- culling
__device__ __forceinline__ float clip_row(const float *M, int r, float x, float y, float z) {
  return __fmaf_rn(M[4 * r + 2], z, __fmaf_rn(M[4 * r + 1], y, __fmaf_rn(M[4 * r + 0], x, M[4 * r + 3])));
}

// Rows 0, 1 and 3 of a clip matrix in registers (clip x, y and w), so that a
// loop whose shared-memory stores could alias the matrix does not reload it.
struct ClipRows {
  float m[12];
};
__device__ __forceinline__ ClipRows clip_rows(const float *M) {
  ClipRows c;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    c.m[i] = M[i];
    c.m[4 + i] = M[4 + i];
    c.m[8 + i] = M[12 + i];
  }
  return c;
}
// clip_row's operation order; r = 0, 1, 2 for rows 0, 1, 3
__device__ __forceinline__ float clip_dot(const ClipRows &c, int r, float x, float y, float z) {
  return __fmaf_rn(c.m[4 * r + 2], z,
                   __fmaf_rn(c.m[4 * r + 1], y, __fmaf_rn(c.m[4 * r + 0], x, c.m[4 * r + 3])));
}

// Camera position of a clip matrix M (row-major, in shared memory): the point
// whose clip x, y and w are zero, from rows r0, r1, r3 and b_i = -M[i][3] by
// the cross-product inverse in FP64,
//   e = (b0 (r1 x r3) + b1 (r3 x r0) + b3 (r0 x r1)) / (r0 . (r1 x r3)),
// rounded to FP32.  Returns false (no camera: affine projection) when the
// determinant is 0 or not finite, or a coordinate is not finite.
__device__ bool view_eye(const float *M, float *eye) {
  double r0[3], r1[3], r3[3];
  for (int c = 0; c < 3; c++) {
    r0[c] = M[c];
    r1[c] = M[4 + c];
    r3[c] = M[12 + c];
  }
  const double b0 = -(double)M[3], b1 = -(double)M[7], b3 = -(double)M[15];
  auto cross = [](const double *u, const double *v, double *w) {
    w[0] = __dsub_rn(__dmul_rn(u[1], v[2]), __dmul_rn(u[2], v[1]));
    w[1] = __dsub_rn(__dmul_rn(u[2], v[0]), __dmul_rn(u[0], v[2]));
    w[2] = __dsub_rn(__dmul_rn(u[0], v[1]), __dmul_rn(u[1], v[0]));
  };
  double k0[3], k1[3], k3[3];
  cross(r1, r3, k0);
  cross(r3, r0, k1);
  cross(r0, r1, k3);
  const double det =
      __dadd_rn(__dadd_rn(__dmul_rn(r0[0], k0[0]), __dmul_rn(r0[1], k0[1])), __dmul_rn(r0[2], k0[2]));
  if (!(det != 0.0) || !isfinite(det)) return false;
  for (int c = 0; c < 3; c++) {
    const double num =
        __dadd_rn(__dadd_rn(__dmul_rn(b0, k0[c]), __dmul_rn(b1, k1[c])), __dmul_rn(b3, k3[c]));
    const double e = __ddiv_rn(num, det);
    if (!isfinite(e)) return false;
    eye[c] = __double2float_rn(e);
  }
  return true;
}

// Normal-cone test (mc_cone) of one meshlet for a camera at eye: true when
// axis . v >= s |v| + radius with v = center - eye, in FP32 with a fixed
// operation order.
__device__ __forceinline__ bool cone_record_faces_away(const float4 c0, const float4 c1,
                                                       const float *eye) {
  const float vx = __fsub_rn(c0.x, eye[0]), vy = __fsub_rn(c0.y, eye[1]), vz = __fsub_rn(c0.z, eye[2]);
  const float d = __fmaf_rn(c1.z, vz, __fmaf_rn(c1.y, vy, __fmul_rn(c1.x, vx)));
  const float l = __fsqrt_rn(__fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx))));
  return (c1.w < 1.0f) & (d >= __fmaf_rn(c1.w, l, c0.w));
}
__device__ __forceinline__ bool cone_faces_away(const mc_cone *cone, const float *eye) {
  const float4 *p = reinterpret_cast<const float4 *>(cone);
  return cone_record_faces_away(__ldg(p), __ldg(p + 1), eye);  // center, radius / axis, s
}

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
        const uint32_t ext = b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
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
// (V <= T' + 2 <= max_tris + 2 entries), the vertex bases of the meshlets
// the survivor buffer references, and the survivor buffer (cap triangles,
// one word each: three local indices and the source slot).
__host__ __device__ inline CullLayout cull_layout(uint32_t max_block_words, uint32_t max_tris,
                                                  uint32_t per_grab) {
  CullLayout l;
  l.stream = grab_loop_bytes(max_block_words, per_grab);
  l.clip = l.stream + kStreamBytes;
  l.n_clip = ((max_tris + 2 < 256 ? max_tris + 2 : 256) + 7) & ~7u;
  l.svb = l.clip + 12 * l.n_clip;
  l.surv = l.svb + 4 * kSurvSources;
  l.cap = kSurvMeshlets * max_tris;
  l.bytes = l.surv + ((4 * l.cap + 15) & ~15u);
  return l;
}
uint32_t cull_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t per_grab) {
  return cull_layout(max_block_words, max_tris, per_grab).bytes;
}

__device__ __forceinline__ void sts_u32_if(uint32_t a, uint32_t x, bool p) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.shared.u32 [%0], %1;\n}" ::"r"(a),
               "r"(x), "r"((uint32_t)p)
               : "memory");
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
// contiguous run of meshlets taken from the queue in order).  Grab g
// publishes its survivor count as an aggregate, the warp sums the values its
// predecessors have published back to the nearest inclusive prefix (32 at a
// time, one per lane), then publishes its own inclusive prefix.  Grabs are
// handed out in order to running warps and no grab waits on a later one, so
// the chain resolves; every wait is bounded (about a second).  State word:
// bits 62-63 = 0 not yet, 1 aggregate, 2 inclusive prefix; bits 0-31 = value.
// Returns the exclusive prefix, or 0xFFFFFFFF when a wait gave up.
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t grab_lookback(uint64_t *state, uint32_t g, uint32_t count,
                                                  uint32_t lane) {
  constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62;
  if (lane == 0) st_release_u64(state + g, (g == 0 ? kInc : kAgg) | count);
  if (g == 0) return 0;
  uint32_t excl = 0;
  int64_t j = (int64_t)g - 1;
  const long long t0 = clock64();
  for (;;) {
    const int64_t idx = j - (int64_t)lane;
    const uint64_t v = idx >= 0 ? ld_acquire_u64(state + idx) : kInc;  // before grab 0: prefix 0
    const uint32_t flag = (uint32_t)(v >> 62);
    const uint32_t inc_mask = __ballot_sync(kFull, flag == 2u);
    const uint32_t wait_mask = __ballot_sync(kFull, flag == 0u);
    const uint32_t stop = inc_mask ? (uint32_t)__ffs(inc_mask) - 1u : 31u;  // lanes 0..stop count
    const uint32_t upto = stop == 31u ? kFull : ((2u << stop) - 1u);
    if (wait_mask & upto) {
      if (__any_sync(kFull, clock64() - t0 > kWaitCycles)) return 0xFFFFFFFFu;
      continue;
    }
    excl += __reduce_add_sync(kFull, lane <= stop ? (uint32_t)v : 0u);
    if (inc_mask) break;
    j -= 32;
  }
  if (lane == 0) st_release_u64(state + g, kInc | (uint64_t)(excl + count));
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
// one atomicAdd.  ORDERED: survivors are written in meshlet order -- each
// grab's survivors (per_grab <= kSurvMeshlets meshlets) at the position the
// look-back over order_state gives it; the last grab writes the count.
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
  const CullLayout L = cull_layout(a.max_block_words, a.max_tris, per_grab);
  uint8_t *base = smem + warp * L.bytes;
  uint8_t *sI = base + L.stream;
  float2 *cxy = reinterpret_cast<float2 *>(base + L.clip);
  float *cw = reinterpret_cast<float *>(cxy + L.n_clip);
  uint32_t *svb = reinterpret_cast<uint32_t *>(base + L.svb);
  uint32_t *surv = reinterpret_cast<uint32_t *>(base + L.surv);
  uint32_t n_keep = 0, n_src = 0;  // buffered survivors, meshlets they reference
  if (threadIdx.x < 16) s_M[threadIdx.x] = view_proj[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) s_eye[3] = cones && view_eye(s_M, s_eye) ? 1.0f : 0.0f;
  __syncthreads();
  const bool eye_ok = s_eye[3] != 0.0f;
  grab_loop(a, per_grab, base, lane, scratch + kQueue, status,
                [&](uint32_t m0, const uint32_t *sdesc, uint32_t cnt) {
                  return grab_outside(a, m0, sdesc, cnt, s_M, cones, s_eye, eye_ok, lane);
                },
                [&](const Desc &d, const uint32_t *sw, uint32_t j, uint32_t outside, uint32_t) {
                  if ((outside >> j) & 1u) return;
                  const Grid g = load_grid(a.grids + d.grid);
                  // d.T <= max_tris (header_ok), so the meshlet fits an emptied buffer
                  // (ordered: a whole grab always fits)
                  if (!ORDERED && (n_keep + d.T > L.cap || n_src == kSurvSources)) {
                    cull_flush(surv, svb, n_keep, lane, tri_out, scratch + kCount);
                    n_keep = 0;
                    n_src = 0;
                  }
                  if (lane == 0) svb[n_src] = d.vbase;
                  const uint32_t r = cull_dispatch<CHECKED>(d, g, s_M, sw, sI, cxy, cw, surv, n_keep,
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
                  const uint32_t g = m0 / per_grab;
                  const uint32_t excl = grab_lookback(order_state, g, n_keep, lane);
                  if (excl == 0xFFFFFFFFu) {
                    if (lane == 0) set_status(status, MC_ERR_TIMEOUT);
                  } else {
                    cull_write_at(surv, svb, n_keep, lane, tri_out, excl);
                    if (lane == 0 && m0 + per_grab >= a.n_meshlets) *tri_count = excl + n_keep;
                  }
                  n_keep = 0;
                  n_src = 0;
                });
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

// ------------------------------------------------------------ multi-view culling
// One launch culls the batch against up to kMaxViews clip matrices: each
// meshlet is staged, its positions dequantised and its strip walked once,
// then the clip coordinates, the triangle tests and the compaction run once
// per view that the meshlet tests leave.  Per view the tests and their FP32
// evaluation are those of decode_cull_kernel, so view v's survivors are the
// ones mc_decode_cull gives for matrix v.

// Meshlet tests of a grab (per_grab <= 4) against n_views matrices: bit
// 8 j + v of the result is set when meshlet j is skipped for view v.  Lane
// 8 j + c holds corner c of meshlet j's quantisation box, dequantised once;
// lane 8 j also holds the meshlet's cone record.
__device__ __forceinline__ uint32_t grab_outside_views(const BatchArgs &a, uint32_t m0,
                                                       const uint32_t *sdesc, uint32_t cnt,
                                                       const float *Ms, const float *eyes,
                                                       uint32_t n_views, const mc_cone *cones,
                                                       uint32_t lane) {
  const uint32_t corner = lane & 7u, j = lane >> 3;
  float p3[3] = {0.0f, 0.0f, 0.0f};
  bool box = false, cone = false;
  float4 c0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), c1 = c0;
  if (j < cnt) {
    const uint32_t *w = sdesc + 8 * j;
    const uint32_t b = (w[4] >> 8) & 0xFFu, grid = w[4] >> 16;
    if (grid < a.n_grids) {
      const Grid g = load_grid(a.grids + grid);
      const uint32_t ext = b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const uint32_t L = w[5 + c];
        p3[c] = dequant((corner >> c) & 1u ? L + ext : L, g.G[c], g.D[c]);
      }
      box = true;
    }
    if (cones && corner == 0) {
      const float4 *cp = reinterpret_cast<const float4 *>(cones + m0 + j);
      c0 = __ldg(cp);
      c1 = __ldg(cp + 1);
      cone = true;
    }
  }
  uint32_t out = 0;
  for (uint32_t v = 0; v < n_views; v++) {
    const float *M = Ms + 16 * v;
    uint32_t mask = 0;
    if (box) {
      const float cw = clip_row(M, 3, p3[0], p3[1], p3[2]);
#pragma unroll
      for (int r = 0; r < 3; r++) {
        const float comp = clip_row(M, r, p3[0], p3[1], p3[2]);
        mask |= (__fadd_rn(cw, comp) < 0.0f ? 1u : 0u) << (2 * r);
        mask |= (__fsub_rn(cw, comp) < 0.0f ? 2u : 0u) << (2 * r);
      }
    }
    const float *eye = eyes + 4 * v;
    const bool away = cone && eye[3] != 0.0f && cone_record_faces_away(c0, c1, eye);
    mask &= __shfl_xor_sync(kFull, mask, 1);
    mask &= __shfl_xor_sync(kFull, mask, 2);
    mask &= __shfl_xor_sync(kFull, mask, 4);
    const uint32_t bal = __ballot_sync(kFull, (mask != 0 || away) && corner == 0);
    out |= (bal & 0x01010101u) << v;
  }
  return out;
}

struct CullViewsLayout {
  uint32_t stream, pos, n_vtx, clip, tri, surv, cap, bytes;
};
// Per-warp shared memory of the multi-view cull: the grab loop's buffers,
// the strip entries, the meshlet's positions (x, y, z arrays) and clip x, y,
// w (V <= min(T' + 2, 256) entries), one packed word per triangle slot of
// the strip walk (32 per word of flags), and one survivor buffer of cap
// bytes per view (the survivors' triangle slots: a quarter of the shared
// memory packed words would take, which leaves room for more warps per SM).
__host__ __device__ inline CullViewsLayout cull_views_layout(uint32_t max_block_words,
                                                             uint32_t max_tris, uint32_t per_grab,
                                                             uint32_t n_views) {
  CullViewsLayout l;
  l.stream = grab_loop_bytes(max_block_words, per_grab);
  l.pos = l.stream + kStreamBytes;
  l.n_vtx = ((max_tris + 2 < 256 ? max_tris + 2 : 256) + 7) & ~7u;
  l.clip = l.pos + 12 * l.n_vtx;
  l.tri = l.clip + 12 * l.n_vtx;
  l.surv = l.tri + 4 * ((max_tris + 31) & ~31u);
  l.cap = (max_tris + 15) & ~15u;
  l.bytes = l.surv + ((l.cap * n_views + 15) & ~15u);
  return l;
}
uint32_t cull_views_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t per_grab,
                                  uint32_t n_views) {
  return cull_views_layout(max_block_words, max_tris, per_grab, n_views).bytes;
}

// One staged meshlet against the views in `views` (bit v = view v): the
// positions go to out_pos and to shared memory, the strip walk leaves one
// word per triangle slot (x | y << 8 | z << 16, or 0 for a dead slot or a
// triangle with two equal indices), then per view the clip coordinates,
// the back-face test and the compaction of the surviving slots (one byte
// each) into that view's buffer.  Lane v
// returns the survivor count of view v (0 for the others); the result is
// false for a corrupt stream (checked build).
template <bool CHECKED, bool B16, int RM>
__device__ __forceinline__ bool cull_views_staged(const Desc &d, const Grid &g, const float *Ms,
                                                  uint32_t views, const uint32_t *sw, uint8_t *sI,
                                                  float *px, uint32_t n_vtx, float2 *cxy, float *cw,
                                                  uint32_t *stri, uint32_t *surv, uint32_t cap,
                                                  uint32_t lane, float *out_pos, uint32_t &my_n) {
  my_n = 0;
  if (CHECKED && !stream_header_ok(d, sw)) return false;
  const uint32_t *pw = sw + conn_words(d);
  const bool small = small_coords(d);
  float *py = px + n_vtx, *pz = py + n_vtx;
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
    px[vv] = p[0];
    py[vv] = p[1];
    pz[vv] = p[2];
  }
  const uint32_t a_tri = smem_addr(stri);
  const bool ok = walk_triangles<CHECKED, RM>(
      d, sw, sI, lane, [&](uint32_t k, uint32_t x, uint32_t y, uint32_t z, bool live) {
        const bool keep = live & (x != y) & (y != z) & (x != z);
        sts_u32_if(a_tri + 4 * k, keep ? (x | (y << 8) | (z << 16)) : 0u, true);
      });
  if (CHECKED && !ok) return false;
  const uint32_t tpasses = (d.T + 31) >> 5;
  for (uint32_t vw = views; vw; vw &= vw - 1) {
    const uint32_t view = __ffs(vw) - 1;
    const ClipRows cr = clip_rows(Ms + 16 * view);
    v = lane;
    for (uint32_t i = 0; i < vpasses; i++, v += 32) {
      const uint32_t vv = min(v, d.V - 1);
      const float x = px[vv], y = py[vv], z = pz[vv];
      cxy[vv] = make_float2(clip_dot(cr, 0, x, y, z), clip_dot(cr, 1, x, y, z));
      cw[vv] = clip_dot(cr, 2, x, y, z);
    }
    __syncwarp();
    const uint32_t a_surv = smem_addr(reinterpret_cast<uint8_t *>(surv) + cap * view);
    uint32_t n = 0;
    uint32_t k = lane;
    for (uint32_t i = 0; i < tpasses; i++, k += 32) {
      const uint32_t t = lds_u32(a_tri + 4 * k);
      const uint32_t xi = t & 0xFFu, yi = (t >> 8) & 0xFFu, zi = t >> 16;
      const float2 p0 = cxy[xi], p1 = cxy[yi], p2 = cxy[zi];
      const float w0 = cw[xi], w1 = cw[yi], w2 = cw[zi];
      const float c0 = __fmaf_rn(p1.y, w2, -__fmul_rn(w1, p2.y));
      const float c1 = __fmaf_rn(p1.x, w2, -__fmul_rn(w1, p2.x));
      const float c2 = __fmaf_rn(p1.x, p2.y, -__fmul_rn(p1.y, p2.x));
      const float det = __fmaf_rn(w0, c2, __fmaf_rn(-p0.y, c1, __fmul_rn(p0.x, c0)));
      const bool behind = (w0 <= 0.0f) | (w1 <= 0.0f) | (w2 <= 0.0f);
      const bool keep = (t != 0u) & (behind | (det > 0.0f));
      const uint32_t bal = __ballot_sync(kFull, keep);
      sts_u8_if(a_surv + n + __popc(bal & ((1u << lane) - 1u)), k, keep);
      n += __popc(bal);
    }
    if (lane == view) my_n = n;
    __syncwarp();  // the next view rewrites the clip coordinates
  }
  return true;
}

template <bool CHECKED>
__device__ __forceinline__ bool cull_views_dispatch(const Desc &d, const Grid &g, const float *Ms,
                                                    uint32_t views, const uint32_t *sw, uint8_t *sI,
                                                    float *px, uint32_t n_vtx, float2 *cxy,
                                                    float *cw, uint32_t *stri, uint32_t *surv,
                                                    uint32_t cap, uint32_t lane, float *out_pos,
                                                    uint32_t &my_n) {
#define MC_CULLV(B, R)                                                                           \
  cull_views_staged<CHECKED, B, R>(d, g, Ms, views, sw, sI, px, n_vtx, cxy, cw, stri, surv, cap, \
                                   lane, out_pos, my_n)
  if (d.b == 16) {
    if (d.w == 8) return MC_CULLV(true, kReuseBytes);
    if (d.w == 0) return MC_CULLV(true, kPlainGts);
    return MC_CULLV(true, kReuseBits);
  }
  if (d.w == 8) return MC_CULLV(false, kReuseBytes);
  if (d.w == 0) return MC_CULLV(false, kPlainGts);
  return MC_CULLV(false, kReuseBits);
#undef MC_CULLV
}

template <bool CHECKED, int MAX_THREADS>
__global__ void __launch_bounds__(MAX_THREADS) decode_cull_views_kernel(
    BatchArgs a, const float *view_projs, uint32_t n_views, const mc_cone *cones,
    uint32_t per_grab, uint32_t *tri_out, uint64_t tri_stride, uint32_t *tri_counts,
    float *out_pos, uint32_t *status, uint32_t *scratch) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float s_M[16 * kMaxViews];
  __shared__ float s_eye[4 * kMaxViews];  // camera positions, [3] = 1 when there is one
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const CullViewsLayout L = cull_views_layout(a.max_block_words, a.max_tris, per_grab, n_views);
  uint8_t *base = smem + warp * L.bytes;
  uint8_t *sI = base + L.stream;
  float *px = reinterpret_cast<float *>(base + L.pos);
  float2 *cxy = reinterpret_cast<float2 *>(base + L.clip);
  float *cw = reinterpret_cast<float *>(cxy + L.n_vtx);
  uint32_t *stri = reinterpret_cast<uint32_t *>(base + L.tri);
  uint32_t *surv = reinterpret_cast<uint32_t *>(base + L.surv);
  for (uint32_t i = threadIdx.x; i < 16 * n_views; i += blockDim.x) s_M[i] = view_projs[i];
  __syncthreads();
  if (threadIdx.x < n_views)
    s_eye[4 * threadIdx.x + 3] =
        cones && view_eye(s_M + 16 * threadIdx.x, s_eye + 4 * threadIdx.x) ? 1.0f : 0.0f;
  __syncthreads();
  const uint32_t all = (1u << n_views) - 1u;
  grab_loop(a, per_grab, base, lane, scratch + kQueue, status,
            [&](uint32_t m0, const uint32_t *sdesc, uint32_t cnt) {
              return grab_outside_views(a, m0, sdesc, cnt, s_M, s_eye, n_views, cones, lane);
            },
            [&](const Desc &d, const uint32_t *sw, uint32_t j, uint32_t skipped, uint32_t) {
              const uint32_t views = ~(skipped >> (8 * j)) & all;
              if (!views) return;
              const Grid g = load_grid(a.grids + d.grid);
              uint32_t my_n = 0;
              if (!cull_views_dispatch<CHECKED>(d, g, s_M, views, sw, sI, px, L.n_vtx, cxy, cw,
                                                stri, surv, L.cap, lane, out_pos, my_n)) {
                if (lane == 0) set_status(status, MC_ERR_CORRUPT);
                __syncwarp();
                return;
              }
              // one atomic per view with survivors (lane v), then the views' writes:
              // a lane per survivor, its packed word looked up by slot
              uint32_t dst = 0;
              if (my_n) dst = atomicAdd(scratch + kViewCount + lane, my_n);
              for (uint32_t vw = __ballot_sync(kFull, my_n != 0); vw; vw &= vw - 1) {
                const uint32_t view = __ffs(vw) - 1;
                const uint32_t n = __shfl_sync(kFull, my_n, view);
                const uint32_t o0 = __shfl_sync(kFull, dst, view);
                // one survivor per lane: three global indices from its packed word
                uint32_t *o = tri_out + tri_stride * view + 3ull * (o0 + lane);
                const uint32_t a_sv = smem_addr(reinterpret_cast<uint8_t *>(surv) + L.cap * view);
                const uint32_t a_tr = smem_addr(stri);
                for (uint32_t t = lane; t < n; t += 32, o += 96) {
                  const uint32_t p = lds_u32(a_tr + 4 * lds_u8(a_sv + t));
                  stg3_u32_if(o, d.vbase + (p & 0xFFu), d.vbase + ((p >> 8) & 0xFFu),
                              d.vbase + (p >> 16), true);
                }
              }
              __syncwarp();
            });
  // the last CTA publishes the counts and resets the scratch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(scratch + kDone, 1u) == gridDim.x - 1) {
      __threadfence();
      for (uint32_t v = 0; v < n_views; v++)
        tri_counts[v] = atomicExch(scratch + kViewCount + v, 0u);
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
template <class K>
const void *fn(K k) {
  return reinterpret_cast<const void *>(k);
}
}  // namespace

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

namespace {
// Small CTAs (up to 4 warps) get a build whose register budget needs no
// spills; larger CTAs the 512-thread build.
template <bool CHECKED, int MAX_THREADS, bool ORDERED>
cudaError_t launch_cull_t(const BatchArgs &a, const float *view_proj, const mc_cone *cones,
                          uint32_t ctas, uint32_t warps, uint32_t per_grab, uint32_t *tri_out,
                          uint32_t *tri_count, float *out_pos, uint32_t *status, uint32_t *scratch,
                          uint64_t *order_state, cudaStream_t s) {
  const uint32_t smem = cull_smem_per_warp(a.max_block_words, a.max_tris, per_grab) * warps;
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

namespace {
template <bool CHECKED, int MAX_THREADS>
cudaError_t launch_cull_views_t(const BatchArgs &a, const float *view_projs, uint32_t n_views,
                                const mc_cone *cones, uint32_t ctas, uint32_t warps,
                                uint32_t per_grab, uint32_t *tri_out, uint64_t tri_stride,
                                uint32_t *tri_counts, float *out_pos, uint32_t *status,
                                uint32_t *scratch, cudaStream_t s) {
  const uint32_t smem =
      cull_views_smem_per_warp(a.max_block_words, a.max_tris, per_grab, n_views) * warps;
  prepare(fn(decode_cull_views_kernel<CHECKED, MAX_THREADS>));
  decode_cull_views_kernel<CHECKED, MAX_THREADS><<<ctas, warps * 32, smem, s>>>(
      a, view_projs, n_views, cones, per_grab, tri_out, tri_stride, tri_counts, out_pos, status,
      scratch);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_cull_views(const BatchArgs &a, const float *view_projs, uint32_t n_views,
                              const mc_cone *cones, uint32_t ctas, uint32_t warps,
                              uint32_t per_grab, bool checked, uint32_t *tri_out,
                              uint64_t tri_stride, uint32_t *tri_counts, float *out_pos,
                              uint32_t *status, uint32_t *scratch, cudaStream_t s) {
  if (warps <= 4)
    return checked ? launch_cull_views_t<true, 128>(a, view_projs, n_views, cones, ctas, warps,
                                                    per_grab, tri_out, tri_stride, tri_counts,
                                                    out_pos, status, scratch, s)
                   : launch_cull_views_t<false, 128>(a, view_projs, n_views, cones, ctas, warps,
                                                     per_grab, tri_out, tri_stride, tri_counts,
                                                     out_pos, status, scratch, s);
  return checked ? launch_cull_views_t<true, 512>(a, view_projs, n_views, cones, ctas, warps,
                                                  per_grab, tri_out, tri_stride, tri_counts,
                                                  out_pos, status, scratch, s)
                 : launch_cull_views_t<false, 512>(a, view_projs, n_views, cones, ctas, warps,
                                                   per_grab, tri_out, tri_stride, tri_counts,
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

int max_ctas_per_sm_cull(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                         uint32_t per_grab) {
  const int smem = (int)(cull_smem_per_warp(max_block_words, max_tris, per_grab) * warps);
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

int max_ctas_per_sm_cull_views(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                               uint32_t per_grab, uint32_t n_views) {
  const int smem =
      (int)(cull_views_smem_per_warp(max_block_words, max_tris, per_grab, n_views) * warps);
  if (warps > 16) return 0;
  if (warps <= 4) {
    prepare(fn(decode_cull_views_kernel<true, 128>));
    return occupancy(fn(decode_cull_views_kernel<false, 128>), warps * 32, smem);
  }
  prepare(fn(decode_cull_views_kernel<true, 512>));
  return occupancy(fn(decode_cull_views_kernel<false, 512>), warps * 32, smem);
}

}  // namespace mcdev
