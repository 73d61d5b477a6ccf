// Fused decode + cull + compaction against up to kMaxViews views per launch,
// for sm_103a.
#include <cuda_runtime.h>

#include "cull_common.cuh"
#include "decode_warp.cuh"
#include "grab_loop.cuh"
#include "kernels.h"

namespace mcdev {

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
      const uint32_t ext = field_max(b);
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
  uint32_t stream, pos, n_vtx, clip, clip_w, tri, surv, cap, bytes;
};
// Per-warp shared memory of the multi-view cull: the grab loop's buffers,
// the strip entries, the meshlet's positions (x, y, z arrays of n_vtx >=
// max_verts entries), the clip coordinates of two views per vertex (x, y of
// both as one 16-byte slot, then w of both as one 8-byte slot), one packed
// word per triangle slot of the strip walk (32 per word of flags), and one
// survivor buffer of cap bytes per view (the survivors' triangle slots).
__host__ __device__ inline CullViewsLayout cull_views_layout(uint32_t max_block_words,
                                                             uint32_t max_tris, uint32_t max_verts,
                                                             uint32_t per_grab, uint32_t n_views) {
  CullViewsLayout l;
  l.stream = grab_loop_bytes(max_block_words, per_grab);
  l.pos = l.stream + kStreamBytes;
  l.n_vtx = (max_verts + 7) & ~7u;
  l.clip = l.pos + 12 * l.n_vtx;
  l.clip_w = l.clip + 16 * l.n_vtx;
  l.tri = l.clip_w + 8 * l.n_vtx;
  l.surv = l.tri + 4 * ((max_tris + 31) & ~31u);
  l.cap = (max_tris + 15) & ~15u;
  l.bytes = l.surv + ((l.cap * n_views + 15) & ~15u);
  return l;
}
uint32_t cull_views_smem_per_warp(uint32_t max_block_words, uint32_t max_tris, uint32_t max_verts,
                                  uint32_t per_grab, uint32_t n_views) {
  return cull_views_layout(max_block_words, max_tris, max_verts, per_grab, n_views).bytes;
}

// The per-triangle test of the fused cull (one view): kept when all three
// indices differ (the packed word is non-zero) and either some clip w is not
// positive or the determinant of the (x, y, w) rows, evaluated in this fixed
// order, is positive.
__device__ __forceinline__ bool tri_kept(bool live, float x0, float y0, float w0, float x1,
                                         float y1, float w1, float x2, float y2, float w2) {
  const float c0 = __fmaf_rn(y1, w2, -__fmul_rn(w1, y2));
  const float c1 = __fmaf_rn(x1, w2, -__fmul_rn(w1, x2));
  const float c2 = __fmaf_rn(x1, y2, -__fmul_rn(y1, x2));
  const float det = __fmaf_rn(w0, c2, __fmaf_rn(-y0, c1, __fmul_rn(x0, c0)));
  const bool behind = (w0 <= 0.0f) | (w1 <= 0.0f) | (w2 <= 0.0f);
  return live & (behind | (det > 0.0f));
}

// One staged meshlet against the views in `views` (bit v = view v): the
// positions go to out_pos and to shared memory, the strip walk packs the
// triangles with three distinct indices densely into stri, one word each
// (x | y << 8 | z << 16; the restart degenerates and the slots past T' are
// left out, which saves a pass over 32 slots per view in most meshlets),
// then the views are taken two at a time:
// the clip coordinates of both (pxy[v] = x, y of the first and second view,
// pw[v] = their w), then one pass over the triangle slots that tests both
// views from the same packed word and shared loads and compacts each view's
// surviving slots (one byte each) into that view's buffer; a last odd view
// runs the same steps alone.  Lane v returns the survivor count of view v
// (0 for the others); the result is false for a corrupt stream (checked
// build).
template <bool CHECKED, bool B16, int RM>
__device__ __forceinline__ bool cull_views_staged(const Desc &d, const Grid &g, const float *Ms,
                                                  uint32_t views, const uint32_t *sw, uint8_t *sI,
                                                  float *px, uint32_t n_vtx, float4 *pxy, float2 *pw,
                                                  uint32_t *stri, uint32_t *surv, uint32_t cap,
                                                  uint32_t lane, float *out_pos, uint32_t &my_n) {
  my_n = 0;
  if (CHECKED && !stream_header_ok(d, sw)) return false;
  const uint32_t *qw = sw + conn_words(d);
  const bool small = small_coords(d);
  float *py = px + n_vtx, *pz = py + n_vtx;
  float *op = out_pos + 3ull * (d.vbase + lane);
  const uint32_t vpasses = (d.V + 31) >> 5;
  uint32_t v = lane;
  for (uint32_t i = 0; i < vpasses; i++, v += 32, op += 96) {
    const uint32_t vv = min(v, d.V - 1);  // idle lanes recompute the last vertex
    uint32_t q[3];
    vertex_q<B16>(qw, vv, d.b, q);
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
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t n_tri = 0;  // triangles with three distinct indices, packed densely in stri
  const bool ok = walk_triangles<CHECKED, RM>(
      d, sw, sI, lane, [&](uint32_t, uint32_t x, uint32_t y, uint32_t z, bool live) {
        const bool keep = live & (x != y) & (y != z) & (x != z);
        const uint32_t bal = __ballot_sync(kFull, keep);
        sts_u32_if(a_tri + 4 * (n_tri + __popc(bal & lt)), x | (y << 8) | (z << 16), keep);
        n_tri += __popc(bal);
      });
  if (CHECKED && !ok) return false;
  // zero the rest of the last 32-slot word: those lanes test index 0 and drop out
  sts_u32_if(a_tri + 4 * (n_tri + lane), 0u, n_tri + lane < ((n_tri + 31) & ~31u));
  const uint32_t tpasses = (n_tri + 31) >> 5;
  const uint32_t a_xy = smem_addr(pxy), a_w = smem_addr(pw);
  for (uint32_t vw = views; vw;) {
    const uint32_t va = __ffs(vw) - 1;
    vw &= vw - 1;
    const bool two = vw != 0;
    const uint32_t vb = two ? __ffs(vw) - 1 : va;
    vw &= vw - 1;
    const ClipRows ra = clip_rows(Ms + 16 * va), rb = clip_rows(Ms + 16 * vb);
    v = lane;
    for (uint32_t i = 0; i < vpasses; i++, v += 32) {
      const uint32_t vv = min(v, d.V - 1);
      const float x = px[vv], y = py[vv], z = pz[vv];
      pxy[vv] = make_float4(clip_dot(ra, 0, x, y, z), clip_dot(ra, 1, x, y, z),
                            clip_dot(rb, 0, x, y, z), clip_dot(rb, 1, x, y, z));
      pw[vv] = make_float2(clip_dot(ra, 2, x, y, z), clip_dot(rb, 2, x, y, z));
    }
    __syncwarp();
    const uint32_t a_sa = smem_addr(reinterpret_cast<uint8_t *>(surv) + cap * va);
    const uint32_t a_sb = smem_addr(reinterpret_cast<uint8_t *>(surv) + cap * vb);
    uint32_t na = 0, nb = 0;
    uint32_t k = lane;
    for (uint32_t i = 0; i < tpasses; i++, k += 32) {
      const uint32_t t = lds_u32(a_tri + 4 * k);
      const uint32_t o0 = t & 0xFFu, o1 = (t >> 8) & 0xFFu, o2 = t >> 16;
      const float4 p0 = lds_f4(a_xy + 16 * o0), p1 = lds_f4(a_xy + 16 * o1), p2 = lds_f4(a_xy + 16 * o2);
      const float2 w0 = lds_f2(a_w + 8 * o0), w1 = lds_f2(a_w + 8 * o1), w2 = lds_f2(a_w + 8 * o2);
      const bool live = t != 0u;
      const bool ka = tri_kept(live, p0.x, p0.y, w0.x, p1.x, p1.y, w1.x, p2.x, p2.y, w2.x);
      const uint32_t ba = __ballot_sync(kFull, ka);
      sts_u8_if(a_sa + na + __popc(ba & lt), k, ka);
      na += __popc(ba);
      if (two) {
        const bool kb = tri_kept(live, p0.z, p0.w, w0.y, p1.z, p1.w, w1.y, p2.z, p2.w, w2.y);
        const uint32_t bb = __ballot_sync(kFull, kb);
        sts_u8_if(a_sb + nb + __popc(bb & lt), k, kb);
        nb += __popc(bb);
      }
    }
    if (lane == va) my_n = na;
    if (two && lane == vb) my_n = nb;
    __syncwarp();  // the next pair rewrites the clip coordinates
  }
  return true;
}

template <bool CHECKED>
__device__ __forceinline__ bool cull_views_dispatch(const Desc &d, const Grid &g, const float *Ms,
                                                    uint32_t views, const uint32_t *sw, uint8_t *sI,
                                                    float *px, uint32_t n_vtx, float4 *pxy,
                                                    float2 *pw, uint32_t *stri, uint32_t *surv,
                                                    uint32_t cap, uint32_t lane, float *out_pos,
                                                    uint32_t &my_n) {
#define MC_CULLV(B, R)                                                                           \
  cull_views_staged<CHECKED, B, R>(d, g, Ms, views, sw, sI, px, n_vtx, pxy, pw, stri, surv, cap, \
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
  const CullViewsLayout L =
      cull_views_layout(a.max_block_words, a.max_tris, a.max_verts, per_grab, n_views);
  uint8_t *base = smem + warp * L.bytes;
  uint8_t *sI = base + L.stream;
  float *px = reinterpret_cast<float *>(base + L.pos);
  float4 *pxy = reinterpret_cast<float4 *>(base + L.clip);
  float2 *pw = reinterpret_cast<float2 *>(base + L.clip_w);
  uint32_t *stri = reinterpret_cast<uint32_t *>(base + L.tri);
  uint32_t *surv = reinterpret_cast<uint32_t *>(base + L.surv);
  for (uint32_t i = threadIdx.x; i < 16 * n_views; i += blockDim.x) s_M[i] = view_projs[i];
  __syncthreads();
  if (threadIdx.x < n_views)
    s_eye[4 * threadIdx.x + 3] =
        cones && view_eye(s_M + 16 * threadIdx.x, s_eye + 4 * threadIdx.x) ? 1.0f : 0.0f;
  __syncthreads();
  const uint32_t all = (1u << n_views) - 1u;
  grab_loop<1>(a, per_grab, base, lane, scratch + kQueue, status,
            [&](uint32_t m0, const uint32_t *sdesc, uint32_t cnt) {
              return grab_outside_views(a, m0, sdesc, cnt, s_M, s_eye, n_views, cones, lane);
            },
            [&](const Desc &d, const uint32_t *sw, uint32_t j, uint32_t skipped, uint32_t) {
              const uint32_t views = ~(skipped >> (8 * j)) & all;
              if (!views) return;
              const Grid g = load_grid(a.grids + d.grid);
              uint32_t my_n = 0;
              if (!cull_views_dispatch<CHECKED>(d, g, s_M, views, sw, sI, px, L.n_vtx, pxy, pw,
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

namespace {
template <bool CHECKED, int MAX_THREADS>
cudaError_t launch_cull_views_t(const BatchArgs &a, const float *view_projs, uint32_t n_views,
                                const mc_cone *cones, uint32_t ctas, uint32_t warps,
                                uint32_t per_grab, uint32_t *tri_out, uint64_t tri_stride,
                                uint32_t *tri_counts, float *out_pos, uint32_t *status,
                                uint32_t *scratch, cudaStream_t s) {
  const uint32_t smem =
      cull_views_smem_per_warp(a.max_block_words, a.max_tris, a.max_verts, per_grab, n_views) * warps;
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

int max_ctas_per_sm_cull_views(uint32_t warps, uint32_t max_block_words, uint32_t max_tris,
                               uint32_t max_verts, uint32_t per_grab, uint32_t n_views) {
  const int smem =
      (int)(cull_views_smem_per_warp(max_block_words, max_tris, max_verts, per_grab, n_views) * warps);
  if (warps > 16) return 0;
  if (warps <= 4) {
    prepare(fn(decode_cull_views_kernel<true, 128>));
    return occupancy(fn(decode_cull_views_kernel<false, 128>), warps * 32, smem);
  }
  prepare(fn(decode_cull_views_kernel<true, 512>));
  return occupancy(fn(decode_cull_views_kernel<false, 512>), warps * 32, smem);
}

}  // namespace mcdev
