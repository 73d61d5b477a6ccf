// Warp-level GTS-Reuse meshlet decode (device side).
//
// One warp decodes one meshlet; lane l owns triangles k = l, l+32, ... and
// vertices v = l, l+32, ...  Everything follows the parallel formulation:
//
//   stream entry of triangle k (Sec. 4.3): with s_k = 2 + (number of
//     increment flags set among triangles 1..k) -- an inclusive add-scan,
//     done per 32-triangle word with __popc on the increment word itself --
//     the entry is s_k if the flag is set, else reuse[k + 1 - s_k]
//     (unpacked from w bits with a funnel shift).  I[0..2] = 0,1,2.
//   third vertex (Sec. 4.2): the last triangle j < k whose L/R flag differs
//     from flag k; old = I[j + 1] (I[0] if none).  The flags equal to flag k
//     form a run ending at k, which starts at the highest flag transition at
//     or below k (transition bits D_p = F_p xor F_(p-1), D_0 = 1), so
//     j + 1 = that position: one masked highest-bit scan of D in the current
//     32-triangle word, or a running "last transition" register when a fan
//     reaches back past the word.
//   triangle (Sec. 4.2, orientation by the flag): R -> (I[k+1], old, I[k+2]),
//     L -> (old, I[k+1], I[k+2]).
//   position (Sec. 4.4): g = L_c + q (q = b bits at (3v+c) b), then
//     x = fma((float)g, D, G) for g < 2^24, else
//     x = fma((float)(g & 0xFFF), D, fma((float)(g >> 12), 4096 D, G)).
// The common widths -- 8-bit reuse entries and 16-bit position fields -- are
// read with byte / halfword shared-memory loads instead of funnel shifts.
#pragma once

#include <cstdint>

#include "meshlet_codec.h"

namespace mcdev {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kSlackWords = 88;  // over-read margin after a staged payload
constexpr uint32_t kStreamBytes = 272;

struct Desc {
  uint32_t off16, vbase, tbase, V, T, w, b, grid, L[3];
  uint32_t aw;  // attribute words after the position words (0 without attribute channels)
};

__device__ __forceinline__ Desc unpack_desc(uint4 a, uint4 c) {
  Desc r;
  r.off16 = a.x;
  r.vbase = a.y;
  r.tbase = a.z;
  r.V = a.w & 0xFFFFu;
  r.T = a.w >> 16;
  r.w = c.x & 0xFFu;
  r.b = (c.x >> 8) & 0xFFu;
  r.grid = c.x >> 16;
  r.L[0] = c.y;
  r.L[1] = c.z;
  r.L[2] = c.w;
  r.aw = 0;
  return r;
}

__device__ __forceinline__ Desc load_desc(const mc_desc *d) {
  const uint4 *p = reinterpret_cast<const uint4 *>(d);
  return unpack_desc(__ldg(p), __ldg(p + 1));
}

struct Grid {
  float G[3], D[3];
};

__device__ __forceinline__ Grid load_grid(const mc_grid *g) {
  const uint4 *p = reinterpret_cast<const uint4 *>(g);
  uint4 a = __ldg(p), c = __ldg(p + 1);
  Grid r;
  r.G[0] = __uint_as_float(a.x);
  r.G[1] = __uint_as_float(a.y);
  r.G[2] = __uint_as_float(a.z);
  r.D[0] = __uint_as_float(c.x);
  r.D[1] = __uint_as_float(c.y);
  r.D[2] = __uint_as_float(c.z);
  return r;
}

// Connectivity encodings of a meshlet: GTS-Reuse with w-bit reuse entries
// (funnel-shift extraction) or with byte entries (w = 8: byte loads), and
// plain GTS (w = 0: every stream entry stored as a byte, Sec. 4.2).
enum : int { kReuseBits = 0, kReuseBytes = 1, kPlainGts = 2 };

// u32 words of the connectivity section: L/R words plus increment and reuse
// words (GTS-Reuse), or plus one byte per triangle k >= 1 (plain GTS).
__device__ __forceinline__ uint32_t conn_words(const Desc &d) {
  const uint32_t nw = (d.T + 31) >> 5;
  return d.w ? 2 * nw + ((d.T + 2 - d.V) * d.w + 31) / 32 : nw + (d.T + 2) / 4;
}

// Payload block size in u32 words (unpadded) of a meshlet.
__device__ __forceinline__ uint32_t block_words(const Desc &d) {
  return conn_words(d) + (3 * d.V * d.b + 31) / 32 + d.aw;
}

struct BatchArgs {
  const mc_desc *desc;
  const uint8_t *payload;
  const mc_grid *grids;
  uint32_t n_meshlets, n_grids;
  uint64_t payload_bytes, total_tris, total_verts;
  uint32_t max_block_words;  // capacity of one meshlet's shared-memory slot
  uint32_t max_tris;         // largest T' of the batch (sizes per-warp output buffers)
  uint32_t max_verts;        // largest V of the batch (sizes per-warp vertex buffers)
  uint32_t n_attr, attr_bits;  // attribute channels after the positions (0 = none)
  const mc_attr_desc *attr_desc;
  const mc_attr_grid *attr_grids;
  uint32_t n_attr_grids;
  uint32_t wait_cycles;  // limit of a wait on another warp (look-back), 0 = the default
};

// The attribute words of a meshlet follow its position words.
__device__ __forceinline__ Desc with_attrs(Desc d, const BatchArgs &a) {
  d.aw = (a.n_attr * d.V * a.attr_bits + 31) / 32;
  return d;
}

// Largest b-bit field value, 2^b - 1 (b <= 32).
__device__ __forceinline__ uint32_t field_max(uint32_t b) {
  return b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
}

// Header sanity (all builds): a descriptor that passes cannot make the decode
// read or write outside its buffers, and its whole quantisation box
// [L, L + 2^b - 1] is representable as 32-bit grid coordinates (the encoder's
// rule), so no g = L + q and no box corner wraps around.
__device__ __forceinline__ bool header_ok(const Desc &d, const BatchArgs &a) {
  // evaluated without short-circuit branches (all terms are cheap)
  const bool shape = (d.V - 3u <= 253u) & (d.T - 1u <= 255u) & (d.V <= d.T + 2) &
                     (d.w <= 8u) & (d.b - 1u <= 31u) & (d.grid < a.n_grids) &
                     (d.T <= a.max_tris) & (d.V <= a.max_verts);
  const uint32_t top = ~field_max(d.b);  // largest L with L + 2^b - 1 < 2^32
  const bool box = (d.L[0] <= top) & (d.L[1] <= top) & (d.L[2] <= top);
  const uint32_t padded = (block_words(d) + 3) & ~3u;
  return shape & box & (padded <= a.max_block_words) &
         (16ull * d.off16 + 4ull * padded <= a.payload_bytes) &
         ((uint64_t)d.tbase + d.T <= a.total_tris) & ((uint64_t)d.vbase + d.V <= a.total_verts);
}

__device__ __forceinline__ uint32_t extract(const uint32_t *w, uint32_t bit, uint32_t nbits) {
  uint32_t i = bit >> 5;
  uint32_t v = __funnelshift_r(w[i], w[i + 1], bit & 31u);
  return nbits >= 32 ? v : (v & ((1u << nbits) - 1u));
}

// Grid coordinate -> FP32 (the evaluation order of Sec. 4.4 fixed above).
__device__ __forceinline__ float dequant_small(uint32_t g, float G, float D) {
  return __fmaf_rn(__uint2float_rn(g), D, G);
}
__device__ __forceinline__ float dequant(uint32_t g, float G, float D) {
  if (g < (1u << 24)) return dequant_small(g, G, D);
  float hi = __uint2float_rn(g >> 12);
  float lo = __uint2float_rn(g & 0xFFFu);
  return __fmaf_rn(lo, D, __fmaf_rn(hi, __fmul_rn(D, 4096.0f), G));
}

__device__ __forceinline__ void set_status(uint32_t *st, uint32_t code) {
  if (st) atomicOr(st, 1u << code);
}

// Copies one meshlet's payload block into shared memory (16-byte vectors).
__device__ __forceinline__ void stage_payload(const Desc &d, const uint8_t *payload,
                                              uint32_t *sw, uint32_t lane) {
  const uint4 *src = reinterpret_cast<const uint4 *>(payload) + d.off16;
  uint4 *dst = reinterpret_cast<uint4 *>(sw);
  uint32_t n4 = (block_words(d) + 3) >> 2;
  for (uint32_t i = lane; i < n4; i += 32) dst[i] = __ldg(src + i);
}

// 32-bit shared-window accessors (explicit LDS/STS addressing).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts_u8(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// position of the highest set bit, 0xFFFFFFFF for 0
__device__ __forceinline__ uint32_t msb(uint32_t x) {
  uint32_t r;
  asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x));
  return r;
}

// Predicated stores (no divergent branches in the strip passes).
__device__ __forceinline__ void sts_u8_if(uint32_t a, uint32_t v, bool p) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.shared.u8 [%0], %1;\n}" ::"r"(a),
               "r"(v), "r"((uint32_t)p)
               : "memory");
}
__device__ __forceinline__ void stg3_u8_if(uint8_t *g, uint32_t x, uint32_t y, uint32_t z, bool p) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n @q st.global.u8 [%0], %1;\n"
      " @q st.global.u8 [%0+1], %2;\n @q st.global.u8 [%0+2], %3;\n}" ::"l"(g),
      "r"(x), "r"(y), "r"(z), "r"((uint32_t)p)
      : "memory");
}
__device__ __forceinline__ void stg3_u32_if(uint32_t *g, uint32_t x, uint32_t y, uint32_t z, bool p) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n @q st.global.u32 [%0], %1;\n"
      " @q st.global.u32 [%0+4], %2;\n @q st.global.u32 [%0+8], %3;\n}" ::"l"(g),
      "r"(x), "r"(y), "r"(z), "r"((uint32_t)p)
      : "memory");
}

// Stream-level consistency checks of the checked build: bit 0 of both flag
// words clear, no flag bit past T', and V = 3 + (number of increment flags);
// plain GTS: every stored entry is a vertex already seen or the next new
// one, and V vertices are introduced in all (a short sequential scan, run by
// every lane alike).
__device__ __forceinline__ bool stream_header_ok(const Desc &d, const uint32_t *sw) {
  const uint32_t nw = (d.T + 31) >> 5;
  if (d.w == 0) {
    const uint32_t tail = d.T & 31u;
    bool ok = !(sw[0] & 1u) && !(tail && (sw[nw - 1] >> tail));
    const uint8_t *e = reinterpret_cast<const uint8_t *>(sw + nw);
    uint32_t next = 3;
    for (uint32_t k = 1; k < d.T; k++) {
      const uint32_t x = e[k - 1];
      ok = ok & (x <= next) & (x < d.V);
      next += x == next ? 1u : 0u;
    }
    return ok && next == d.V;
  }
  uint32_t incs = 0;
  for (uint32_t i = 0; i < nw; i++) incs += __popc(sw[nw + i]);
  const uint32_t tail = d.T & 31u;
  return incs + 3 == d.V && !(sw[0] & 1u) && !(sw[nw] & 1u) &&
         !(tail && ((sw[nw - 1] >> tail) | (sw[2 * nw - 1] >> tail)));
}

// Walks the meshlet's triangles 32 at a time, calling
//   emit(k, a, b, c, live)
// on every lane (live = k < T') with triangle k = (a, b, c).  Per 32-triangle
// word: strip entries from the increment-word add-scan (triangle 0 folded in
// as "new" with the scan seeded at 1) or the reuse buffer, stored to sI;
// I[k+1] from the neighbouring lane.  The third vertex I[j+1] uses the flag
// transitions D_p = [F_p != F_(p-1)] (D_0 = 1): the run of equal flags that
// ends at k starts at r = the highest set D bit at or below k, so the last
// differing flag is j = r - 1 and old = I[r] -- one masked bit scan, or a
// running "last transition" register when the run starts in an earlier word.
// CHECKED: returns false (warp-uniform) if a reuse entry names a vertex not
// yet seen.
template <bool CHECKED, int RM, class Emit>
__device__ __forceinline__ bool walk_triangles(const Desc &d, const uint32_t *sw, uint8_t *sI,
                                               uint32_t lane, Emit &&emit) {
  const uint32_t nw = (d.T + 31) >> 5;
  const uint32_t a_sw = smem_addr(sw);
  const uint32_t a_rb = a_sw + 8 * nw;
  const uint32_t a_eb = a_sw + 4 * nw;  // plain GTS: byte k-1 = entry of triangle k
  const uint32_t a_sI = smem_addr(sI);
  if (lane < 2) sts_u8(a_sI + lane, lane);
  const uint32_t le = (2u << lane) - 1u;
  uint32_t base = 1, carry = 1, cf = 1, lastT = 0;
  bool bad = false;
  uint32_t k = lane;
  for (uint32_t i = 0; i < nw; i++, k += 32) {
    const uint32_t f = lds_u32(a_sw + 4 * i);
    uint32_t n;
    if (RM == kPlainGts) {
      const uint32_t e = lds_u8(a_eb + (k ? k - 1 : 0u));
      n = k ? e : 2u;
    } else {
      const uint32_t inc = lds_u32(a_sw + 4 * (nw + i)) | (i == 0 ? 1u : 0u);
      const uint32_t s = base + __popc(inc & le);
      const bool is_new = (inc & (1u << lane)) != 0;
      const uint32_t slot = is_new ? 0u : k + 1 - s;
      const uint32_t r = RM == kReuseBytes ? lds_u8(a_rb + slot) : extract(sw + 2 * nw, slot * d.w, d.w);
      n = is_new ? s : r;
      if (CHECKED && k < d.T && !is_new && r > s) bad = true;
      base += __popc(inc);
    }
    const bool live = k < d.T;
    sts_u8_if(a_sI + k + 2, n, live);
    uint32_t prev = __shfl_up_sync(kFull, n, 1);
    if (lane == 0) prev = carry;
    carry = __shfl_sync(kFull, n, 31);
    const uint32_t D = f ^ ((f << 1) | cf);
    cf = f >> 31;
    __syncwarp();
    const uint32_t m = msb(D & le);
    const uint32_t run = m == 0xFFFFFFFFu ? lastT : 32 * i + m;
    const uint32_t old = lds_u8(a_sI + run);
    const bool fk = (f >> lane) & 1u;
    emit(k, fk ? prev : old, fk ? old : prev, n, live);
    if (D) lastT = 32 * i + msb(D);
  }
  if (CHECKED) bad = __any_sync(kFull, bad);
  __syncwarp();
  return !bad;
}

// Position fields of vertex v (q for x, y, z).
template <bool B16>
__device__ __forceinline__ void vertex_q(const uint32_t *pw, uint32_t v, uint32_t b, uint32_t q[3]) {
  if (B16) {
    const uint16_t *p = reinterpret_cast<const uint16_t *>(pw) + 3 * v;
    q[0] = p[0];
    q[1] = p[1];
    q[2] = p[2];
  } else {
    const uint32_t bit = 3 * v * b;
    q[0] = extract(pw, bit, b);
    q[1] = extract(pw, bit + b, b);
    q[2] = extract(pw, bit + 2 * b, b);
  }
}
// vertex_q for b <= 21: the vertex's 3b bits read as one 64-bit window of
// three words (two funnel shifts) instead of three two-word extractions.
__device__ __forceinline__ void vertex_q_window(const uint32_t *pw, uint32_t v, uint32_t b,
                                                uint32_t q[3]) {
  const uint32_t bit = 3 * v * b;
  const uint32_t i = bit >> 5, sh = bit & 31u;
  const uint32_t lo = __funnelshift_r(pw[i], pw[i + 1], sh);
  const uint32_t hi = __funnelshift_r(pw[i + 1], pw[i + 2], sh);
  const unsigned long long win = ((unsigned long long)hi << 32) | lo;
  const uint32_t m = (1u << b) - 1u;
  q[0] = lo & m;
  q[1] = (uint32_t)(win >> b) & m;
  q[2] = (uint32_t)(win >> (2 * b)) & m;
}

// true when every grid coordinate of the meshlet is below 2^24
__device__ __forceinline__ bool small_coords(const Desc &d) {
  const uint32_t lim = (1u << 24) - (1u << min(d.b, 24u));  // L + 2^b - 1 < 2^24
  return (d.b <= 24) & (d.L[0] <= lim) & (d.L[1] <= lim) & (d.L[2] <= lim);
}

__device__ __forceinline__ void stg3_f32_if(float *g, float x, float y, float z, bool p) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n @q st.global.f32 [%0], %1;\n"
      " @q st.global.f32 [%0+4], %2;\n @q st.global.f32 [%0+8], %3;\n}" ::"l"(g),
      "f"(x), "f"(y), "f"(z), "r"((uint32_t)p)
      : "memory");
}

__device__ __forceinline__ void stg4_f32_if(float *g, float x, float y, float z, float w, bool p) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %5, 0;\n @q st.global.v4.f32 [%0], {%1, %2, %3, %4};\n}" ::"l"(g),
      "f"(x), "f"(y), "f"(z), "f"(w), "r"((uint32_t)p)
      : "memory");
}

// Full vertices of one staged meshlet: 8 FP32 per vertex -- x, y, z, then
// the n_attr attribute channels (q at bit (n_attr v + c) attr_bits of the
// attribute words that follow the position words; La_c + q dequantised with
// the channel's G_c and D_c like a position), then zeros -- written as two
// 16-byte stores.  sa holds La[0..4], G[5..9] and D[10..14] (float bits) of
// the meshlet in shared memory (a 64-byte slot).
template <bool B16>
__device__ __forceinline__ void vertex_stage_full(const Desc &d, const Grid &g, const uint32_t *sw,
                                                  const uint32_t *sa, uint32_t n_attr,
                                                  uint32_t attr_bits, uint32_t lane,
                                                  float *out_vertex) {
  const uint32_t *pw = sw + conn_words(d);
  const uint32_t *aw = pw + (3 * d.V * d.b + 31) / 32;
  float *ov = out_vertex + 8ull * (d.vbase + lane);
  const uint32_t vpasses = (d.V + 31) >> 5;
  uint32_t v = lane;
  for (uint32_t i = 0; i < vpasses; i++, v += 32, ov += 256) {
    const uint32_t vv = min(v, d.V - 1);  // idle lanes recompute the last vertex
    uint32_t q[3];
    vertex_q<B16>(pw, vv, d.b, q);
    float a[5];
#pragma unroll
    for (uint32_t c = 0; c < 5; c++) {
      a[c] = 0.0f;
      if (c < n_attr) {
        const uint32_t qa = extract(aw, (n_attr * vv + c) * attr_bits, attr_bits);
        a[c] = dequant(sa[c] + qa, __uint_as_float(sa[5 + c]), __uint_as_float(sa[10 + c]));
      }
    }
    const bool live = v < d.V;
    stg4_f32_if(ov, dequant(d.L[0] + q[0], g.G[0], g.D[0]), dequant(d.L[1] + q[1], g.G[1], g.D[1]),
                dequant(d.L[2] + q[2], g.G[2], g.D[2]), a[0], live);
    stg4_f32_if(ov + 4, a[1], a[2], a[3], a[4], live);
  }
  __syncwarp();
}

// Positions of one staged meshlet by the general path: q from vertex_q,
// dequantised with the 2^24 split where needed (SMALL: every coordinate of
// the meshlet is below 2^24, so the split never applies).
template <bool B16, bool SMALL>
__device__ __forceinline__ void positions_general(const Desc &d, const Grid &g, const uint32_t *pw,
                                                  float *op, uint32_t lane) {
  const uint32_t vpasses = (d.V + 31) >> 5;
  uint32_t v = lane;
  for (uint32_t i = 0; i < vpasses; i++, v += 32, op += 96) {
    uint32_t q[3];
    if (!B16 && SMALL)  // SMALL implies b <= 24; the window takes b <= 21
      d.b <= 21 ? vertex_q_window(pw, min(v, d.V - 1), d.b, q) : vertex_q<false>(pw, min(v, d.V - 1), d.b, q);
    else
      vertex_q<B16>(pw, min(v, d.V - 1), d.b, q);  // idle lanes re-read the last vertex
    if (SMALL)
      stg3_f32_if(op, dequant_small(d.L[0] + q[0], g.G[0], g.D[0]),
                  dequant_small(d.L[1] + q[1], g.G[1], g.D[1]),
                  dequant_small(d.L[2] + q[2], g.G[2], g.D[2]), v < d.V);
    else
      stg3_f32_if(op, dequant(d.L[0] + q[0], g.G[0], g.D[0]), dequant(d.L[1] + q[1], g.G[1], g.D[1]),
                  dequant(d.L[2] + q[2], g.G[2], g.D[2]), v < d.V);
  }
}

// Full decode of one staged meshlet into the batch outputs: the strip walk
// of walk_triangles (same arithmetic) written out flat, with predicated
// stores and per-lane output pointers advanced by one word of triangles per
// pass.  The walk does not depend on the position width, so one build per
// reuse form serves every b (the vertex stage branches on b = 16).
template <bool CHECKED, int RM, bool VTX>
__device__ __forceinline__ bool decode_staged(const Desc &d, const Grid &g, const uint32_t *sw,
                                              uint8_t *sI, uint32_t lane, uint8_t *out_local,
                                              uint32_t *out_global, float *out_pos,
                                              const uint32_t *sa, uint32_t n_attr,
                                              uint32_t attr_bits) {
  if (CHECKED && !stream_header_ok(d, sw)) return false;
  const uint32_t nw = (d.T + 31) >> 5;
  const uint32_t a_sw = smem_addr(sw);
  const uint32_t a_rb = a_sw + 8 * nw;  // reuse section (bytes)
  const uint32_t a_eb = a_sw + 4 * nw;  // plain GTS entries (byte k-1 = triangle k)
  const uint32_t a_sI = smem_addr(sI);
  if (lane < 2) sts_u8(a_sI + lane, lane);  // I[0], I[1]; I[2] is triangle 0's entry
  const uint32_t le = (2u << lane) - 1u;
  uint8_t *pl = out_local ? out_local + 3ull * (d.tbase + lane) : nullptr;
  uint32_t *pg = out_global ? out_global + 3ull * (d.tbase + lane) : nullptr;
  const bool want_l = pl != nullptr, want_g = pg != nullptr;
  const uint32_t vb = d.vbase;
  uint32_t base = 1, carry = 1, cf = 1, lastT = 0;
  bool bad = false;
  uint32_t k = lane;
  for (uint32_t i = 0; i < nw; i++, k += 32) {
    const uint32_t f = lds_u32(a_sw + 4 * i);
    uint32_t n;
    if (RM == kPlainGts) {
      const uint32_t e = lds_u8(a_eb + (k ? k - 1 : 0u));
      n = k ? e : 2u;
    } else {
      const uint32_t inc = lds_u32(a_sw + 4 * (nw + i)) | (i == 0 ? 1u : 0u);
      const uint32_t s = base + __popc(inc & le);
      const bool is_new = (inc & (1u << lane)) != 0;
      const uint32_t slot = is_new ? 0u : k + 1 - s;
      const uint32_t r = RM == kReuseBytes ? lds_u8(a_rb + slot) : extract(sw + 2 * nw, slot * d.w, d.w);
      n = is_new ? s : r;
      if (CHECKED && k < d.T && !is_new && r > s) bad = true;  // entries seen so far: 0..s
      base += __popc(inc);
    }
    const bool live = k < d.T;
    sts_u8_if(a_sI + k + 2, n, live);
    uint32_t prev = __shfl_up_sync(kFull, n, 1);
    if (lane == 0) prev = carry;
    carry = __shfl_sync(kFull, n, 31);
    const uint32_t D = f ^ ((f << 1) | cf);  // flag transitions (D_0 = 1)
    cf = f >> 31;
    __syncwarp();
    const uint32_t m = msb(D & le);
    const uint32_t run = m == 0xFFFFFFFFu ? lastT : 32 * i + m;  // start of k's flag run
    const uint32_t old = lds_u8(a_sI + run);                    // I[j+1], j = run - 1
    const bool fk = (f >> lane) & 1u;
    const uint32_t ta = fk ? prev : old, tb = fk ? old : prev;
    stg3_u8_if(pl, ta, tb, n, live && want_l);
    stg3_u32_if(pg, vb + ta, vb + tb, vb + n, live && want_g);
    pl += 96;
    pg += 96;
    if (D) lastT = 32 * i + msb(D);
  }
  if (CHECKED && __any_sync(kFull, bad)) return false;
  if (VTX) {
    if (d.b == 16)
      vertex_stage_full<true>(d, g, sw, sa, n_attr, attr_bits, lane, out_pos);
    else
      vertex_stage_full<false>(d, g, sw, sa, n_attr, attr_bits, lane, out_pos);
    return true;
  }
  // positions
  const uint32_t *pw = sw + conn_words(d);
  float *op = out_pos + 3ull * (d.vbase + lane);
  if (d.b == 16 && small_coords(d)) {
    const uint32_t vpasses = (d.V + 31) >> 5;
    uint32_t a = smem_addr(pw) + 6 * lane;
    uint32_t v = lane;
    for (uint32_t i = 0; i < vpasses; i++, v += 32, a += 192, op += 96) {
      const float x = dequant_small(d.L[0] + lds_u16(a), g.G[0], g.D[0]);
      const float y = dequant_small(d.L[1] + lds_u16(a + 2), g.G[1], g.D[1]);
      const float z = dequant_small(d.L[2] + lds_u16(a + 4), g.G[2], g.D[2]);
      stg3_f32_if(op, x, y, z, v < d.V);
    }
  } else if (small_coords(d)) {  // b != 16
    positions_general<false, true>(d, g, pw, op, lane);
  } else if (d.b == 16) {
    positions_general<true, false>(d, g, pw, op, lane);
  } else {
    positions_general<false, false>(d, g, pw, op, lane);
  }
  __syncwarp();
  return true;
}

// Two meshlets per warp: half h = lane / 16 decodes its own staged meshlet
// (d, sw; live = false for a half without one) with lanes hl = lane % 16
// owning triangles k = hl, hl + 16, ... and vertices v = hl, hl + 16, ...
// The arithmetic is decode_staged's, on 16-triangle halves of the 32-bit
// flag words: s_k from the add-scan of the increment bits up to k, the
// third vertex from the highest flag transition at or below k (or the
// carried last transition), orientation by the flag.  Shuffles stay within a
// half (width 16); both halves run max(passes) iterations, a half past its
// own triangles idle (its loads stay inside the staged block and its slack).
// sI points at this half's strip-stream buffer.  Returns false when this
// half's meshlet is corrupt (CHECKED only).
template <bool CHECKED, bool B16, int RM>
__device__ __forceinline__ bool decode_pair(const Desc &d, bool live_half, const Grid &g,
                                            const uint32_t *sw, uint8_t *sI, uint32_t lane,
                                            uint8_t *out_local, uint32_t *out_global,
                                            float *out_pos) {
  bool ok = live_half;
  if (CHECKED && ok) ok = stream_header_ok(d, sw);
  const uint32_t hl = lane & 15u;
  const uint32_t T = ok ? d.T : 0u, V = ok ? d.V : 0u;
  const uint32_t np = (T + 15) >> 4, vp = (V + 15) >> 4;
  const uint32_t npass = max(np, __shfl_xor_sync(kFull, np, 16));
  const uint32_t nvpass = max(vp, __shfl_xor_sync(kFull, vp, 16));
  const uint32_t nw = (d.T + 31) >> 5;
  const uint32_t a_sw = smem_addr(sw);
  const uint32_t a_rb = a_sw + 8 * nw;
  const uint32_t a_eb = a_sw + 4 * nw;
  const uint32_t a_sI = smem_addr(sI);
  if (hl < 2) sts_u8(a_sI + hl, hl);
  const uint32_t le = (2u << hl) - 1u;
  uint8_t *pl = out_local ? out_local + 3ull * (d.tbase + hl) : nullptr;
  uint32_t *pg = out_global ? out_global + 3ull * (d.tbase + hl) : nullptr;
  const bool want_l = pl != nullptr, want_g = pg != nullptr;
  const uint32_t vb = d.vbase;
  uint32_t base = 1, carry = 1, cf = 1, lastT = 0;
  bool bad = false;
  uint32_t k = hl;
  for (uint32_t p = 0; p < npass; p++, k += 16) {
    const uint32_t wa = a_sw + 4 * (p >> 1), sh = (p & 1u) << 4;
    const uint32_t f = (lds_u32(wa) >> sh) & 0xFFFFu;
    uint32_t n;
    if (RM == kPlainGts) {
      const uint32_t e = lds_u8(a_eb + (k ? k - 1 : 0u));
      n = k ? e : 2u;
    } else {
      const uint32_t inc = ((lds_u32(wa + 4 * nw) >> sh) & 0xFFFFu) | (p == 0 ? 1u : 0u);
      const uint32_t s = base + __popc(inc & le);
      const bool is_new = (inc >> hl) & 1u;
      const uint32_t slot = is_new ? 0u : k + 1 - s;
      const uint32_t r = RM == kReuseBytes ? lds_u8(a_rb + slot) : extract(sw + 2 * nw, slot * d.w, d.w);
      n = is_new ? s : r;
      if (CHECKED && k < T && !is_new && r > s) bad = true;
      base += __popc(inc);
    }
    const bool live = k < T;
    sts_u8_if(a_sI + k + 2, n, live);
    uint32_t prev = __shfl_up_sync(kFull, n, 1, 16);
    if (hl == 0) prev = carry;
    carry = __shfl_sync(kFull, n, 15, 16);
    const uint32_t D = (f ^ ((f << 1) | cf)) & 0xFFFFu;  // flag transitions of this half word
    cf = f >> 15;
    __syncwarp();
    const uint32_t m = msb(D & le);
    const uint32_t run = m == 0xFFFFFFFFu ? lastT : 16 * p + m;
    const uint32_t old = lds_u8(a_sI + run);
    const bool fk = (f >> hl) & 1u;
    const uint32_t ta = fk ? prev : old, tb = fk ? old : prev;
    stg3_u8_if(pl, ta, tb, n, live && want_l);
    stg3_u32_if(pg, vb + ta, vb + tb, vb + n, live && want_g);
    pl += 48;
    pg += 48;
    if (D) lastT = 16 * p + msb(D);
  }
  if (CHECKED) ok = ok && !bad;
  const uint32_t *pw = sw + conn_words(d);
  float *op = out_pos + 3ull * (d.vbase + hl);
  if (B16 && small_coords(d)) {
    uint32_t a = smem_addr(pw) + 6 * hl;
    uint32_t v = hl;
    for (uint32_t i = 0; i < nvpass; i++, v += 16, a += 96, op += 48) {
      const bool lv = v < V;
      const uint32_t aa = lv ? a : smem_addr(pw);
      const float x = dequant_small(d.L[0] + lds_u16(aa), g.G[0], g.D[0]);
      const float y = dequant_small(d.L[1] + lds_u16(aa + 2), g.G[1], g.D[1]);
      const float z = dequant_small(d.L[2] + lds_u16(aa + 4), g.G[2], g.D[2]);
      stg3_f32_if(op, x, y, z, lv);
    }
  } else {
    uint32_t v = hl;
    for (uint32_t i = 0; i < nvpass; i++, v += 16, op += 48) {
      uint32_t q[3];
      vertex_q<B16>(pw, v < V ? v : 0u, d.b, q);  // idle lanes re-read vertex 0
      stg3_f32_if(op, dequant(d.L[0] + q[0], g.G[0], g.D[0]), dequant(d.L[1] + q[1], g.G[1], g.D[1]),
                  dequant(d.L[2] + q[2], g.G[2], g.D[2]), v < V);
    }
  }
  __syncwarp();
  return ok || !live_half;
}

// Pair dispatch: both halves take the connectivity / position path of their
// meshlets when these agree; otherwise the generic one (funnel-shift reads
// serve every width), or, when one half holds plain GTS and the other
// GTS-Reuse, each path in turn with the other half idle.  Returns this
// half's status as decode_pair.
template <bool CHECKED>
__device__ __forceinline__ bool decode_pair_dispatch(const Desc &d, bool live_half, const Grid &g,
                                                     const uint32_t *sw, uint8_t *sI, uint32_t lane,
                                                     uint8_t *out_local, uint32_t *out_global,
                                                     float *out_pos) {
  // 0 idle, 1 plain GTS, 2 byte reuse entries + 16-bit positions, 3 any other
  const uint32_t mode = !live_half ? 0u : d.w == 0 ? 1u : (d.b == 16 && d.w == 8) ? 2u : 3u;
  const uint32_t other = __shfl_xor_sync(kFull, mode, 16);
#define MC_PAIR(B, R, LIVE) \
  decode_pair<CHECKED, B, R>(d, LIVE, g, sw, sI, lane, out_local, out_global, out_pos)
  if (mode == other || mode == 0 || other == 0) {
    const uint32_t m = mode | other;  // the one live mode (or both alike)
    if (m == 2) return MC_PAIR(true, kReuseBytes, live_half);
    if (m == 1) return MC_PAIR(false, kPlainGts, live_half);
    return MC_PAIR(false, kReuseBits, live_half);
  }
  if (mode != 1 && other != 1) return MC_PAIR(false, kReuseBits, live_half);
  // plain GTS beside GTS-Reuse: one round each, the other half idle
  const bool a = MC_PAIR(false, kPlainGts, live_half && mode == 1);
  const bool b = MC_PAIR(false, kReuseBits, live_half && mode != 1);
  return mode == 1 ? a : b;
#undef MC_PAIR
}

// out_pos: positions (3 FP32 per vertex) or, VTX, full vertices (8 FP32 per
// vertex, sa / n_attr / attr_bits as for vertex_stage_full).
template <bool CHECKED, bool VTX = false>
__device__ __forceinline__ bool decode_dispatch(const Desc &d, const Grid &g, const uint32_t *sw,
                                                uint8_t *sI, uint32_t lane, uint8_t *out_local,
                                                uint32_t *out_global, float *out_pos,
                                                const uint32_t *sa = nullptr, uint32_t n_attr = 0,
                                                uint32_t attr_bits = 0) {
#define MC_DEC(R) \
  decode_staged<CHECKED, R, VTX>(d, g, sw, sI, lane, out_local, out_global, out_pos, sa, n_attr, attr_bits)
  if (d.w == 8) return MC_DEC(kReuseBytes);
  if (d.w == 0) return MC_DEC(kPlainGts);
  return MC_DEC(kReuseBits);
#undef MC_DEC
}

}  // namespace mcdev
