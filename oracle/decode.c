/*
 * Oracle: sequential GTS-Reuse decode, dequantisation and culling.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Decode walks the strip one triangle at a time exactly as Sec. 2 defines it:
 * the state is the current triangle (a,b,c) as entered through (a,b); the
 * next triangle with new stream entry x is (c,b,x) if its L/R flag says
 * "right" and (a,c,x) if it says "left".  The stream entry x is the next
 * unused vertex number when the increment flag is set and the next reuse
 * buffer entry otherwise (Sec. 4.3).  The implicit first triangle is (0,1,2).
 * This is the serial definition; the parallel closed form the GPU evaluates
 * (Sec. 4.2 bit scan, Sec. 4.3 add-scan) is not used here.
 *
 * Dequantisation (Sec. 4.4): integer add g = L_c + q, then the grid
 * coordinate maps back to float as G_c + g * Delta_c.  In FP32 this oracle
 * fixes the evaluation order
 *     g < 2^24:  x = fmaf((float)g, Delta, G)           (one rounding)
 *     otherwise: x = fmaf((float)(g & 0xFFF), Delta,
 *                         fmaf((float)(g >> 12), Delta * 4096, G))
 * (every integer-to-float conversion and the power-of-two scale are exact,
 * and x depends on g alone, so shared boundary vertices stay crack-free);
 * the FP64 reference is G + g * Delta in double.
 *
 * Culling: a meshlet is dropped when all 8 corners of its quantisation box
 * [L_c, L_c + 2^b - 1] lie outside one clip plane (-w <= x,y,z <= w); a
 * triangle is dropped when two of its indices coincide, or when all three
 * clip w are positive and the determinant of the (x, y, w) rows is not
 * positive (back-facing for counter-clockwise front faces).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static uint32_t get_u16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static float get_f32(const uint8_t *p) {
  uint32_t u = get_u32(p);
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* nbits (<= 32) starting at bit offset `bit` of the LSB-first u32 word array */
static uint32_t get_bits(const uint8_t *words, uint64_t bit, uint32_t nbits) {
  uint64_t v = 0;
  for (uint32_t i = 0; i < nbits; i++) {
    uint64_t p = bit + i;
    uint32_t word = get_u32(words + 4 * (p >> 5));
    v |= (uint64_t)((word >> (p & 31u)) & 1u) << i;
  }
  return (uint32_t)v;
}

float orc_dequant32(uint32_t g, float G, float D) {
  if (g < (1u << 24)) return fmaf((float)g, D, G); /* (float)g is exact */
  float hi = (float)(g >> 12);
  float lo = (float)(g & 0xFFFu);
  float D4096 = D * 4096.0f;
  return fmaf(lo, D, fmaf(hi, D4096, G));
}

typedef struct {
  uint32_t off16, vbase, tbase, V, tp, w, b, grid, L[3];
} desc_t;

static void parse_desc(const uint8_t *d, desc_t *x) {
  x->off16 = get_u32(d);
  x->vbase = get_u32(d + 4);
  x->tbase = get_u32(d + 8);
  x->V = get_u16(d + 12);
  x->tp = get_u16(d + 14);
  x->w = d[16];
  x->b = d[17];
  x->grid = get_u16(d + 18);
  for (int c = 0; c < 3; c++) x->L[c] = get_u32(d + 20 + 4 * c);
}

int orc_decode_meshlet(const uint8_t *desc32, const uint8_t *payload,
                       uint64_t payload_bytes, const uint8_t *grids,
                       uint32_t n_grids, uint8_t *local, float *pos,
                       double *pos64) {
  desc_t d;
  parse_desc(desc32, &d);
  if (d.V < 3 || d.V > 256 || d.tp < 1 || d.tp > 256 || d.w > 8 || d.b < 1 ||
      d.b > 32 || d.grid >= n_grids || d.V > d.tp + 2)
    return ORC_ERR_CORRUPT;
  /* the meshlet's quantisation box [L, L + 2^b - 1] must be representable as
   * 32-bit grid coordinates (Sec. 4.4: the decoder adds q to L as integers);
   * the encoder never writes a minimum closer than 2^b - 1 to 2^32 */
  for (int ch = 0; ch < 3; ch++)
    if ((uint64_t)d.L[ch] + ((1ull << d.b) - 1) > 0xFFFFFFFFull) return ORC_ERR_CORRUPT;
  const int gts = d.w == 0; /* plain GTS: one stored 8-bit entry per triangle */
  uint32_t R = d.tp + 2 - d.V;
  uint64_t nw = (d.tp + 31) / 32;
  uint64_t cw = gts ? nw + ((uint64_t)d.tp - 1 + 3) / 4 : 2 * nw + ((uint64_t)R * d.w + 31) / 32;
  uint64_t pw = (3 * (uint64_t)d.V * d.b + 31) / 32;
  uint64_t start = 16 * (uint64_t)d.off16;
  if (start + 4 * (cw + pw) > payload_bytes) return ORC_ERR_CORRUPT;
  const uint8_t *F = payload + start;
  const uint8_t *INC = F + 4 * nw; /* plain GTS: the entry bytes */
  const uint8_t *RB = INC + 4 * nw;
  const uint8_t *PB = F + 4 * cw;
  if (get_bits(F, 0, 1) || (!gts && get_bits(INC, 0, 1))) return ORC_ERR_CORRUPT;

  /* strip walk */
  uint32_t a = 0, b = 1, c = 2, next_new = 3, slot = 0;
  if (local) { local[0] = 0; local[1] = 1; local[2] = 2; }
  for (uint32_t k = 1; k < d.tp; k++) {
    uint32_t x;
    if (gts) {
      x = get_bits(INC, 8 * (uint64_t)(k - 1), 8);
      if (x > next_new || x >= d.V) return ORC_ERR_CORRUPT;
      if (x == next_new) next_new++;
    } else if (get_bits(INC, k, 1)) {
      if (next_new >= d.V) return ORC_ERR_CORRUPT;
      x = next_new++;
    } else {
      if (slot >= R) return ORC_ERR_CORRUPT;
      x = get_bits(RB, (uint64_t)slot * d.w, d.w);
      slot++;
      if (x >= next_new) return ORC_ERR_CORRUPT;
    }
    if (get_bits(F, k, 1)) { /* right: (c, b, x) */
      uint32_t na = c;
      a = na; c = x;
    } else { /* left: (a, c, x) */
      b = c; c = x;
    }
    if (local) {
      local[3 * k] = (uint8_t)a;
      local[3 * k + 1] = (uint8_t)b;
      local[3 * k + 2] = (uint8_t)c;
    }
  }
  if (next_new != d.V || (!gts && slot != R)) return ORC_ERR_CORRUPT;

  /* positions */
  const uint8_t *g = grids + 32 * (size_t)d.grid;
  if (get_u32(g + 12) != d.b) return ORC_ERR_CORRUPT;
  for (uint32_t v = 0; v < d.V; v++)
    for (int ch = 0; ch < 3; ch++) {
      uint32_t q = get_bits(PB, (3 * (uint64_t)v + ch) * d.b, d.b);
      uint64_t gg = (uint64_t)d.L[ch] + q;
      if (gg > 0xFFFFFFFFull) return ORC_ERR_CORRUPT;
      float G = get_f32(g + 4 * ch), D = get_f32(g + 16 + 4 * ch);
      if (pos) pos[3 * v + ch] = orc_dequant32((uint32_t)gg, G, D);
      if (pos64) pos64[3 * v + ch] = (double)G + (double)gg * (double)D;
    }
  return ORC_OK;
}

int orc_decode(const uint8_t *desc, uint32_t n_meshlets, const uint8_t *payload,
               uint64_t payload_bytes, const uint8_t *grids, uint32_t n_grids,
               uint32_t first, uint32_t count, uint8_t *local, uint32_t *global,
               float *pos, double *pos64) {
  if (!desc || !payload || !grids || (uint64_t)first + count > n_meshlets) return ORC_ERR_ARG;
  uint8_t tl[3 * 256];
  float tp[3 * 256];
  double tp64[3 * 256];
  for (uint32_t m = first; m < first + count; m++) {
    desc_t d;
    parse_desc(desc + 32 * (size_t)m, &d);
    int rc = orc_decode_meshlet(desc + 32 * (size_t)m, payload, payload_bytes, grids, n_grids,
                                tl, tp, tp64);
    if (rc != ORC_OK) return rc;
    for (uint32_t i = 0; i < 3 * d.tp; i++) {
      if (local) local[3 * (size_t)d.tbase + i] = tl[i];
      if (global) global[3 * (size_t)d.tbase + i] = d.vbase + tl[i];
    }
    for (uint32_t i = 0; i < 3 * d.V; i++) {
      if (pos) pos[3 * (size_t)d.vbase + i] = tp[i];
      if (pos64) pos64[3 * (size_t)d.vbase + i] = tp64[i];
    }
  }
  return ORC_OK;
}

/* row r of the row-major clip matrix applied to (x, y, z, 1) */
static float clip_row(const float *M, int r, float x, float y, float z) {
  return fmaf(M[4 * r + 2], z, fmaf(M[4 * r + 1], y, fmaf(M[4 * r + 0], x, M[4 * r + 3])));
}

int orc_decode_attrs(const uint8_t *desc, const uint8_t *adesc, uint32_t n_meshlets,
                     const uint8_t *payload, uint64_t payload_bytes, const uint8_t *agrids,
                     uint32_t n_agrids, uint32_t n_attr, uint32_t attr_bits, uint32_t first,
                     uint32_t count, float *attr) {
  if (!desc || !adesc || !payload || !agrids || !attr || n_attr < 1 || n_attr > 5 ||
      attr_bits < 1 || attr_bits > 32 || (uint64_t)first + count > n_meshlets)
    return ORC_ERR_ARG;
  for (uint32_t m = first; m < first + count; m++) {
    desc_t d;
    parse_desc(desc + 32 * (size_t)m, &d);
    if (d.V < 3 || d.V > 256 || d.tp < 1 || d.tp > 256 || d.w > 8 || d.b < 1 || d.b > 32 ||
        d.V > d.tp + 2)
      return ORC_ERR_CORRUPT;
    const uint8_t *ar = adesc + 32 * (size_t)m;
    uint32_t ag = get_u16(ar + 20);
    if (ag >= n_agrids) return ORC_ERR_CORRUPT;
    const uint8_t *g = agrids + 48 * (size_t)ag;
    if (get_u32(g + 40) != attr_bits) return ORC_ERR_CORRUPT;
    for (uint32_t c = 0; c < n_attr; c++) /* the attribute box fits 32 bits, as for positions */
      if ((uint64_t)get_u32(ar + 4 * c) + ((1ull << attr_bits) - 1) > 0xFFFFFFFFull)
        return ORC_ERR_CORRUPT;
    uint64_t nw = (d.tp + 31) / 32;
    uint64_t cw = d.w == 0 ? nw + ((uint64_t)d.tp - 1 + 3) / 4
                           : 2 * nw + ((uint64_t)(d.tp + 2 - d.V) * d.w + 31) / 32;
    uint64_t pw = (3 * (uint64_t)d.V * d.b + 31) / 32;
    uint64_t aw = ((uint64_t)n_attr * d.V * attr_bits + 31) / 32;
    uint64_t start = 16 * (uint64_t)d.off16;
    if (start + 4 * (cw + pw + aw) > payload_bytes) return ORC_ERR_CORRUPT;
    const uint8_t *AB = payload + start + 4 * (cw + pw);
    for (uint32_t v = 0; v < d.V; v++)
      for (uint32_t c = 0; c < n_attr; c++) {
        uint64_t gg = (uint64_t)get_u32(ar + 4 * c) +
                      get_bits(AB, ((uint64_t)n_attr * v + c) * attr_bits, attr_bits);
        if (gg > 0xFFFFFFFFull) return ORC_ERR_CORRUPT;
        attr[(size_t)n_attr * ((size_t)d.vbase + v) + c] =
            orc_dequant32((uint32_t)gg, get_f32(g + 4 * c), get_f32(g + 20 + 4 * c));
      }
  }
  return ORC_OK;
}

int orc_view_eye(const float *vp, float eye[3]) {
  double r0[3], r1[3], r3[3];
  for (int c = 0; c < 3; c++) {
    r0[c] = vp[c];
    r1[c] = vp[4 + c];
    r3[c] = vp[12 + c];
  }
  const double b0 = -(double)vp[3], b1 = -(double)vp[7], b3 = -(double)vp[15];
  /* cross products r1 x r3, r3 x r0, r0 x r1 */
  double k0[3] = {r1[1] * r3[2] - r1[2] * r3[1], r1[2] * r3[0] - r1[0] * r3[2],
                  r1[0] * r3[1] - r1[1] * r3[0]};
  double k1[3] = {r3[1] * r0[2] - r3[2] * r0[1], r3[2] * r0[0] - r3[0] * r0[2],
                  r3[0] * r0[1] - r3[1] * r0[0]};
  double k3[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2],
                  r0[0] * r1[1] - r0[1] * r1[0]};
  double det = r0[0] * k0[0] + r0[1] * k0[1] + r0[2] * k0[2];
  if (!(det != 0.0) || !isfinite(det)) return 0;
  for (int c = 0; c < 3; c++) {
    double e = (b0 * k0[c] + b1 * k1[c] + b3 * k3[c]) / det;
    if (!isfinite(e)) return 0;
    eye[c] = (float)e;
  }
  return 1;
}

int orc_cone_test(const uint8_t *cone32, const float eye[3]) {
  float ctr[3], ax[3];
  for (int c = 0; c < 3; c++) {
    ctr[c] = get_f32(cone32 + 4 * c);
    ax[c] = get_f32(cone32 + 16 + 4 * c);
  }
  float radius = get_f32(cone32 + 12), sn = get_f32(cone32 + 28);
  if (!(sn < 1.0f)) return 0;
  float vx = ctr[0] - eye[0], vy = ctr[1] - eye[1], vz = ctr[2] - eye[2];
  float d = fmaf(ax[2], vz, fmaf(ax[1], vy, ax[0] * vx));
  float l = sqrtf(fmaf(vz, vz, fmaf(vy, vy, vx * vx)));
  return d >= fmaf(sn, l, radius);
}

int orc_decode_cull(const uint8_t *desc, uint32_t n_meshlets,
                    const uint8_t *payload, uint64_t payload_bytes,
                    const uint8_t *grids, uint32_t n_grids, uint32_t first,
                    uint32_t count, const float *vp, const uint8_t *cones,
                    uint32_t *tri_out, uint64_t *count_io, float *pos, uint8_t *pass_out) {
  if (!desc || !payload || !grids || !vp || !tri_out || !count_io ||
      (uint64_t)first + count > n_meshlets)
    return ORC_ERR_ARG;
  float eye[3];
  const int use_cones = cones && orc_view_eye(vp, eye);
  uint8_t tl[3 * 256];
  float tp[3 * 256];
  float cx[256], cy[256], cw[256];
  for (uint32_t m = first; m < first + count; m++) {
    desc_t d;
    parse_desc(desc + 32 * (size_t)m, &d);
    if (d.grid >= n_grids || d.b < 1 || d.b > 32) return ORC_ERR_CORRUPT;
    const uint8_t *g = grids + 32 * (size_t)d.grid;
    /* frustum test on the quantisation box */
    float lo[3], hi[3];
    for (int ch = 0; ch < 3; ch++) {
      uint64_t top = (uint64_t)d.L[ch] + ((1ull << d.b) - 1);
      if (top > 0xFFFFFFFFull) return ORC_ERR_CORRUPT;
      float G = get_f32(g + 4 * ch), D = get_f32(g + 16 + 4 * ch);
      lo[ch] = orc_dequant32(d.L[ch], G, D);
      hi[ch] = orc_dequant32((uint32_t)top, G, D);
    }
    int culled = 0;
    for (int plane = 0; plane < 6 && !culled; plane++) {
      int all_out = 1;
      for (int k = 0; k < 8 && all_out; k++) {
        float x = (k & 1) ? hi[0] : lo[0];
        float y = (k & 2) ? hi[1] : lo[1];
        float z = (k & 4) ? hi[2] : lo[2];
        float comp = clip_row(vp, plane >> 1, x, y, z);
        float w = clip_row(vp, 3, x, y, z);
        float dist = (plane & 1) ? w - comp : w + comp;
        if (!(dist < 0.0f)) all_out = 0;
      }
      if (all_out) culled = 1;
    }
    if (!culled && use_cones && orc_cone_test(cones + 32 * (size_t)m, eye)) culled = 1;
    if (pass_out) pass_out[m] = (uint8_t)!culled;
    if (culled) continue;
    int rc = orc_decode_meshlet(desc + 32 * (size_t)m, payload, payload_bytes, grids, n_grids,
                                tl, tp, NULL);
    if (rc != ORC_OK) return rc;
    for (uint32_t v = 0; v < d.V; v++) {
      float x = tp[3 * v], y = tp[3 * v + 1], z = tp[3 * v + 2];
      if (pos) {
        pos[3 * ((size_t)d.vbase + v)] = x;
        pos[3 * ((size_t)d.vbase + v) + 1] = y;
        pos[3 * ((size_t)d.vbase + v) + 2] = z;
      }
      cx[v] = clip_row(vp, 0, x, y, z);
      cy[v] = clip_row(vp, 1, x, y, z);
      cw[v] = clip_row(vp, 3, x, y, z);
    }
    for (uint32_t k = 0; k < d.tp; k++) {
      uint32_t i0 = tl[3 * k], i1 = tl[3 * k + 1], i2 = tl[3 * k + 2];
      if (i0 == i1 || i1 == i2 || i0 == i2) continue;
      int keep;
      if (cw[i0] <= 0.0f || cw[i1] <= 0.0f || cw[i2] <= 0.0f) {
        keep = 1;
      } else {
        float x0 = cx[i0], y0 = cy[i0], w0 = cw[i0];
        float x1 = cx[i1], y1 = cy[i1], w1 = cw[i1];
        float x2 = cx[i2], y2 = cy[i2], w2 = cw[i2];
        float c0 = fmaf(y1, w2, -(w1 * y2));
        float c1 = fmaf(x1, w2, -(w1 * x2));
        float c2 = fmaf(x1, y2, -(y1 * x2));
        float det = fmaf(w0, c2, fmaf(-y0, c1, x0 * c0));
        keep = det > 0.0f;
      }
      if (!keep) continue;
      uint64_t o = 3 * (*count_io);
      tri_out[o] = d.vbase + i0;
      tri_out[o + 1] = d.vbase + i1;
      tri_out[o + 2] = d.vbase + i2;
      (*count_io)++;
    }
  }
  return ORC_OK;
}
