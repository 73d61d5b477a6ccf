/*
 * Oracle: GTS-Reuse packing (Sec. 4.3) and crack-free quantisation (Sec. 4.4).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Index reuse packing (Sec. 4.3): meshlet vertices are renumbered in the
 * order they first appear in the strip stream, so the stream starts 0,1,2 and
 * the first triangle needs no storage.  Triangle k >= 1 brings one stream
 * entry n_k; its increment flag is 1 if n_k appears for the first time (then
 * n_k is simply the next unused number) and 0 otherwise, in which case n_k is
 * appended to the reuse buffer at w bits.
 *
 * Quantisation (Sec. 4.4), per mesh and per bit width b in use:
 *   G_c     = minimum of channel c over the mesh's vertices (FP32, exact);
 *   w_c     = largest extent of channel c over the meshlets quantised at b;
 *   Delta_c = w_c / (2^b - 1), computed in FP64 and rounded up to FP32
 *             (1 if w_c = 0), raised by one FP32 step at a time should a
 *             meshlet still need more than b bits after rounding;
 *   global grid coordinate of x:  floor((x - G_c) / Delta_c + 1/2)  (FP64);
 *   L_c     = the meshlet's smallest grid coordinate; stored q = coord - L_c.
 * A vertex duplicated in two meshlets of the same b therefore has the same
 * grid coordinate in both and decodes to the same float: no cracks.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  uint32_t tp, V, R, w, b, strips;
  uint8_t f[256], inc[256]; /* per triangle */
  uint8_t reuse[256];       /* reuse buffer values */
  uint8_t ent[256];         /* plain GTS: stream entry n_k of triangle k */
  uint32_t gv[256];         /* global vertex id of local vertex */
  uint32_t L[3];
  uint32_t q[256][3];
  uint32_t La[5];           /* attribute channels: meshlet minimum on their grid */
  uint32_t qa[256][5];
} meshlet_t;

static void put_bits(uint32_t *words, uint64_t bit, uint32_t nbits, uint64_t value) {
  for (uint32_t i = 0; i < nbits; i++)
    if ((value >> i) & 1u) words[(bit + i) >> 5] |= 1u << ((bit + i) & 31u);
}

static void put_u16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t *p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void put_f32(uint8_t *p, float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  put_u32(p, u);
}

/* Normal cone of one meshlet (record layout in oracle.h), from its decoded
 * FP32 positions P[3 V] and its nt input triangles lt[3 nt] (local ids, input
 * winding), all in FP64:
 *   center = middle of the positions' bounding box, rounded to FP32;
 *   radius = largest distance of a position from that center, times
 *            1 + 2^-20, rounded up to FP32;
 *   n_t    = normalised (p1 - p0) x (p2 - p0) of each non-degenerate triangle;
 *   axis   = normalised sum of the n_t, rounded to FP32;
 *   s      = sqrt(1 - c^2) + 2^-20 rounded up to FP32, c = min_t n_t . axis;
 *            1 (no cone) when c <= 0, when no triangle has an area, or when s
 *            would reach 1. */
static void meshlet_cone(const float *P, uint32_t V, const uint32_t *lt, uint32_t nt,
                         uint8_t *out) {
  double lo[3], hi[3];
  for (int c = 0; c < 3; c++) lo[c] = hi[c] = P[c];
  for (uint32_t v = 1; v < V; v++)
    for (int c = 0; c < 3; c++) {
      double x = P[3 * v + c];
      if (x < lo[c]) lo[c] = x;
      if (x > hi[c]) hi[c] = x;
    }
  float cf[3];
  for (int c = 0; c < 3; c++) cf[c] = (float)((lo[c] + hi[c]) * 0.5);
  double r = 0.0;
  for (uint32_t v = 0; v < V; v++) {
    double dx = (double)P[3 * v] - (double)cf[0];
    double dy = (double)P[3 * v + 1] - (double)cf[1];
    double dz = (double)P[3 * v + 2] - (double)cf[2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (d > r) r = d;
  }
  r = r * (1.0 + ldexp(1.0, -20));
  float rf = (float)r;
  if ((double)rf < r) rf = nextafterf(rf, INFINITY);
  double n[256][3], S[3] = {0.0, 0.0, 0.0};
  uint32_t k = 0;
  for (uint32_t t = 0; t < nt; t++) {
    const float *p0 = P + 3 * lt[3 * t], *p1 = P + 3 * lt[3 * t + 1], *p2 = P + 3 * lt[3 * t + 2];
    double e1[3], e2[3];
    for (int c = 0; c < 3; c++) {
      e1[c] = (double)p1[c] - (double)p0[c];
      e2[c] = (double)p2[c] - (double)p0[c];
    }
    double x = e1[1] * e2[2] - e1[2] * e2[1];
    double y = e1[2] * e2[0] - e1[0] * e2[2];
    double z = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(x * x + y * y + z * z);
    if (!(len > 0.0)) continue;
    n[k][0] = x / len;
    n[k][1] = y / len;
    n[k][2] = z / len;
    for (int c = 0; c < 3; c++) S[c] += n[k][c];
    k++;
  }
  float af[3] = {0.0f, 0.0f, 1.0f}, sf = 1.0f;
  double sl = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  if (k > 0 && sl > 0.0) {
    double a[3] = {S[0] / sl, S[1] / sl, S[2] / sl};
    double cmin = 1.0;
    for (uint32_t t = 0; t < k; t++) {
      double d = n[t][0] * a[0] + n[t][1] * a[1] + n[t][2] * a[2];
      if (d < cmin) cmin = d;
    }
    for (int c = 0; c < 3; c++) af[c] = (float)a[c];
    if (cmin > 0.0) {
      double sn = sqrt(1.0 - cmin * cmin) + ldexp(1.0, -20);
      if (sn < 1.0) {
        sf = (float)sn;
        if ((double)sf < sn) sf = nextafterf(sf, INFINITY);
        if (sf > 1.0f) sf = 1.0f;
      }
    }
  }
  for (int c = 0; c < 3; c++) put_f32(out + 4 * c, cf[c]);
  put_f32(out + 12, rf);
  for (int c = 0; c < 3; c++) put_f32(out + 16 + 4 * c, af[c]);
  put_f32(out + 28, sf);
}

/* u32 words of a meshlet's connectivity section: GTS-Reuse (w >= 1): L/R
 * words, increment words, reuse words; plain GTS (w = 0): L/R words and one
 * byte per triangle k >= 1 holding its stream entry. */
static uint64_t conn_words(const meshlet_t *x) {
  uint64_t nw = (x->tp + 31) / 32;
  if (x->w == 0) return nw + ((uint64_t)x->tp - 1 + 3) / 4;
  return 2 * nw + ((uint64_t)x->R * x->w + 31) / 32;
}

static uint32_t ceil_log2(uint32_t v) {
  uint32_t w = 0;
  while ((1u << w) < v) w++;
  return w;
}

static int build_meshlet(const uint32_t *tris, const uint32_t *ids, uint32_t T,
                         uint32_t reuse_mode, uint32_t search_nodes, meshlet_t *m) {
  uint32_t stream[5 * 256 + 8];
  uint8_t flags[5 * 256 + 8];
  uint32_t order[257];
  uint32_t tp = 0, strips = 0;
  if (T == 0 || T > 256) return ORC_ERR_LIMIT;
  int rc = orc_stripify(tris, ids, T, search_nodes, stream, flags, order, &tp, &strips);
  if (rc != ORC_OK) return rc;
  if (tp > 256) return ORC_ERR_LIMIT;
  m->tp = tp;
  m->strips = strips;
  /* first-appearance renumbering */
  uint32_t V = 0;
  uint32_t local[5 * 256 + 8];
  for (uint32_t i = 0; i < tp + 2; i++) {
    uint32_t g = stream[i], found = V;
    for (uint32_t j = 0; j < V; j++)
      if (m->gv[j] == g) { found = j; break; }
    if (found == V) {
      if (V == 256) return ORC_ERR_LIMIT;
      m->gv[V++] = g;
    }
    local[i] = found;
  }
  m->V = V;
  uint32_t R = 0, seen = 3;
  m->f[0] = 0;
  m->inc[0] = 0;
  m->ent[0] = 2;
  for (uint32_t k = 1; k < tp; k++) {
    m->f[k] = flags[k];
    uint32_t n = local[k + 2];
    m->ent[k] = (uint8_t)n;
    if (n == seen) {
      m->inc[k] = 1;
      seen++;
    } else {
      m->inc[k] = 0;
      m->reuse[R++] = (uint8_t)n;
    }
  }
  m->R = R;
  m->w = reuse_mode == 0 ? 8u : reuse_mode == 1 ? ceil_log2(V) : 0u;
  return ORC_OK;
}

/* Crack-free quantisation of n_ch extra attribute channels (Sec. 4.4, the
 * attribute vector beyond the position) at `bits` bits, one grid for the
 * mesh, by the same rules as the positions:
 *   G_c = smallest value of channel c over the mesh's vertices (FP32);
 *   Delta_c = largest meshlet extent of channel c / (2^bits - 1), in FP64,
 *             rounded up to FP32 (1 when 0), raised one FP32 step at a time
 *             while a meshlet still needs more than `bits` bits;
 *   grid coordinate floor((a - G_c) / Delta_c + 1/2), La_c = meshlet minimum. */
static int quantise_attrs(const float *attrs, uint32_t n_verts, uint32_t n_ch, uint32_t bits,
                          meshlet_t *ms, uint32_t n_meshlets, float *G, float *D) {
  double qmax = ldexp(1.0, (int)bits) - 1.0;
  for (uint32_t c = 0; c < n_ch; c++) {
    G[c] = attrs[c];
    for (uint32_t v = 1; v < n_verts; v++)
      if (attrs[(size_t)n_ch * v + c] < G[c]) G[c] = attrs[(size_t)n_ch * v + c];
    double wmax = 0.0;
    for (uint32_t m = 0; m < n_meshlets; m++) {
      float lo = attrs[(size_t)n_ch * ms[m].gv[0] + c], hi = lo;
      for (uint32_t i = 1; i < ms[m].V; i++) {
        float x = attrs[(size_t)n_ch * ms[m].gv[i] + c];
        if (x < lo) lo = x;
        if (x > hi) hi = x;
      }
      if ((double)hi - (double)lo > wmax) wmax = (double)hi - (double)lo;
    }
    float Df = 1.0f;
    if (wmax > 0.0) {
      double d = wmax / qmax;
      Df = (float)d;
      if ((double)Df < d) Df = nextafterf(Df, INFINITY);
    }
    for (;;) {
      int ok = 1;
      for (uint32_t m = 0; m < n_meshlets && ok; m++) {
        double lo = 0, hi = 0;
        for (uint32_t i = 0; i < ms[m].V; i++) {
          double y = ((double)attrs[(size_t)n_ch * ms[m].gv[i] + c] - (double)G[c]) / (double)Df;
          double g = floor(y + 0.5);
          if (g > 4294967295.0) return ORC_ERR_LIMIT;
          if (i == 0 || g < lo) lo = g;
          if (i == 0 || g > hi) hi = g;
        }
        if (hi - lo > qmax) { ok = 0; break; }
        if (lo + qmax > 4294967295.0) return ORC_ERR_LIMIT;
        ms[m].La[c] = (uint32_t)lo;
        for (uint32_t i = 0; i < ms[m].V; i++) {
          double y = ((double)attrs[(size_t)n_ch * ms[m].gv[i] + c] - (double)G[c]) / (double)Df;
          ms[m].qa[i][c] = (uint32_t)(floor(y + 0.5) - lo);
        }
      }
      if (ok) break;
      Df = nextafterf(Df, INFINITY);
    }
    D[c] = Df;
  }
  return ORC_OK;
}

int orc_encode(const float *pos, uint32_t n_verts, const uint32_t *tris,
               const uint32_t *mtri, const uint32_t *mstart,
               uint32_t n_meshlets, const uint8_t *bits, uint32_t reuse_mode,
               const uint32_t *perm, uint32_t mesh_id, const float *attrs, uint32_t n_attr,
               uint32_t attr_bits, uint32_t strip_search_nodes, orc_blob **out) {
  if (!pos || !tris || !mtri || !mstart || !bits || !out || n_verts == 0 || reuse_mode > 2 ||
      n_attr > 5 || (n_attr && (!attrs || attr_bits < 1 || attr_bits > 32)))
    return ORC_ERR_ARG;
  *out = NULL;
  for (uint32_t m = 0; m < n_meshlets; m++)
    if (bits[m] < 1 || bits[m] > 32) return ORC_ERR_ARG;
  meshlet_t *ms = (meshlet_t *)calloc(n_meshlets ? n_meshlets : 1, sizeof(meshlet_t));
  if (!ms) return ORC_ERR_NOMEM;
  int rc = ORC_OK;
  for (uint32_t m = 0; m < n_meshlets && rc == ORC_OK; m++) {
    rc = build_meshlet(tris, mtri + mstart[m], mstart[m + 1] - mstart[m], reuse_mode,
                       strip_search_nodes, &ms[m]);
    ms[m].b = bits[m];
  }
  if (rc != ORC_OK) { free(ms); return rc; }

  /* ---- quantisation ---- */
  float G[3];
  for (int c = 0; c < 3; c++) {
    G[c] = pos[c];
    for (uint32_t v = 1; v < n_verts; v++)
      if (pos[3 * (size_t)v + c] < G[c]) G[c] = pos[3 * (size_t)v + c];
  }
  float D[33][3];
  int present[33] = {0};
  for (uint32_t m = 0; m < n_meshlets; m++) present[ms[m].b] = 1;
  for (uint32_t b = 1; b <= 32 && rc == ORC_OK; b++) {
    if (!present[b]) continue;
    double qmax = ldexp(1.0, (int)b) - 1.0;
    for (int c = 0; c < 3 && rc == ORC_OK; c++) {
      double wmax = 0.0;
      for (uint32_t m = 0; m < n_meshlets; m++) {
        if (ms[m].b != b) continue;
        float lo = pos[3 * (size_t)ms[m].gv[0] + c], hi = lo;
        for (uint32_t i = 1; i < ms[m].V; i++) {
          float x = pos[3 * (size_t)ms[m].gv[i] + c];
          if (x < lo) lo = x;
          if (x > hi) hi = x;
        }
        double ext = (double)hi - (double)lo;
        if (ext > wmax) wmax = ext;
      }
      float Df = 1.0f;
      if (wmax > 0.0) {
        double d = wmax / qmax;
        Df = (float)d;
        if ((double)Df < d) Df = nextafterf(Df, INFINITY);
      }
      for (;;) {
        int ok = 1;
        for (uint32_t m = 0; m < n_meshlets && ok; m++) {
          if (ms[m].b != b) continue;
          double lo = 0, hi = 0;
          for (uint32_t i = 0; i < ms[m].V; i++) {
            double y = ((double)pos[3 * (size_t)ms[m].gv[i] + c] - (double)G[c]) / (double)Df;
            double g = floor(y + 0.5);
            if (g > 4294967295.0) { rc = ORC_ERR_LIMIT; ok = 0; break; }
            if (i == 0 || g < lo) lo = g;
            if (i == 0 || g > hi) hi = g;
          }
          if (rc != ORC_OK) break;
          if (hi - lo > qmax) ok = 0;
          else if (lo + qmax > 4294967295.0) { rc = ORC_ERR_LIMIT; ok = 0; }
          else {
            ms[m].L[c] = (uint32_t)lo;
            for (uint32_t i = 0; i < ms[m].V; i++) {
              double y = ((double)pos[3 * (size_t)ms[m].gv[i] + c] - (double)G[c]) / (double)Df;
              ms[m].q[i][c] = (uint32_t)(floor(y + 0.5) - lo);
            }
          }
        }
        if (rc != ORC_OK || ok) break;
        Df = nextafterf(Df, INFINITY);
      }
      D[b][c] = Df;
    }
  }
  if (rc != ORC_OK) { free(ms); return rc; }
  float GA[5] = {0}, DA[5] = {0};
  if (n_attr) rc = quantise_attrs(attrs, n_verts, n_attr, attr_bits, ms, n_meshlets, GA, DA);
  if (rc != ORC_OK) { free(ms); return rc; }

  /* ---- grids: one per bit width in use, ascending b ---- */
  uint32_t grid_of[33], n_grids = 0;
  for (uint32_t b = 1; b <= 32; b++) grid_of[b] = present[b] ? n_grids++ : 0;

  /* ---- sizes ---- */
  orc_blob *blob = (orc_blob *)calloc(1, sizeof(orc_blob));
  if (!blob) { free(ms); return ORC_ERR_NOMEM; }
  uint64_t total_words = 0;
  for (uint32_t m = 0; m < n_meshlets; m++) {
    meshlet_t *x = &ms[m];
    uint64_t words = conn_words(x) + (3 * (uint64_t)x->V * x->b + 31) / 32 +
                     ((uint64_t)n_attr * x->V * attr_bits + 31) / 32;
    total_words += (words + 3) / 4 * 4;
  }
  blob->n_meshlets = n_meshlets;
  blob->n_grids = n_grids;
  blob->payload_bytes = total_words * 4;
  blob->desc = (uint8_t *)calloc((size_t)n_meshlets * 32 + 1, 1);
  blob->payload = (uint8_t *)calloc((size_t)total_words * 4 + 16, 1);
  blob->grids = (uint8_t *)calloc((size_t)n_grids * 32 + 1, 1);
  uint64_t all_v = 0;
  for (uint32_t m = 0; m < n_meshlets; m++) all_v += ms[m].V;
  blob->vmap = (uint32_t *)calloc((size_t)all_v + 1, sizeof(uint32_t));
  blob->cones = (uint8_t *)calloc((size_t)n_meshlets * 32 + 1, 1);
  blob->n_attr = n_attr;
  blob->attr_bits = n_attr ? attr_bits : 0;
  blob->adesc = (uint8_t *)calloc((size_t)n_meshlets * 32 + 1, 1);
  blob->agrids = (uint8_t *)calloc(48, 1);
  /* >= 2*8 + 64 + 768 + 5*256*32/32 + 3 words */
  uint32_t *words = (uint32_t *)calloc(2304, sizeof(uint32_t));
  if (!blob->desc || !blob->payload || !blob->grids || !blob->vmap || !blob->cones ||
      !blob->adesc || !blob->agrids || !words) {
    free(words); free(ms); orc_blob_free(blob);
    return ORC_ERR_NOMEM;
  }
  if (n_attr) {
    for (uint32_t c = 0; c < n_attr; c++) {
      put_f32(blob->agrids + 4 * c, GA[c]);
      put_f32(blob->agrids + 20 + 4 * c, DA[c]);
    }
    put_u32(blob->agrids + 40, attr_bits);
    put_u32(blob->agrids + 44, mesh_id);
  }
  for (uint32_t b = 1; b <= 32; b++) {
    if (!present[b]) continue;
    uint8_t *g = blob->grids + 32 * (size_t)grid_of[b];
    for (int c = 0; c < 3; c++) put_f32(g + 4 * c, G[c]);
    put_u32(g + 12, b);
    for (int c = 0; c < 3; c++) put_f32(g + 16 + 4 * c, D[b][c]);
    put_u32(g + 28, mesh_id);
  }

  /* ---- emit in blob order ---- */
  uint64_t off_words = 0, vbase = 0, tbase = 0;
  for (uint32_t p = 0; p < n_meshlets; p++) {
    uint32_t mi = perm ? perm[p] : p;
    if (mi >= n_meshlets) { free(words); free(ms); orc_blob_free(blob); return ORC_ERR_ARG; }
    meshlet_t *x = &ms[mi];
    uint32_t nw = (x->tp + 31) / 32;
    uint64_t cw = conn_words(x);
    uint64_t pw = (3 * (uint64_t)x->V * x->b + 31) / 32;
    uint64_t aw = ((uint64_t)n_attr * x->V * attr_bits + 31) / 32;
    uint64_t n = (cw + pw + aw + 3) / 4 * 4;
    memset(words, 0, n * 4);
    for (uint32_t k = 0; k < x->tp; k++) put_bits(words, k, 1, x->f[k]);
    if (x->w == 0) {
      for (uint32_t k = 1; k < x->tp; k++) put_bits(words + nw, 8 * (uint64_t)(k - 1), 8, x->ent[k]);
    } else {
      for (uint32_t k = 0; k < x->tp; k++) put_bits(words + nw, k, 1, x->inc[k]);
      for (uint32_t r = 0; r < x->R; r++) put_bits(words + 2 * nw, (uint64_t)r * x->w, x->w, x->reuse[r]);
    }
    for (uint32_t v = 0; v < x->V; v++)
      for (int c = 0; c < 3; c++)
        put_bits(words + cw, (3 * (uint64_t)v + c) * x->b, x->b, x->q[v][c]);
    for (uint32_t v = 0; v < x->V; v++)
      for (uint32_t c = 0; c < n_attr; c++)
        put_bits(words + cw + pw, ((uint64_t)n_attr * v + c) * attr_bits, attr_bits, x->qa[v][c]);
    for (uint32_t c = 0; c < n_attr; c++) put_u32(blob->adesc + 32 * (size_t)p + 4 * c, x->La[c]);
    for (uint64_t i = 0; i < n; i++) put_u32(blob->payload + 4 * (off_words + i), words[i]);
    uint8_t *d = blob->desc + 32 * (size_t)p;
    if (vbase + x->V > 0xFFFFFFFFull || tbase + x->tp > 0xFFFFFFFFull ||
        off_words / 4 > 0xFFFFFFFFull) {
      free(words); free(ms); orc_blob_free(blob);
      return ORC_ERR_LIMIT;
    }
    put_u32(d + 0, (uint32_t)(off_words / 4));
    put_u32(d + 4, (uint32_t)vbase);
    put_u32(d + 8, (uint32_t)tbase);
    put_u16(d + 12, x->V);
    put_u16(d + 14, x->tp);
    d[16] = (uint8_t)x->w;
    d[17] = (uint8_t)x->b;
    put_u16(d + 18, grid_of[x->b]);
    for (int c = 0; c < 3; c++) put_u32(d + 20 + 4 * c, x->L[c]);
    for (uint32_t i = 0; i < x->V; i++) blob->vmap[vbase + i] = x->gv[i];
    {
      /* decoded positions and local input triangles for the normal cone */
      float P[3 * 256];
      uint32_t lt[3 * 256];
      const uint8_t *g = blob->grids + 32 * (size_t)grid_of[x->b];
      for (uint32_t i = 0; i < x->V; i++)
        for (int c = 0; c < 3; c++) {
          float Gc, Dc;
          uint32_t gu = (uint32_t)g[4 * c] | (uint32_t)g[4 * c + 1] << 8 |
                        (uint32_t)g[4 * c + 2] << 16 | (uint32_t)g[4 * c + 3] << 24;
          uint32_t du = (uint32_t)g[16 + 4 * c] | (uint32_t)g[17 + 4 * c] << 8 |
                        (uint32_t)g[18 + 4 * c] << 16 | (uint32_t)g[19 + 4 * c] << 24;
          memcpy(&Gc, &gu, 4);
          memcpy(&Dc, &du, 4);
          P[3 * i + c] = orc_dequant32(x->L[c] + x->q[i][c], Gc, Dc);
        }
      uint32_t nt = mstart[mi + 1] - mstart[mi];
      for (uint32_t t = 0; t < nt; t++)
        for (int c = 0; c < 3; c++) {
          uint32_t gvid = tris[3 * (size_t)mtri[mstart[mi] + t] + c], li = 0;
          while (li < x->V && x->gv[li] != gvid) li++;
          lt[3 * t + c] = li;
        }
      meshlet_cone(P, x->V, lt, nt, blob->cones + 32 * (size_t)p);
    }
    off_words += n;
    vbase += x->V;
    tbase += x->tp;
    blob->restarts += x->strips - 1;
    blob->degenerates += 4 * (uint64_t)(x->strips - 1);
    blob->conn_bits += x->w ? 2 * (uint64_t)x->tp + (uint64_t)x->w * x->R
                            : (uint64_t)x->tp + 8 * (uint64_t)(x->tp - 1);
    blob->reuse_entries += x->R;
  }
  blob->total_tris = tbase;
  blob->total_verts = vbase;
  free(words);
  free(ms);
  *out = blob;
  return ORC_OK;
}

void orc_blob_free(orc_blob *b) {
  if (!b) return;
  free(b->desc);
  free(b->payload);
  free(b->grids);
  free(b->vmap);
  free(b->cones);
  free(b->adesc);
  free(b->agrids);
  free(b);
}
