// Index reuse packing (Sec. 4.3), crack-free quantisation (Sec. 4.4) and the
// blob container of the C ABI.
//
// Reuse packing: vertices of a meshlet are numbered by first appearance in
// its strip stream, so the stream starts (0, 1, 2) and the first triangle is
// implicit.  For triangle k >= 1 the increment flag says whether its stream
// entry is new (then it equals the count of vertices seen so far) or a reuse,
// stored in the reuse buffer at w bits.
//
// Quantisation, per mesh and per position bit width b:
//   G      minimum over the mesh's vertices (FP32, exact);
//   w_c    largest extent of channel c over the meshlets at width b;
//   Delta  w_c / (2^b - 1) in FP64, rounded up to FP32 (1 when w_c = 0),
//          raised by one FP32 step while some meshlet would need > b bits;
//   grid coordinate g = floor((x - G) / Delta + 1/2) in FP64;
//   L_c    the meshlet's smallest g; stored q = g - L_c.
// Equal input vertices get equal g at equal b, so boundary vertices shared by
// meshlets decode to identical floats: no cracks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "host_internal.h"

using namespace mc;

namespace {

struct Packed {
  uint32_t V = 0, R = 0, w = 0, b = 0, tp = 0, strips = 0;
  uint32_t words = 0;  // padded block size in u32 words
  std::vector<uint32_t> gv;     // global vertex id per local id
  std::vector<uint8_t> reuse;   // reuse entries
  std::vector<uint8_t> ent;     // plain GTS (w = 0): stream entry of triangles 1..T'-1
  uint32_t flag_words[8], inc_words[8];
  uint32_t L[3];
  uint32_t La[5];  // attribute channels: meshlet minimum on their grid
};

inline void put_bits(uint32_t *w, uint64_t bit, uint32_t nbits, uint32_t value) {
  uint64_t v = (uint64_t)(nbits == 32 ? value : (value & ((1u << nbits) - 1u))) << (bit & 31u);
  w[bit >> 5] |= (uint32_t)v;
  if ((bit & 31u) + nbits > 32) w[(bit >> 5) + 1] |= (uint32_t)(v >> 32);
}

uint32_t ceil_log2(uint32_t v) {
  uint32_t w = 0;
  while ((1u << w) < v) w++;
  return w;
}

// smallest float >= d (d > 0)
float round_up_float(double d) {
  float f = (float)d;
  if ((double)f < d) f = std::nextafter(f, INFINITY);
  return f;
}

// FP32 position of grid coordinate g (the dequantisation of Sec. 4.4, as the
// decoder evaluates it)
float grid_to_float(uint32_t g, float G, float D) {
  if (g < (1u << 24)) return std::fma((float)g, D, G);
  return std::fma((float)(g & 0xFFFu), D, std::fma((float)(g >> 12), D * 4096.0f, G));
}

// Normal cone of one meshlet (mc_cone) from its decoded positions P (V
// vertices) and its triangles in local ids tl (nt of them, input winding).
mc_cone meshlet_cone(const float *P, uint32_t V, const uint32_t *tl, uint32_t nt) {
  mc_cone k{};
  double lo[3], hi[3];
  for (int c = 0; c < 3; c++) lo[c] = hi[c] = P[c];
  for (uint32_t v = 1; v < V; v++)
    for (int c = 0; c < 3; c++) {
      const double x = P[3 * v + c];
      lo[c] = x < lo[c] ? x : lo[c];
      hi[c] = x > hi[c] ? x : hi[c];
    }
  for (int c = 0; c < 3; c++) k.center[c] = (float)((lo[c] + hi[c]) * 0.5);
  double r = 0.0;
  for (uint32_t v = 0; v < V; v++) {
    const double dx = (double)P[3 * v] - (double)k.center[0];
    const double dy = (double)P[3 * v + 1] - (double)k.center[1];
    const double dz = (double)P[3 * v + 2] - (double)k.center[2];
    const double d = std::sqrt(dx * dx + dy * dy + dz * dz);
    if (d > r) r = d;
  }
  k.radius = round_up_float(r * (1.0 + std::ldexp(1.0, -20)));
  double nrm[256][3], sum[3] = {0.0, 0.0, 0.0};
  uint32_t cnt = 0;
  for (uint32_t t = 0; t < nt; t++) {
    const float *a = P + 3 * tl[3 * t], *b = P + 3 * tl[3 * t + 1], *c = P + 3 * tl[3 * t + 2];
    const double u0 = (double)b[0] - (double)a[0], u1 = (double)b[1] - (double)a[1],
                 u2 = (double)b[2] - (double)a[2];
    const double w0 = (double)c[0] - (double)a[0], w1 = (double)c[1] - (double)a[1],
                 w2 = (double)c[2] - (double)a[2];
    const double x = u1 * w2 - u2 * w1, y = u2 * w0 - u0 * w2, z = u0 * w1 - u1 * w0;
    const double len = std::sqrt(x * x + y * y + z * z);
    if (!(len > 0.0)) continue;
    nrm[cnt][0] = x / len;
    nrm[cnt][1] = y / len;
    nrm[cnt][2] = z / len;
    for (int i = 0; i < 3; i++) sum[i] += nrm[cnt][i];
    cnt++;
  }
  k.axis[0] = 0.0f;
  k.axis[1] = 0.0f;
  k.axis[2] = 1.0f;
  k.s = 1.0f;
  const double sl = std::sqrt(sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2]);
  if (cnt == 0 || !(sl > 0.0)) return k;
  const double ax[3] = {sum[0] / sl, sum[1] / sl, sum[2] / sl};
  double cmin = 1.0;
  for (uint32_t t = 0; t < cnt; t++) {
    const double d = nrm[t][0] * ax[0] + nrm[t][1] * ax[1] + nrm[t][2] * ax[2];
    cmin = d < cmin ? d : cmin;
  }
  for (int i = 0; i < 3; i++) k.axis[i] = (float)ax[i];
  if (cmin > 0.0) {
    const double sn = std::sqrt(1.0 - cmin * cmin) + std::ldexp(1.0, -20);
    if (sn < 1.0) k.s = std::min(1.0f, round_up_float(sn));
  }
  return k;
}

}  // namespace

extern "C" mc_status mc_encode(const mc_meshlets *m, const float *pos, uint32_t n_verts,
                               const mc_encode_params *p, mc_blob **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!m || !pos || !p || n_verts != m->n_verts || p->reuse_mode > 2) return MC_ERR_INVALID_ARG;
  const uint32_t nm = mc_meshlets_count(m);
  if (!p->pos_bits_per_meshlet && (p->pos_bits < 1 || p->pos_bits > 32)) return MC_ERR_INVALID_ARG;
  if (p->pos_bits_per_meshlet)
    for (uint32_t i = 0; i < nm; i++)
      if (p->pos_bits_per_meshlet[i] < 1 || p->pos_bits_per_meshlet[i] > 32)
        return MC_ERR_INVALID_ARG;
  const uint32_t n_attr = p->n_attr;
  if (n_attr > 5 || (n_attr && (!p->attrs || p->attr_bits < 1 || p->attr_bits > 32)))
    return MC_ERR_INVALID_ARG;
  const uint32_t attr_bits = n_attr ? p->attr_bits : 0;
  if (p->order) {
    std::vector<uint8_t> seen(nm, 0);
    for (uint32_t i = 0; i < nm; i++) {
      if (p->order[i] >= nm || seen[p->order[i]]) return MC_ERR_INVALID_ARG;
      seen[p->order[i]] = 1;
    }
  }
  const uint32_t threads = default_threads(p->n_threads);
  mc_blob *blob = new (std::nothrow) mc_blob();
  if (!blob) return MC_ERR_OOM;
  try {
    std::vector<Packed> pk(nm);
    std::atomic<int> err{0};
    // ---- per meshlet: renumbering, flags, reuse entries
    parallel_for(
        nm, threads,
        [&](uint64_t i) {
          Packed &x = pk[i];
          const uint64_t s0 = m->stream_start[i];
          uint32_t tp = m->tp[i];
          const uint32_t *st = m->stream.data() + s0;
          const uint8_t *fl = m->flags.data() + s0;
          x.strips = m->strips[i];
          thread_local StripScratch scratch;
          thread_local StripOut searched;
          if (p->strip_search_nodes && x.strips > 1) {  // fewer strips by the search
            const uint32_t t0 = m->start[i], T = m->start[i + 1] - t0;
            build_strip(nullptr, m->tri.data() + t0, T, scratch, searched, p->strip_search_nodes,
                        m->corners.data() + 3 * (size_t)t0);
            if (searched.strips < x.strips) {
              tp = searched.tp;
              st = searched.stream.data();
              fl = searched.flags.data();
              x.strips = searched.strips;
            }
          }
          x.tp = tp;
          x.b = p->pos_bits_per_meshlet ? p->pos_bits_per_meshlet[i] : p->pos_bits;
          x.gv.clear();
          std::memset(x.flag_words, 0, sizeof(x.flag_words));
          std::memset(x.inc_words, 0, sizeof(x.inc_words));
          // first-appearance numbering (V <= 256: linear lookup in gv)
          uint8_t local[260 * 5];
          for (uint32_t k = 0; k < tp + 2; k++) {
            uint32_t g = st[k];
            uint32_t id = (uint32_t)x.gv.size();
            for (uint32_t j = 0; j < x.gv.size(); j++)
              if (x.gv[j] == g) {
                id = j;
                break;
              }
            if (id == x.gv.size()) {
              if (x.gv.size() == 256) {
                err.store(MC_ERR_LIMIT);
                return;
              }
              x.gv.push_back(g);
            }
            local[k] = (uint8_t)id;
          }
          x.V = (uint32_t)x.gv.size();
          uint32_t seen = 3;
          x.ent.clear();
          for (uint32_t k = 1; k < tp; k++) {
            if (fl[k]) x.flag_words[k >> 5] |= 1u << (k & 31);
            x.ent.push_back(local[k + 2]);
            if (local[k + 2] == seen) {
              x.inc_words[k >> 5] |= 1u << (k & 31);
              seen++;
            } else {
              x.reuse.push_back(local[k + 2]);
            }
          }
          x.R = (uint32_t)x.reuse.size();
          x.w = p->reuse_mode == 0 ? 8u : p->reuse_mode == 1 ? ceil_log2(x.V) : 0u;
          // connectivity words: GTS-Reuse = L/R + increment + reuse words;
          // plain GTS (w = 0) = L/R words + one byte per triangle k >= 1
          const uint32_t conn = x.w ? 2 * ((tp + 31) / 32) + (x.R * x.w + 31) / 32
                                    : (tp + 31) / 32 + (tp + 2) / 4;
          const uint32_t words = conn + (3 * x.V * x.b + 31) / 32 + (n_attr * x.V * attr_bits + 31) / 32;
          x.words = (words + 3) / 4 * 4;
        },
        256);
    if (err.load()) {
      delete blob;
      return (mc_status)err.load();
    }

    // ---- quantisation grid per bit width
    float G[3];
    for (int c = 0; c < 3; c++) {
      float g = pos[c];
      for (uint32_t v = 1; v < n_verts; v++) g = std::min(g, pos[3 * (size_t)v + c]);
      G[c] = g;
    }
    bool present[33] = {false};
    for (uint32_t i = 0; i < nm; i++) present[pk[i].b] = true;
    float delta[33][3];
    uint32_t grid_of[33] = {0}, n_grids = 0;
    for (uint32_t b = 1; b <= 32; b++) {
      if (!present[b]) continue;
      grid_of[b] = n_grids++;
      const double qmax = std::ldexp(1.0, (int)b) - 1.0;
      for (int c = 0; c < 3; c++) {
        double wmax = 0;
        for (uint32_t i = 0; i < nm; i++) {
          if (pk[i].b != b) continue;
          float lo = pos[3 * (size_t)pk[i].gv[0] + c], hi = lo;
          for (uint32_t g : pk[i].gv) {
            float x = pos[3 * (size_t)g + c];
            lo = std::min(lo, x);
            hi = std::max(hi, x);
          }
          wmax = std::max(wmax, (double)hi - (double)lo);
        }
        float D = wmax > 0 ? round_up_float(wmax / qmax) : 1.0f;
        for (;;) {
          std::atomic<int> over{0};
          parallel_for(
              nm, threads,
              [&](uint64_t i) {
                Packed &x = pk[i];
                if (x.b != b) return;
                double lo = 0, hi = 0;
                for (uint32_t j = 0; j < x.V; j++) {
                  double y = ((double)pos[3 * (size_t)x.gv[j] + c] - (double)G[c]) / (double)D;
                  double g = std::floor(y + 0.5);
                  if (j == 0 || g < lo) lo = g;
                  if (j == 0 || g > hi) hi = g;
                }
                if (hi > 4294967295.0 || lo + qmax > 4294967295.0) over.store(2);
                else if (hi - lo > qmax) over.store(std::max(over.load(), 1));
                else x.L[c] = (uint32_t)lo;
              },
              1024);
          if (over.load() == 2) {
            delete blob;
            return MC_ERR_LIMIT;
          }
          if (over.load() == 0) break;
          D = std::nextafter(D, INFINITY);
        }
        delta[b][c] = D;
      }
    }

    // ---- attribute channels: one crack-free grid per channel for the mesh,
    // by the rules of the positions (Sec. 4.4)
    float GA[5] = {0, 0, 0, 0, 0}, DA[5] = {0, 0, 0, 0, 0};
    if (n_attr) {
      const float *at = p->attrs;
      const double qmax = std::ldexp(1.0, (int)attr_bits) - 1.0;
      for (uint32_t c = 0; c < n_attr; c++) {
        float g0 = at[c];
        for (uint32_t v = 1; v < n_verts; v++) g0 = std::min(g0, at[(size_t)n_attr * v + c]);
        GA[c] = g0;
        double wmax = 0;
        for (uint32_t i = 0; i < nm; i++) {
          float lo = at[(size_t)n_attr * pk[i].gv[0] + c], hi = lo;
          for (uint32_t g : pk[i].gv) {
            const float x = at[(size_t)n_attr * g + c];
            lo = std::min(lo, x);
            hi = std::max(hi, x);
          }
          wmax = std::max(wmax, (double)hi - (double)lo);
        }
        float D = wmax > 0 ? round_up_float(wmax / qmax) : 1.0f;
        for (;;) {
          std::atomic<int> over{0};
          parallel_for(
              nm, threads,
              [&](uint64_t i) {
                Packed &x = pk[i];
                double lo = 0, hi = 0;
                for (uint32_t j = 0; j < x.V; j++) {
                  const double y = ((double)at[(size_t)n_attr * x.gv[j] + c] - (double)GA[c]) / (double)D;
                  const double g = std::floor(y + 0.5);
                  if (j == 0 || g < lo) lo = g;
                  if (j == 0 || g > hi) hi = g;
                }
                if (hi > 4294967295.0 || lo + qmax > 4294967295.0) over.store(2);
                else if (hi - lo > qmax) over.store(std::max(over.load(), 1));
                else x.La[c] = (uint32_t)lo;
              },
              1024);
          if (over.load() == 2) {
            delete blob;
            return MC_ERR_LIMIT;
          }
          if (over.load() == 0) break;
          D = std::nextafter(D, INFINITY);
        }
        DA[c] = D;
      }
    }

    // ---- layout in blob order
    std::vector<uint32_t> slot(nm);
    for (uint32_t s = 0; s < nm; s++) slot[s] = p->order ? p->order[s] : s;
    blob->desc.resize(nm);
    std::vector<uint64_t> off(nm + 1, 0), vb(nm + 1, 0), tb(nm + 1, 0);
    for (uint32_t s = 0; s < nm; s++) {
      const Packed &x = pk[slot[s]];
      off[s + 1] = off[s] + x.words;
      vb[s + 1] = vb[s] + x.V;
      tb[s + 1] = tb[s] + x.tp;
    }
    if (vb[nm] > 0xFFFFFFFFull || tb[nm] > 0xFFFFFFFFull || off[nm] / 4 > 0xFFFFFFFFull) {
      delete blob;
      return MC_ERR_LIMIT;
    }
    blob->payload.assign(off[nm] * 4, 0);
    blob->vmap.resize(vb[nm]);
    blob->cones.resize(nm);
    blob->n_attr = n_attr;
    blob->attr_bits = attr_bits;
    if (n_attr) blob->attr_desc.assign(nm, mc_attr_desc{});
    uint32_t *words = reinterpret_cast<uint32_t *>(blob->payload.data());
    parallel_for(
        nm, threads,
        [&](uint64_t s) {
          const Packed &x = pk[slot[s]];
          uint32_t *w = words + off[s];
          const uint32_t nw = (x.tp + 31) / 32;
          uint32_t *pw;
          if (x.w == 0) {
            for (uint32_t i = 0; i < nw; i++) w[i] = x.flag_words[i];
            uint8_t *eb = reinterpret_cast<uint8_t *>(w + nw);  // little-endian byte k-1
            for (uint32_t k = 1; k < x.tp; k++) eb[k - 1] = x.ent[k - 1];
            pw = w + nw + (x.tp + 2) / 4;
          } else {
            for (uint32_t i = 0; i < nw; i++) {
              w[i] = x.flag_words[i];
              w[nw + i] = x.inc_words[i];
            }
            uint32_t *rw = w + 2 * nw;
            for (uint32_t r = 0; r < x.R; r++) put_bits(rw, (uint64_t)r * x.w, x.w, x.reuse[r]);
            pw = rw + (x.R * x.w + 31) / 32;
          }
          float P[3 * 256];  // decoded positions, for the normal cone
          for (uint32_t v = 0; v < x.V; v++)
            for (int c = 0; c < 3; c++) {
              double y = ((double)pos[3 * (size_t)x.gv[v] + c] - (double)G[c]) /
                         (double)delta[x.b][c];
              uint32_t q = (uint32_t)(std::floor(y + 0.5) - (double)x.L[c]);
              put_bits(pw, (3 * (uint64_t)v + c) * x.b, x.b, q);
              P[3 * v + c] = grid_to_float(x.L[c] + q, G[c], delta[x.b][c]);
            }
          if (n_attr) {
            uint32_t *aw = pw + (3 * x.V * x.b + 31) / 32;
            for (uint32_t v = 0; v < x.V; v++)
              for (uint32_t c = 0; c < n_attr; c++) {
                const double y = ((double)p->attrs[(size_t)n_attr * x.gv[v] + c] - (double)GA[c]) /
                                 (double)DA[c];
                const uint32_t q = (uint32_t)(std::floor(y + 0.5) - (double)x.La[c]);
                put_bits(aw, ((uint64_t)n_attr * v + c) * attr_bits, attr_bits, q);
              }
            mc_attr_desc &ad = blob->attr_desc[s];
            for (uint32_t c = 0; c < n_attr; c++) ad.La[c] = x.La[c];
          }
          {
            // the meshlet's input triangles in local ids (vertex -> local id
            // through a per-thread table over the mesh's vertices)
            thread_local std::vector<uint16_t> local_of;
            if (local_of.size() < n_verts) local_of.resize(n_verts);
            for (uint32_t v = 0; v < x.V; v++) local_of[x.gv[v]] = (uint16_t)v;
            const uint32_t mi = slot[s], t0 = m->start[mi], nt = m->start[mi + 1] - t0;
            uint32_t tl[3 * 256];
            for (uint32_t i = 0; i < 3 * nt; i++) tl[i] = local_of[m->corners[3 * (size_t)t0 + i]];
            blob->cones[s] = meshlet_cone(P, x.V, tl, nt);
          }
          mc_desc &d = blob->desc[s];
          d.payload_off16 = (uint32_t)(off[s] / 4);
          d.vertex_base = (uint32_t)vb[s];
          d.tri_base = (uint32_t)tb[s];
          d.n_verts = (uint16_t)x.V;
          d.n_tris = (uint16_t)x.tp;
          d.reuse_bits = (uint8_t)x.w;
          d.pos_bits = (uint8_t)x.b;
          d.grid = (uint16_t)grid_of[x.b];
          for (int c = 0; c < 3; c++) d.L[c] = x.L[c];
          std::memcpy(blob->vmap.data() + vb[s], x.gv.data(), x.V * sizeof(uint32_t));
        },
        256);

    if (n_attr) {
      mc_attr_grid ag{};
      for (uint32_t c = 0; c < n_attr; c++) {
        ag.G[c] = GA[c];
        ag.delta[c] = DA[c];
      }
      ag.attr_bits = attr_bits;
      ag.mesh_id = p->mesh_id;
      blob->attr_grids.push_back(ag);
    }
    blob->grids.resize(n_grids);
    for (uint32_t b = 1; b <= 32; b++) {
      if (!present[b]) continue;
      mc_grid &g = blob->grids[grid_of[b]];
      for (int c = 0; c < 3; c++) {
        g.G[c] = G[c];
        g.delta[c] = delta[b][c];
      }
      g.pos_bits = b;
      g.mesh_id = p->mesh_id;
    }
    mc_mesh_info mi{};
    mi.first_meshlet = 0;
    mi.n_meshlets = nm;
    mi.tri_base = 0;
    mi.n_tris = tb[nm];
    mi.vertex_base = 0;
    mi.n_verts = vb[nm];
    mi.input_tris = m->n_tris;
    blob->meshes.push_back(mi);
    blob->total_tris = tb[nm];
    blob->total_verts = vb[nm];
    blob->input_tris = m->n_tris;
    blob->split_meshlets = nm - m->n_grown;
    for (uint32_t i = 0; i < nm; i++) {
      const Packed &x = pk[i];
      blob->restarts += x.strips - 1;
      blob->conn_bits += x.w ? 2ull * x.tp + (uint64_t)x.w * x.R : x.tp + 8ull * (x.tp - 1);
      blob->pos_bits_total += 3ull * x.V * x.b;
      blob->max_block_words = std::max(blob->max_block_words, x.words);
      blob->max_tris = std::max(blob->max_tris, x.tp);
      blob->max_verts = std::max(blob->max_verts, x.V);
    }
  } catch (const std::bad_alloc &) {
    delete blob;
    return MC_ERR_OOM;
  }
  *out = blob;
  return MC_OK;
}

extern "C" mc_status mc_blob_concat(const mc_blob *const *blobs, uint32_t n, mc_blob **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!blobs || n == 0) return MC_ERR_INVALID_ARG;
  uint64_t nm = 0, pay = 0, ng = 0, nv = 0, nt = 0;
  for (uint32_t i = 0; i < n; i++) {
    if (!blobs[i]) return MC_ERR_INVALID_ARG;
    nm += blobs[i]->desc.size();
    pay += blobs[i]->payload.size();
    ng += blobs[i]->grids.size();
    nv += blobs[i]->total_verts;
    nt += blobs[i]->total_tris;
  }
  if (nm > 0xFFFFFFFFull || ng > 0xFFFF || nv > 0xFFFFFFFFull || nt > 0xFFFFFFFFull ||
      pay / 16 > 0xFFFFFFFFull)
    return MC_ERR_LIMIT;
  mc_blob *b = new (std::nothrow) mc_blob();
  if (!b) return MC_ERR_OOM;
  try {
    b->desc.reserve(nm);
    b->payload.reserve(pay);
    b->grids.reserve(ng);
    b->vmap.reserve(nv);
    b->cones.reserve(nm);
    b->n_attr = blobs[0]->n_attr;
    b->attr_bits = blobs[0]->attr_bits;
    for (uint32_t i = 0; i < n; i++)
      if (blobs[i]->n_attr != b->n_attr || blobs[i]->attr_bits != b->attr_bits) {
        delete b;
        return MC_ERR_INVALID_ARG;  // attribute channels must agree
      }
    uint64_t o16 = 0, vb = 0, tb = 0, gb = 0, mb = 0, ab = 0;
    for (uint32_t i = 0; i < n; i++) {
      const mc_blob *s = blobs[i];
      for (mc_desc d : s->desc) {
        d.payload_off16 += (uint32_t)o16;
        d.vertex_base += (uint32_t)vb;
        d.tri_base += (uint32_t)tb;
        d.grid = (uint16_t)(d.grid + gb);
        b->desc.push_back(d);
      }
      b->payload.insert(b->payload.end(), s->payload.begin(), s->payload.end());
      for (mc_grid g : s->grids) {
        g.mesh_id = i;
        b->grids.push_back(g);
      }
      for (mc_mesh_info mi : s->meshes) {
        mi.first_meshlet += (uint32_t)mb;
        mi.tri_base += tb;
        mi.vertex_base += vb;
        b->meshes.push_back(mi);
      }
      b->vmap.insert(b->vmap.end(), s->vmap.begin(), s->vmap.end());
      b->cones.insert(b->cones.end(), s->cones.begin(), s->cones.end());
      for (mc_attr_desc ad : s->attr_desc) {
        ad.grid = (uint16_t)(ad.grid + ab);
        b->attr_desc.push_back(ad);
      }
      for (mc_attr_grid ag : s->attr_grids) {
        ag.mesh_id = i;
        b->attr_grids.push_back(ag);
      }
      ab += s->attr_grids.size();
      o16 += s->payload.size() / 16;
      vb += s->total_verts;
      tb += s->total_tris;
      gb += s->grids.size();
      mb += s->desc.size();
      b->input_tris += s->input_tris;
      b->restarts += s->restarts;
      b->split_meshlets += s->split_meshlets;
      b->conn_bits += s->conn_bits;
      b->pos_bits_total += s->pos_bits_total;
      b->max_block_words = std::max(b->max_block_words, s->max_block_words);
      b->max_tris = std::max(b->max_tris, s->max_tris);
      b->max_verts = std::max(b->max_verts, s->max_verts);
    }
    b->total_tris = tb;
    b->total_verts = vb;
  } catch (const std::bad_alloc &) {
    delete b;
    return MC_ERR_OOM;
  }
  *out = b;
  return MC_OK;
}

extern "C" mc_status mc_blob_view(const mc_blob *b, mc_blob_view_t *v) {
  if (!b || !v) return MC_ERR_INVALID_ARG;
  std::memset(v, 0, sizeof(*v));
  v->desc = b->desc.data();
  v->n_meshlets = (uint32_t)b->desc.size();
  v->payload = b->payload.data();
  v->payload_bytes = b->payload.size();
  v->grids = b->grids.data();
  v->n_grids = (uint32_t)b->grids.size();
  v->meshes = b->meshes.data();
  v->n_meshes = (uint32_t)b->meshes.size();
  v->vertex_map = b->vmap.data();
  v->total_tris = b->total_tris;
  v->total_verts = b->total_verts;
  v->input_tris = b->input_tris;
  v->restarts = b->restarts;
  v->split_meshlets = b->split_meshlets;
  v->conn_bits = b->conn_bits;
  v->pos_bits_total = b->pos_bits_total;
  v->max_block_words = b->max_block_words;
  v->max_tris = b->max_tris;
  v->max_verts = b->max_verts;
  v->cones = b->cones.data();
  v->n_attr = b->n_attr;
  v->attr_bits = b->attr_bits;
  v->attr_desc = b->attr_desc.empty() ? nullptr : b->attr_desc.data();
  v->attr_grids = b->attr_grids.empty() ? nullptr : b->attr_grids.data();
  v->n_attr_grids = (uint32_t)b->attr_grids.size();
  return MC_OK;
}

extern "C" void mc_blob_free(mc_blob *b) { delete b; }

extern "C" const char *mc_status_string(mc_status s) {
  switch (s) {
    case MC_OK: return "MC_OK";
    case MC_ERR_INVALID_ARG: return "MC_ERR_INVALID_ARG";
    case MC_ERR_LIMIT: return "MC_ERR_LIMIT";
    case MC_ERR_CORRUPT: return "MC_ERR_CORRUPT";
    case MC_ERR_CUDA: return "MC_ERR_CUDA";
    case MC_ERR_OOM: return "MC_ERR_OOM";
    case MC_ERR_TIMEOUT: return "MC_ERR_TIMEOUT";
  }
  return "MC_ERR_UNKNOWN";
}

extern "C" const char *mc_version(void) { return "meshlet-codec 0.1 (sm_103a)"; }
