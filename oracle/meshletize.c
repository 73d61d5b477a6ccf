/*
 * Oracle: greedy meshletization (Sec. 3) and the meshlet split of Sec. 4.2.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper takes its meshlets from a third-party splitter; this oracle uses
 * a small deterministic greedy rule instead:
 *   - seed: the lowest-index unassigned triangle; its class fixes the limits;
 *   - frontier: unassigned same-class triangles sharing an edge with the
 *     meshlet, numbered in the order they join the frontier (edges of a newly
 *     added triangle visited as (v0,v1), (v1,v2), (v2,v0); the triangles on
 *     one edge in increasing id);
 *   - pick: the frontier triangle that adds the fewest new vertices (0 or 1:
 *     a frontier triangle adds at most one); among those, the one with the
 *     most edges already shared with an assigned triangle of its class (any
 *     meshlet: this takes triangles that would otherwise be left stranded
 *     between full meshlets first); among those, the earliest-joined;
 *   - stop when the pick would exceed V~ vertices or T~ triangles.
 * A meshlet whose strip (restart degenerates included) is longer than T~ is
 * split into the first ceil(T/2) triangles of its strip order and the rest,
 * recursively (Sec. 4.2: restart degenerates can push a meshlet past T~,
 * which forces a split).
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* vertex -> incident triangles, ascending triangle id */
static int vertex_triangles(uint32_t nv, const uint32_t *tri, uint32_t nt,
                            uint32_t **off_out, uint32_t **lst_out) {
  uint32_t *off = (uint32_t *)calloc((size_t)nv + 1, sizeof(uint32_t));
  uint32_t *lst = (uint32_t *)malloc(((size_t)nt * 3 + 1) * sizeof(uint32_t));
  uint32_t *fill = (uint32_t *)calloc((size_t)nv + 1, sizeof(uint32_t));
  if (!off || !lst || !fill) {
    free(off); free(lst); free(fill);
    return ORC_ERR_NOMEM;
  }
  for (size_t i = 0; i < (size_t)nt * 3; i++) off[tri[i] + 1]++;
  for (uint32_t v = 0; v < nv; v++) off[v + 1] += off[v];
  for (uint32_t t = 0; t < nt; t++)
    for (int i = 0; i < 3; i++) {
      uint32_t v = tri[3 * (size_t)t + i];
      lst[off[v] + fill[v]++] = t;
    }
  free(fill);
  *off_out = off;
  *lst_out = lst;
  return ORC_OK;
}

static int has_vertex(const uint32_t *tri, uint32_t t, uint32_t v) {
  return tri[3 * (size_t)t] == v || tri[3 * (size_t)t + 1] == v ||
         tri[3 * (size_t)t + 2] == v;
}

/* Edges of triangle t that an assigned triangle of the same class shares. */
static uint32_t assigned_edges(const uint32_t *tri, const uint8_t *tri_class, uint32_t t,
                               const uint32_t *vt_off, const uint32_t *vt,
                               const uint8_t *assigned) {
  uint32_t n = 0, cls = tri_class ? tri_class[t] : 0;
  for (int e = 0; e < 3; e++) {
    uint32_t u = tri[3 * (size_t)t + e], w = tri[3 * (size_t)t + (e + 1) % 3];
    for (uint32_t k = vt_off[u]; k < vt_off[u + 1]; k++) {
      uint32_t t3 = vt[k];
      if (t3 != t && assigned[t3] && (tri_class ? tri_class[t3] : 0) == cls &&
          has_vertex(tri, t3, w)) {
        n++;
        break;
      }
    }
  }
  return n;
}

/* Split driver: appends the final meshlets for the triangle list ids[0..T). */
static int emit_final(const uint32_t *tris, const uint32_t *ids, uint32_t T,
                      uint32_t max_tris, uint32_t *out_tri, uint32_t *out_start,
                      uint32_t *n_out_tri, uint32_t *n_meshlets) {
  uint32_t *stream = (uint32_t *)malloc(sizeof(uint32_t) * (5 * (size_t)T + 8));
  uint8_t *flags = (uint8_t *)malloc(5 * (size_t)T + 8);
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)T + 1));
  uint32_t tp = 0, strips = 0;
  int rc = ORC_ERR_NOMEM;
  if (!stream || !flags || !order) goto done;
  rc = orc_stripify(tris, ids, T, 0, stream, flags, order, &tp, &strips);
  if (rc != ORC_OK) goto done;
  if (tp <= max_tris) {
    out_start[*n_meshlets] = *n_out_tri;
    (*n_meshlets)++;
    for (uint32_t i = 0; i < T; i++) out_tri[(*n_out_tri)++] = ids[i];
  } else {
    /* halves of the strip order */
    uint32_t h = (T + 1) / 2;
    uint32_t *sub = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)T + 1));
    if (!sub) { rc = ORC_ERR_NOMEM; goto done; }
    for (uint32_t i = 0; i < T; i++) sub[i] = ids[order[i]];
    rc = emit_final(tris, sub, h, max_tris, out_tri, out_start, n_out_tri, n_meshlets);
    if (rc == ORC_OK)
      rc = emit_final(tris, sub + h, T - h, max_tris, out_tri, out_start, n_out_tri,
                      n_meshlets);
    free(sub);
  }
done:
  free(stream); free(flags); free(order);
  return rc;
}

int orc_meshletize(uint32_t n_verts, const uint32_t *tris, uint32_t n_tris,
                   const uint8_t *tri_class, const uint32_t *limits,
                   uint32_t n_classes, uint32_t *out_tri, uint32_t *out_start,
                   uint32_t *out_n_meshlets, uint32_t *out_n_grown) {
  if (!tris || !limits || !out_tri || !out_start || !out_n_meshlets || n_classes == 0)
    return ORC_ERR_ARG;
  for (uint32_t c = 0; c < n_classes; c++)
    if (limits[2 * c] < 3 || limits[2 * c] > 256 || limits[2 * c + 1] < 1 ||
        limits[2 * c + 1] > 256)
      return ORC_ERR_ARG;
  for (uint32_t t = 0; t < n_tris; t++) {
    uint32_t a = tris[3 * (size_t)t], b = tris[3 * (size_t)t + 1], c = tris[3 * (size_t)t + 2];
    if (a >= n_verts || b >= n_verts || c >= n_verts || a == b || b == c || a == c)
      return ORC_ERR_ARG;
    if (tri_class && tri_class[t] >= n_classes) return ORC_ERR_ARG;
  }

  uint32_t *vt_off = NULL, *vt = NULL;
  int rc = vertex_triangles(n_verts, tris, n_tris, &vt_off, &vt);
  if (rc != ORC_OK) return rc;
  uint8_t *assigned = (uint8_t *)calloc((size_t)n_tris + 1, 1);
  uint32_t *fstamp = (uint32_t *)calloc((size_t)n_tris + 1, sizeof(uint32_t));
  uint32_t *vstamp = (uint32_t *)calloc((size_t)n_verts + 1, sizeof(uint32_t));
  uint32_t *front = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n_tris + 1));
  uint32_t *grown = (uint32_t *)malloc(sizeof(uint32_t) * 257);
  if (!assigned || !fstamp || !vstamp || !front || !grown) {
    rc = ORC_ERR_NOMEM;
    goto done;
  }

  uint32_t seed_scan = 0, n_grown = 0, n_final = 0, n_out = 0;
  for (;;) {
    while (seed_scan < n_tris && assigned[seed_scan]) seed_scan++;
    if (seed_scan == n_tris) break;
    uint32_t stamp = n_grown + 1;
    uint32_t cls = tri_class ? tri_class[seed_scan] : 0;
    uint32_t max_v = limits[2 * cls], max_t = limits[2 * cls + 1];
    uint32_t nf = 0, nV = 0, nT = 0;
    uint32_t t = seed_scan;
    for (;;) {
      /* add t */
      assigned[t] = 1;
      grown[nT++] = t;
      for (int i = 0; i < 3; i++) {
        uint32_t v = tris[3 * (size_t)t + i];
        if (vstamp[v] != stamp) { vstamp[v] = stamp; nV++; }
      }
      for (int e = 0; e < 3; e++) {
        uint32_t u = tris[3 * (size_t)t + e], w = tris[3 * (size_t)t + (e + 1) % 3];
        for (uint32_t k = vt_off[u]; k < vt_off[u + 1]; k++) {
          uint32_t t2 = vt[k];
          if (t2 == t || assigned[t2] || fstamp[t2] == stamp) continue;
          if ((tri_class ? tri_class[t2] : 0) != cls) continue;
          if (!has_vertex(tris, t2, w)) continue;
          fstamp[t2] = stamp;
          front[nf++] = t2;
        }
      }
      /* pick: fewest new vertices, then most assigned edges, then earliest */
      int64_t best = -1;
      uint32_t best_cost = 0, best_nb = 0;
      for (uint32_t i = 0; i < nf; i++) {
        uint32_t t2 = front[i];
        if (assigned[t2]) continue;
        uint32_t cost = 0;
        for (int j = 0; j < 3; j++) cost += vstamp[tris[3 * (size_t)t2 + j]] != stamp;
        uint32_t nb = assigned_edges(tris, tri_class, t2, vt_off, vt, assigned);
        if (best < 0 || cost < best_cost || (cost == best_cost && nb > best_nb)) {
          best = t2;
          best_cost = cost;
          best_nb = nb;
        }
      }
      if (best < 0) break;
      if (nT + 1 > max_t || nV + best_cost > max_v) break;
      t = (uint32_t)best;
    }
    n_grown++;
    rc = emit_final(tris, grown, nT, max_t, out_tri, out_start, &n_out, &n_final);
    if (rc != ORC_OK) goto done;
  }
  out_start[n_final] = n_out;
  *out_n_meshlets = n_final;
  if (out_n_grown) *out_n_grown = n_grown;
  rc = ORC_OK;
done:
  free(vt_off); free(vt); free(assigned); free(fstamp); free(vstamp);
  free(front); free(grown);
  return rc;
}
