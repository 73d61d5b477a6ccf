/*
 * Oracle: greedy generalized triangle strip of one meshlet.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Strip semantics (Sec. 2): a strip enters triangle (a,b,c) through its edge
 * (a,b) and leaves across the right edge (b,c) or the left edge (c,a); the
 * L/R flag of the next triangle records which.  Keeping the counter-clockwise
 * winding of the mesh, the triangle across the right edge is (c,b,x) and the
 * one across the left edge is (a,c,x), x being its one new vertex.
 *
 * The paper finds optimal strips with a MILP (Sec. 4.1, Eq. 1-3); that needs
 * a commercial solver and is not restated.  This greedy rule stands in:
 *   - start a strip at the unvisited triangle with the fewest unvisited
 *     neighbours (ties: lowest list position), rotated so that its entry edge
 *     has no unvisited neighbour (first such rotation of (v0,v1,v2),
 *     (v1,v2,v0), (v2,v0,v1); else the first);
 *   - continue across the right or left edge into an unvisited neighbour;
 *     if both exist take the one with fewer unvisited neighbours (ties: R);
 *   - when stuck, restart.
 * A restart is emulated by four degenerate triangles (Sec. 4.2): after the
 * strip's last triangle (a,b,c) the stream continues with the entries
 * c, p, p, q, r flagged L, R, R, L, L, where (p,q,r) is the next strip's first
 * triangle.  Walking the strip rule gives (a,c,c), (c,c,p), (p,c,p), (p,p,q)
 * (all degenerate) and then (p,q,r), whatever (a,b,c) was.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define V_OF(t, i) (tris[3 * (size_t)ids[(t)] + ((i) % 3)])

int orc_stripify(const uint32_t *tris, const uint32_t *ids, uint32_t T,
                 uint32_t *stream, uint8_t *flags, uint32_t *strip_order,
                 uint32_t *out_tp, uint32_t *out_strips) {
  if (!tris || !ids || !stream || !flags || !strip_order || T == 0) return ORC_ERR_ARG;
  int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
  uint8_t *visited = (uint8_t *)calloc(T, 1);
  if (!nb || !visited) {
    free(nb); free(visited);
    return ORC_ERR_NOMEM;
  }
  /* nb[3i+e]: the lowest list position j != i whose triangle has the
   * directed edge opposite to edge e = (v_e -> v_{e+1}) of triangle i */
  for (uint32_t i = 0; i < T; i++)
    for (int e = 0; e < 3; e++) {
      uint32_t x = V_OF(i, e), y = V_OF(i, e + 1);
      nb[3 * i + e] = -1;
      for (uint32_t j = 0; j < T && nb[3 * i + e] < 0; j++) {
        if (j == i) continue;
        for (int f = 0; f < 3; f++)
          if (V_OF(j, f) == y && V_OF(j, f + 1) == x) { nb[3 * i + e] = (int32_t)j; break; }
      }
    }

#define FREE_NB(i, e) (nb[3 * (i) + (e)] >= 0 && !visited[nb[3 * (i) + (e)]])
#define UNVISITED_NB(i) (FREE_NB(i, 0) + FREE_NB(i, 1) + FREE_NB(i, 2))

  uint32_t n_stream = 0, tp = 0, n_strips = 0, count = 0;
  while (count < T) {
    /* start triangle */
    uint32_t start = T, best_u = 4;
    for (uint32_t i = 0; i < T; i++) {
      if (visited[i]) continue;
      uint32_t u = (uint32_t)UNVISITED_NB(i);
      if (u < best_u) { best_u = u; start = i; }
    }
    int rot = 0;
    for (int r = 0; r < 3; r++)
      if (!FREE_NB(start, r)) { rot = r; break; }
    uint32_t a = V_OF(start, rot), b = V_OF(start, rot + 1), c = V_OF(start, rot + 2);
    if (n_strips == 0) {
      stream[n_stream++] = a;
      stream[n_stream++] = b;
      stream[n_stream++] = c;
      flags[tp++] = 0;
    } else {
      uint32_t last = stream[n_stream - 1];
      const uint32_t ent[5] = {last, a, a, b, c};
      const uint8_t fl[5] = {0, 1, 1, 0, 0};
      for (int i = 0; i < 5; i++) {
        stream[n_stream++] = ent[i];
        flags[tp++] = fl[i];
      }
    }
    n_strips++;
    visited[start] = 1;
    strip_order[count++] = start;
    uint32_t cur = start;
    int cr = rot;
    for (;;) {
      int eR = (cr + 1) % 3, eL = (cr + 2) % 3;
      int32_t tR = FREE_NB(cur, eR) ? nb[3 * cur + eR] : -1;
      int32_t tL = FREE_NB(cur, eL) ? nb[3 * cur + eL] : -1;
      if (tR < 0 && tL < 0) break;
      int go_right;
      if (tR >= 0 && tL >= 0)
        go_right = UNVISITED_NB((uint32_t)tR) <= UNVISITED_NB((uint32_t)tL);
      else
        go_right = tR >= 0;
      uint32_t nxt = (uint32_t)(go_right ? tR : tL);
      /* entry edge of the next triangle: (c,b) for R, (a,c) for L */
      uint32_t e0 = go_right ? c : a, e1 = go_right ? b : c;
      int f = -1;
      for (int k = 0; k < 3; k++)
        if (V_OF(nxt, k) == e0 && V_OF(nxt, k + 1) == e1) { f = k; break; }
      if (f < 0) { free(nb); free(visited); return ORC_ERR_CORRUPT; }
      uint32_t x = V_OF(nxt, f + 2);
      a = e0; b = e1; c = x;
      stream[n_stream++] = x;
      flags[tp++] = (uint8_t)go_right;
      visited[nxt] = 1;
      strip_order[count++] = nxt;
      cur = nxt;
      cr = f;
    }
  }
#undef FREE_NB
#undef UNVISITED_NB
  free(nb);
  free(visited);
  *out_tp = tp;
  if (out_strips) *out_strips = n_strips;
  return ORC_OK;
}
