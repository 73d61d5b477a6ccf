/*
 * Oracle: generalized triangle strips of one meshlet.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Strip semantics (Sec. 2): a strip enters triangle (a,b,c) through its edge
 * (a,b) and leaves across the right edge (b,c) or the left edge (c,a); the
 * L/R flag of the next triangle records which.  Keeping the counter-clockwise
 * winding of the mesh, the triangle across the right edge is (c,b,x) and the
 * one across the left edge is (a,c,x), x being its one new vertex.  Any
 * simple path in the triangles' edge-adjacency graph is therefore one strip,
 * and the strips of a meshlet are a path cover of that graph.
 *
 * The paper finds a minimum path cover with a MILP (Sec. 4.1, Eq. 1-3); that
 * needs a commercial solver and is not restated.  Instead, the best of
 * K_TRIES randomised greedy covers (fewest strips, the first on ties):
 *   - a strip starts at an unvisited triangle with the fewest unvisited
 *     neighbours (a random one among the ties, in list order);
 *   - it grows at its end into an unvisited neighbour with the fewest
 *     unvisited neighbours (a random one among the ties, in edge order);
 *   - when stuck it may rotate (Posa): if its end is adjacent to the strip
 *     member at position k (k < length - 2), the part after k is reversed,
 *     making the former successor of k the end -- at most R_ROTATIONS times
 *     per strip, choosing at random among the members adjacent to the end;
 *   - it then grows the same way from its other end, and is emitted as it
 *     stands.
 * Random numbers come from SplitMix64 (Steele, Lea, Flood 2014: the state
 * advances by 0x9E3779B97F4A7C15 and is mixed by two xor-shift-multiply
 * rounds), seeded per meshlet with first-triangle-id * 0x9E3779B97F4A7C15 + T;
 * a choice among n candidates takes the next number modulo n.
 * Two triangles are adjacent across edge e = (v_e -> v_{e+1}) of the first
 * when the second is the lowest list position holding the opposite directed
 * edge and the first is likewise a neighbour of the second (mutual pairs).
 *
 * The first triangle of a strip is rotated so that its entry edge is the
 * first of its edges (input order) that does not lead to the next triangle.
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
#define K_TRIES 16
#define R_ROTATIONS 32

static uint64_t splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct {
  const int32_t *adj; /* adj[3t+e]: mutual neighbour across edge e, or -1 */
  uint8_t *vis;
  int32_t *pos;       /* position in the current strip, -1 if not in it */
  uint32_t *path;
  uint32_t len;
} cover_t;

static uint32_t free_deg(const cover_t *c, uint32_t t) {
  uint32_t n = 0;
  for (int e = 0; e < 3; e++) {
    int32_t j = c->adj[3 * t + e];
    if (j >= 0 && !c->vis[j]) n++;
  }
  return n;
}

static void reverse_from(cover_t *c, uint32_t from) {
  for (uint32_t i = from, j = c->len - 1; i < j; i++, j--) {
    uint32_t x = c->path[i];
    c->path[i] = c->path[j];
    c->path[j] = x;
  }
  for (uint32_t i = from; i < c->len; i++) c->pos[c->path[i]] = (int32_t)i;
}

/* One randomised cover; writes the strips' triangles to order (concatenated)
 * and each strip's length to lens; returns the number of strips. */
static uint32_t one_cover(cover_t *c, uint32_t T, uint64_t *rng, uint32_t *order, uint32_t *lens) {
  memset(c->vis, 0, T);
  for (uint32_t t = 0; t < T; t++) c->pos[t] = -1;
  uint32_t covered = 0, n_strips = 0, n_order = 0;
  while (covered < T) {
    uint32_t best = 4, ties = 0;
    for (uint32_t t = 0; t < T; t++) {
      if (c->vis[t]) continue;
      uint32_t d = free_deg(c, t);
      if (d < best) { best = d; ties = 1; }
      else if (d == best) ties++;
    }
    uint32_t pick = (uint32_t)(splitmix64(rng) % ties), start = 0;
    for (uint32_t t = 0; t < T; t++) {
      if (c->vis[t] || free_deg(c, t) != best) continue;
      if (pick-- == 0) { start = t; break; }
    }
    c->len = 0;
    c->path[c->len++] = start;
    c->pos[start] = 0;
    c->vis[start] = 1;
    covered++;
    uint32_t rotations = 0;
    for (int side = 0; side < 2; side++) {
      for (;;) {
        uint32_t cur = c->path[c->len - 1];
        uint32_t cand[3], dmin = 4, n = 0;
        for (int e = 0; e < 3; e++) {
          int32_t j = c->adj[3 * cur + e];
          if (j < 0 || c->vis[j]) continue;
          uint32_t d = free_deg(c, (uint32_t)j);
          if (d < dmin) { dmin = d; n = 0; }
          if (d == dmin) cand[n++] = (uint32_t)j;
        }
        if (n) {
          uint32_t j = cand[splitmix64(rng) % n];
          c->pos[j] = (int32_t)c->len;
          c->path[c->len++] = j;
          c->vis[j] = 1;
          covered++;
          continue;
        }
        if (rotations == R_ROTATIONS) break;
        uint32_t opt[3], m = 0;
        for (int e = 0; e < 3; e++) {
          int32_t y = c->adj[3 * cur + e];
          if (y >= 0 && c->pos[y] >= 0 && (uint32_t)c->pos[y] + 2 < c->len) opt[m++] = (uint32_t)c->pos[y];
        }
        if (!m) break;
        reverse_from(c, opt[splitmix64(rng) % m] + 1);
        rotations++;
      }
      reverse_from(c, 0);
    }
    for (uint32_t i = 0; i < c->len; i++) {
      order[n_order++] = c->path[i];
      c->pos[c->path[i]] = -1;
    }
    lens[n_strips++] = c->len;
  }
  return n_strips;
}

int orc_stripify(const uint32_t *tris, const uint32_t *ids, uint32_t T,
                 uint32_t *stream, uint8_t *flags, uint32_t *strip_order,
                 uint32_t *out_tp, uint32_t *out_strips) {
  if (!tris || !ids || !stream || !flags || !strip_order || T == 0) return ORC_ERR_ARG;
  int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
  int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
  uint8_t *vis = (uint8_t *)malloc(T);
  int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * T);
  uint32_t *path = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint32_t *lens = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint32_t *best_lens = (uint32_t *)malloc(sizeof(uint32_t) * T);
  if (!nb || !adj || !vis || !pos || !path || !order || !lens || !best_lens) {
    free(nb); free(adj); free(vis); free(pos); free(path); free(order); free(lens); free(best_lens);
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
  /* mutual pairs only */
  for (uint32_t i = 0; i < T; i++)
    for (int e = 0; e < 3; e++) {
      int32_t j = nb[3 * i + e];
      int mutual = 0;
      if (j >= 0)
        for (int f = 0; f < 3; f++) mutual |= nb[3 * (uint32_t)j + f] == (int32_t)i;
      adj[3 * i + e] = mutual ? j : -1;
    }

  cover_t c = {adj, vis, pos, path, 0};
  uint64_t rng = (uint64_t)ids[0] * 0x9E3779B97F4A7C15ull + T;
  uint32_t best_strips = 0;
  for (int k = 0; k < K_TRIES; k++) {
    uint32_t n = one_cover(&c, T, &rng, order, lens);
    if (k == 0 || n < best_strips) {
      best_strips = n;
      memcpy(strip_order, order, sizeof(uint32_t) * T);
      memcpy(best_lens, lens, sizeof(uint32_t) * n);
    }
  }

  /* emission */
  uint32_t n_stream = 0, tp = 0, at = 0;
  for (uint32_t s = 0; s < best_strips; s++) {
    const uint32_t *p = strip_order + at;
    uint32_t len = best_lens[s];
    at += len;
    /* entry rotation of the first triangle: first edge not leading to p[1] */
    int rot = 0;
    if (len > 1)
      while (rot < 3 && adj[3 * p[0] + rot] == (int32_t)p[1]) rot++;
    uint32_t a = V_OF(p[0], rot), b = V_OF(p[0], rot + 1), cc = V_OF(p[0], rot + 2);
    if (s == 0) {
      stream[n_stream++] = a;
      stream[n_stream++] = b;
      stream[n_stream++] = cc;
      flags[tp++] = 0;
    } else {
      uint32_t last = stream[n_stream - 1];
      const uint32_t ent[5] = {last, a, a, b, cc};
      const uint8_t fl[5] = {0, 1, 1, 0, 0};
      for (int i = 0; i < 5; i++) {
        stream[n_stream++] = ent[i];
        flags[tp++] = fl[i];
      }
    }
    int cr = rot;
    for (uint32_t i = 0; i + 1 < len; i++) {
      uint32_t cur = p[i], nxt = p[i + 1];
      int eR = (cr + 1) % 3, eL = (cr + 2) % 3, go_right;
      if (adj[3 * cur + eR] == (int32_t)nxt) go_right = 1;
      else if (adj[3 * cur + eL] == (int32_t)nxt) go_right = 0;
      else break; /* cannot happen for a path of mutual neighbours */
      uint32_t e0 = go_right ? cc : a, e1 = go_right ? b : cc;
      int f = -1;
      for (int k = 0; k < 3; k++)
        if (V_OF(nxt, k) == e0 && V_OF(nxt, k + 1) == e1) { f = k; break; }
      if (f < 0) break;
      uint32_t x = V_OF(nxt, f + 2);
      a = e0; b = e1; cc = x;
      stream[n_stream++] = x;
      flags[tp++] = (uint8_t)go_right;
      cr = f;
    }
  }
  free(nb); free(adj); free(vis); free(pos); free(path); free(order); free(lens); free(best_lens);
  if (tp != T + 4 * (best_strips - 1)) return ORC_ERR_CORRUPT;
  *out_tp = tp;
  if (out_strips) *out_strips = best_strips;
  return ORC_OK;
}
