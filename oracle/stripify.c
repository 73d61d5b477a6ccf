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

/* adj[3i+e] for the triangles ids[0..T): the mutual neighbour across edge
 * e = (v_e -> v_{e+1}) of triangle i, or -1.  nb is scratch (3T entries):
 * nb[3i+e] = the lowest list position j != i whose triangle has the directed
 * edge opposite to edge e; only mutual pairs count as adjacent. */
static void build_adjacency(const uint32_t *tris, const uint32_t *ids, uint32_t T, int32_t *nb,
                            int32_t *adj) {
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
  for (uint32_t i = 0; i < T; i++)
    for (int e = 0; e < 3; e++) {
      int32_t j = nb[3 * i + e];
      int mutual = 0;
      if (j >= 0)
        for (int f = 0; f < 3; f++) mutual |= nb[3 * (uint32_t)j + f] == (int32_t)i;
      adj[3 * i + e] = mutual ? j : -1;
    }
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

/* ------------------------------------------------------------------------
 * Fewest strips of a meshlet, exactly, for small meshlets.
 *
 * The strips are a path cover of the adjacency graph (above), so the fewest
 * strips is T minus the largest set of adjacency edges that forms paths only
 * -- every triangle on at most two chosen edges (a strip does not fork) and
 * no cycle (Sec. 4.1 maximises the same count of used edges under the same
 * two conditions).  Found by depth-first branch and bound over the edges in
 * list order (take the edge if it keeps every chosen set a path, then leave
 * it out), pruned by the count that is still reachable: every triangle can
 * gain at most min(2 - its chosen edges, its undecided edges), and an edge
 * serves two triangles.  The search starts from the greedy cover's count.
 * A chosen edge (u, v) may join two paths only at their ends and never the
 * two ends of one path; the ends of every path are tracked to test that.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_edges, n_nodes, max_nodes;
  const uint32_t (*edge)[2];
  uint8_t *deg;        /* chosen edges at each triangle */
  uint32_t *end;       /* end[x]: the other end of the path x ends (x itself alone) */
  uint32_t *rem;       /* rem[x]: undecided edges at x */
  uint8_t *sel;        /* sel[i]: edge i chosen on the current branch */
  uint8_t *best_sel;   /* the choice of the best cover found (may be NULL) */
  uint32_t chosen, best;
  int aborted, improved;
} search_t;

static uint32_t reachable(const search_t *s, uint32_t T) {
  uint32_t sum = 0;
  for (uint32_t x = 0; x < T; x++) {
    uint32_t room = 2u - s->deg[x];
    sum += s->rem[x] < room ? s->rem[x] : room;
  }
  return sum / 2;
}

static void search(search_t *s, uint32_t T, uint32_t i) {
  if (s->aborted) return;
  if (++s->n_nodes > s->max_nodes) { s->aborted = 1; return; }
  if (s->chosen > s->best) {
    s->best = s->chosen;
    s->improved = 1;
    if (s->best_sel) memcpy(s->best_sel, s->sel, s->n_edges);
  }
  if (i == s->n_edges) return;
  if (s->chosen + reachable(s, T) <= s->best) return;
  const uint32_t u = s->edge[i][0], v = s->edge[i][1];
  s->rem[u]--;
  s->rem[v]--;
  if (s->deg[u] < 2 && s->deg[v] < 2 && s->end[u] != v) {
    const uint32_t a = s->end[u], b = s->end[v];  /* the new path runs a .. u - v .. b */
    s->deg[u]++;
    s->deg[v]++;
    s->end[a] = b;
    s->end[b] = a;
    s->chosen++;
    s->sel[i] = 1;
    search(s, T, i + 1);
    s->sel[i] = 0;
    s->chosen--;
    s->end[a] = u;  /* undo: u and v end their own paths again */
    s->end[b] = v;
    s->end[u] = a;
    s->end[v] = b;
    s->deg[u]--;
    s->deg[v]--;
  }
  search(s, T, i + 1);
  s->rem[u]++;
  s->rem[v]++;
}

/* The adjacency edges (i, j), i < j, in the order of i, then of i's edge
 * slots; rem[x] = the edges at x.  Returns their count. */
static uint32_t edge_list(const int32_t *adj, uint32_t T, uint32_t (*edge)[2], uint32_t *rem) {
  uint32_t n_edges = 0;
  for (uint32_t i = 0; i < T; i++) rem[i] = 0;
  for (uint32_t i = 0; i < T; i++)
    for (int e = 0; e < 3; e++) {
      int32_t j = adj[3 * i + e];
      if (j > (int32_t)i) {
        edge[n_edges][0] = i;
        edge[n_edges][1] = (uint32_t)j;
        n_edges++;
        rem[i]++;
        rem[j]++;
      }
    }
  return n_edges;
}

/* Runs the search over the adjacency adj from an incumbent of T - strips
 * chosen edges.  Returns the number of edges of the best cover found (the
 * incumbent's if none is better), with its choice in best_sel when one was
 * better (*improved), and whether the search ended within max_nodes. */
static int search_cover(const int32_t *adj, uint32_t T, uint32_t strips, uint32_t max_nodes,
                        uint8_t *best_sel_out, uint32_t *n_edges_out, uint32_t (**edges_out)[2],
                        uint32_t *best_out, int *improved_out, int *finished_out) {
  uint32_t (*edge)[2] = (uint32_t(*)[2])malloc(sizeof(uint32_t) * 3 * (size_t)T);
  uint8_t *deg = (uint8_t *)calloc(T, 1);
  uint32_t *end = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint32_t *rem = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint8_t *sel = (uint8_t *)calloc(3 * (size_t)T, 1);
  if (!edge || !deg || !end || !rem || !sel) {
    free(edge); free(deg); free(end); free(rem); free(sel);
    return ORC_ERR_NOMEM;
  }
  uint32_t n_edges = edge_list(adj, T, edge, rem);
  for (uint32_t i = 0; i < T; i++) end[i] = i;
  search_t s = {n_edges, 0, max_nodes, (const uint32_t(*)[2])edge, deg, end, rem, sel,
                best_sel_out, 0, T - strips, 0, 0};
  if (max_nodes) search(&s, T, 0);
  *best_out = s.best;
  *improved_out = s.improved;
  *finished_out = max_nodes && !s.aborted;
  *n_edges_out = n_edges;
  if (edges_out) *edges_out = edge; else free(edge);
  free(deg); free(end); free(rem); free(sel);
  return ORC_OK;
}

/* The strips of a chosen edge set (every triangle on at most two chosen
 * edges, no cycle): from each triangle in list order that ends a path (at
 * most one chosen edge) and is not yet emitted, the path is walked to its
 * other end; order and lens as one_cover writes them.  Returns the number of
 * strips. */
static uint32_t paths_of(const int32_t *adj, uint32_t T, uint32_t n_edges, const uint32_t (*edge)[2],
                         const uint8_t *sel, uint8_t *vis, uint32_t *order, uint32_t *lens) {
  /* chosen neighbours: up to two per triangle, -1 for none */
  int32_t *cn = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)T);
  if (!cn) return 0;
  for (uint32_t i = 0; i < 2 * T; i++) cn[i] = -1;
  for (uint32_t i = 0; i < n_edges; i++) {
    if (!sel[i]) continue;
    uint32_t u = edge[i][0], v = edge[i][1];
    cn[2 * u + (cn[2 * u] >= 0)] = (int32_t)v;
    cn[2 * v + (cn[2 * v] >= 0)] = (int32_t)u;
  }
  (void)adj;
  memset(vis, 0, T);
  uint32_t n_order = 0, n_strips = 0;
  for (uint32_t t = 0; t < T; t++) {
    if (vis[t] || (cn[2 * t] >= 0 && cn[2 * t + 1] >= 0)) continue;
    uint32_t len = 0;
    int32_t prev = -1, cur = (int32_t)t;
    while (cur >= 0) {
      vis[cur] = 1;
      order[n_order++] = (uint32_t)cur;
      len++;
      int32_t nxt = cn[2 * cur] != prev ? cn[2 * cur] : cn[2 * cur + 1];
      if (nxt >= 0 && vis[nxt]) nxt = -1;
      prev = cur;
      cur = nxt;
    }
    lens[n_strips++] = len;
  }
  free(cn);
  return n_order == T ? n_strips : 0;
}

int orc_stripify(const uint32_t *tris, const uint32_t *ids, uint32_t T, uint32_t search_nodes,
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
  build_adjacency(tris, ids, T, nb, adj);

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

  /* optional search for fewer strips, from the greedy cover */
  if (search_nodes && best_strips > 1) {
    uint8_t *best_sel = (uint8_t *)calloc(3 * (size_t)T, 1);
    uint32_t n_edges = 0, best = 0;
    uint32_t (*edge)[2] = NULL;
    int improved = 0, finished = 0;
    int rc = best_sel ? search_cover(adj, T, best_strips, search_nodes, best_sel, &n_edges, &edge,
                                     &best, &improved, &finished)
                      : ORC_ERR_NOMEM;
    if (rc == ORC_OK && improved) {
      uint32_t n = paths_of(adj, T, n_edges, (const uint32_t(*)[2])edge, best_sel, vis, order, lens);
      if (n && n == T - best) {
        best_strips = n;
        memcpy(strip_order, order, sizeof(uint32_t) * T);
        memcpy(best_lens, lens, sizeof(uint32_t) * n);
      }
    }
    free(best_sel);
    free(edge);
    if (rc != ORC_OK) {
      free(nb); free(adj); free(vis); free(pos); free(path); free(order); free(lens); free(best_lens);
      return rc;
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

int orc_min_strips(const uint32_t *tris, const uint32_t *ids, uint32_t T, uint32_t greedy_strips,
                   uint32_t max_nodes, uint32_t *out_min, uint32_t *out_lower, uint32_t *out_best) {
  if (!tris || !ids || T == 0 || !out_min || !out_lower || greedy_strips == 0 || greedy_strips > T)
    return ORC_ERR_ARG;
  int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
  int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)T);
  uint32_t (*edge)[2] = (uint32_t(*)[2])malloc(sizeof(uint32_t) * 3 * (size_t)T);
  uint32_t *rem = (uint32_t *)calloc(T, sizeof(uint32_t));
  uint32_t *comp = (uint32_t *)malloc(sizeof(uint32_t) * T);
  uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * T);
  if (!nb || !adj || !edge || !rem || !comp || !stack) {
    free(nb); free(adj); free(edge); free(rem); free(comp); free(stack);
    return ORC_ERR_NOMEM;
  }
  build_adjacency(tris, ids, T, nb, adj);
  edge_list(adj, T, edge, rem);
  /* lower bound: a strip has two ends, and a triangle with at most one
   * neighbour is an end (alone it is a whole strip), so each connected part
   * of the graph needs max(1, ceil(ends / 2)) strips */
  uint32_t lower = 0;
  for (uint32_t i = 0; i < T; i++) comp[i] = 0xFFFFFFFFu;
  for (uint32_t r = 0; r < T; r++) {
    if (comp[r] != 0xFFFFFFFFu) continue;
    uint32_t sp = 0, ends = 0;
    comp[r] = r;
    stack[sp++] = r;
    while (sp) {
      uint32_t x = stack[--sp];
      if (rem[x] <= 1) ends++;
      for (int e = 0; e < 3; e++) {
        int32_t j = adj[3 * x + e];
        if (j >= 0 && comp[j] == 0xFFFFFFFFu) {
          comp[j] = r;
          stack[sp++] = (uint32_t)j;
        }
      }
    }
    lower += ends > 2 ? (ends + 1) / 2 : 1;
  }
  uint32_t n_edges = 0, best = 0;
  int improved = 0, finished = 0;
  int rc = search_cover(adj, T, greedy_strips, max_nodes, NULL, &n_edges, NULL, &best, &improved,
                        &finished);
  if (rc == ORC_OK) {
    *out_lower = lower;
    *out_min = finished ? T - best : 0; /* 0: not searched to the end */
    if (out_best) *out_best = T - best; /* the fewest found, proven or not */
  }
  free(nb); free(adj); free(edge); free(rem); free(comp); free(stack);
  return rc;
}
