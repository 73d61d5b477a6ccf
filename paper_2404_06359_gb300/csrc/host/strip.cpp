// Generalized triangle strips of one meshlet (Sec. 2, 4.2).
//
// Strip rule: a strip enters triangle (a,b,c) through (a,b) and continues
// across the right edge (b,c) into (c,b,x) or across the left edge (c,a) into
// (a,c,x), so any simple path of edge-adjacent triangles is one strip and a
// meshlet's strips are a path cover of its triangles.  The minimum cover of
// Sec. 4.1 needs a MILP solver; this builder keeps the best (fewest strips,
// first on ties) of kTries randomised greedy covers:
//   * a strip starts at an unvisited triangle with the fewest unvisited
//     neighbours, picked at random among the ties (list order);
//   * it grows at its end into an unvisited neighbour with the fewest
//     unvisited neighbours (random among the ties, edge order); when stuck
//     and its end borders the strip member at position k < length - 2, the
//     part after k is reversed (a Posa rotation, random among such members,
//     at most kRotations per strip) and growth resumes at the new end;
//   * it then grows the same way from its other end.
// Random numbers: SplitMix64 (the state advances by 0x9E3779B97F4A7C15 and
// is mixed by two xor-shift-multiply rounds), seeded per meshlet with
// first-triangle-id * 0x9E3779B97F4A7C15 + T; a choice among n candidates
// takes the next number modulo n.
// A strip's first triangle enters through the first of its edges (input
// order) that does not lead to the second; between strips a restart is four
// degenerate triangles (Sec. 4.2): entries (c, p, p, q) flagged (L, R, R, L),
// then r flagged L, which a decoder walks as (a,c,c), (c,c,p), (p,c,p),
// (p,p,q), (p,q,r).
// Neighbours are found on directed edges: the triangle across edge x->y of a
// triangle is the one holding y->x (lowest list position if several), and
// only mutual pairs count as adjacent.
#include <algorithm>

#include "host_internal.h"

namespace mc {

namespace {
constexpr uint32_t kTries = 16;      // randomised covers per meshlet
constexpr uint32_t kRotations = 32;  // rotations per strip
}  // namespace

namespace {
// Fewest strips by branch and bound (Sec. 4.1's objective: the most
// adjacency edges used with no triangle on three of them and no cycle).
// Edges (u, v), u < v, are taken in the order of u and its edge slots; at
// each edge the branch that takes it (when both ends have room and they do
// not end one path) is searched before the one that leaves it; a branch is
// cut when the edges taken plus the most still reachable -- half the sum over
// triangles of min(room, undecided edges) -- cannot beat the best so far.
// Every call counts one node; past node_limit the search stops.
struct CoverSearch {
  StripScratch &s;
  uint32_t T, n_edges, nodes = 0, node_limit, chosen = 0, best;
  bool stopped = false, improved = false;

  uint32_t reachable() const {
    uint32_t sum = 0;
    for (uint32_t x = 0; x < T; x++) sum += std::min<uint32_t>(s.rem[x], 2u - s.deg[x]);
    return sum / 2;
  }

  void run(uint32_t i) {
    if (stopped) return;
    if (++nodes > node_limit) {
      stopped = true;
      return;
    }
    if (chosen > best) {
      best = chosen;
      improved = true;
      std::copy(s.sel.begin(), s.sel.begin() + n_edges, s.best_sel.begin());
    }
    if (i == n_edges || chosen + reachable() <= best) return;
    const uint32_t u = s.eu[i], v = s.ev[i];
    s.rem[u]--;
    s.rem[v]--;
    if (s.deg[u] < 2 && s.deg[v] < 2 && s.end_of[u] != v) {
      const uint32_t a = s.end_of[u], b = s.end_of[v];  // joined path: a .. u - v .. b
      s.deg[u]++;
      s.deg[v]++;
      s.end_of[a] = b;
      s.end_of[b] = a;
      chosen++;
      s.sel[i] = 1;
      run(i + 1);
      s.sel[i] = 0;
      chosen--;
      s.end_of[a] = u;
      s.end_of[b] = v;
      s.end_of[u] = a;
      s.end_of[v] = b;
      s.deg[u]--;
      s.deg[v]--;
    }
    run(i + 1);
    s.rem[u]++;
    s.rem[v]++;
  }
};

// Strips of the chosen edges in s.best_sel: from every path end (at most one
// chosen edge) in list order not yet emitted, the path walked to its other
// end, into s.order / s.lens.  Returns the number of strips (0 if some
// triangle was not reached).
uint32_t chosen_paths(StripScratch &s, uint32_t T, uint32_t n_edges) {
  s.chosen_nb.assign(2 * (size_t)T, -1);
  for (uint32_t i = 0; i < n_edges; i++) {
    if (!s.best_sel[i]) continue;
    const uint32_t u = s.eu[i], v = s.ev[i];
    s.chosen_nb[2 * u + (s.chosen_nb[2 * u] >= 0 ? 1 : 0)] = (int32_t)v;
    s.chosen_nb[2 * v + (s.chosen_nb[2 * v] >= 0 ? 1 : 0)] = (int32_t)u;
  }
  std::fill(s.visited.begin(), s.visited.begin() + T, 0);
  uint32_t n_order = 0, n_strips = 0;
  for (uint32_t t = 0; t < T; t++) {
    if (s.visited[t] || (s.chosen_nb[2 * t] >= 0 && s.chosen_nb[2 * t + 1] >= 0)) continue;
    uint32_t len = 0;
    int32_t prev = -1, cur = (int32_t)t;
    while (cur >= 0) {
      s.visited[cur] = 1;
      s.order[n_order++] = (uint32_t)cur;
      len++;
      int32_t nxt = s.chosen_nb[2 * cur] != prev ? s.chosen_nb[2 * cur] : s.chosen_nb[2 * cur + 1];
      if (nxt >= 0 && s.visited[nxt]) nxt = -1;
      prev = cur;
      cur = nxt;
    }
    s.lens[n_strips++] = len;
  }
  return n_order == T ? n_strips : 0;
}
}  // namespace

void build_strip(const uint32_t *tri, const uint32_t *ids, uint32_t T, StripScratch &s,
                 StripOut &out, uint32_t search_nodes, const uint32_t *list_corners) {
  auto vert = [&](uint32_t t, uint32_t i) {
    return list_corners ? list_corners[3 * (size_t)t + (i % 3)] : tri[3 * (size_t)ids[t] + (i % 3)];
  };
  // directed edges t*3+e, sorted by (x, y, position) of edge x -> y
  s.keys.resize(3 * (size_t)T);
  for (uint32_t i = 0; i < 3 * T; i++) s.keys[i] = i;
  std::sort(s.keys.begin(), s.keys.end(), [&](uint64_t p, uint64_t q) {
    uint32_t tp = (uint32_t)(p / 3), ep = (uint32_t)(p % 3);
    uint32_t tq = (uint32_t)(q / 3), eq = (uint32_t)(q % 3);
    uint32_t xp = vert(tp, ep), yp = vert(tp, ep + 1), xq = vert(tq, eq), yq = vert(tq, eq + 1);
    if (xp != xq) return xp < xq;
    if (yp != yq) return yp < yq;
    return tp < tq;
  });
  s.nb.assign(3 * (size_t)T, -1);
  for (uint32_t t = 0; t < T; t++)
    for (uint32_t e = 0; e < 3; e++) {
      uint32_t x = vert(t, e), y = vert(t, e + 1);
      // first entry with directed edge (y -> x)
      auto it = std::lower_bound(s.keys.begin(), s.keys.end(), 0ull, [&](uint64_t p, uint64_t) {
        uint32_t tp = (uint32_t)(p / 3), ep = (uint32_t)(p % 3);
        uint32_t xp = vert(tp, ep), yp = vert(tp, ep + 1);
        if (xp != y) return xp < y;
        return yp < x;
      });
      if (it != s.keys.end()) {
        uint32_t tp = (uint32_t)(*it / 3), ep = (uint32_t)(*it % 3);
        if (vert(tp, ep) == y && vert(tp, ep + 1) == x) s.nb[3 * t + e] = (int32_t)tp;
      }
    }
  // mutual neighbour pairs only
  s.adj.assign(3 * (size_t)T, -1);
  for (uint32_t t = 0; t < T; t++)
    for (uint32_t e = 0; e < 3; e++) {
      const int32_t j = s.nb[3 * t + e];
      if (j < 0) continue;
      for (uint32_t f = 0; f < 3; f++)
        if (s.nb[3 * (uint32_t)j + f] == (int32_t)t) s.adj[3 * t + e] = j;
    }

  // best of kTries randomised greedy path covers (fewest strips, first on ties)
  s.visited.resize(T);
  s.pos.resize(T);
  s.path.resize(T);
  s.order.resize(T);
  s.lens.resize(T);
  s.best_order.resize(T);
  s.best_lens.resize(T);
  uint64_t rng = (uint64_t)ids[0] * 0x9E3779B97F4A7C15ull + T;
  auto next = [&]() {
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto free_deg = [&](uint32_t t) {
    uint32_t n = 0;
    for (uint32_t e = 0; e < 3; e++) {
      const int32_t j = s.adj[3 * t + e];
      n += (j >= 0 && !s.visited[j]) ? 1u : 0u;
    }
    return n;
  };
  uint32_t len = 0;
  auto reverse_from = [&](uint32_t from) {
    std::reverse(s.path.begin() + from, s.path.begin() + len);
    for (uint32_t i = from; i < len; i++) s.pos[s.path[i]] = (int32_t)i;
  };
  uint32_t best_strips = 0;
  for (uint32_t attempt = 0; attempt < kTries; attempt++) {
    std::fill(s.visited.begin(), s.visited.end(), 0);
    std::fill(s.pos.begin(), s.pos.end(), -1);
    uint32_t covered = 0, n_strips = 0, n_order = 0;
    while (covered < T) {
      uint32_t best = 4, ties = 0;
      for (uint32_t t = 0; t < T; t++) {
        if (s.visited[t]) continue;
        const uint32_t d = free_deg(t);
        if (d < best) {
          best = d;
          ties = 1;
        } else if (d == best) {
          ties++;
        }
      }
      uint32_t pick = (uint32_t)(next() % ties), start = 0;
      for (uint32_t t = 0; t < T; t++) {
        if (s.visited[t] || free_deg(t) != best) continue;
        if (pick-- == 0) {
          start = t;
          break;
        }
      }
      len = 0;
      s.path[len++] = start;
      s.pos[start] = 0;
      s.visited[start] = 1;
      covered++;
      uint32_t rotations = 0;
      for (int side = 0; side < 2; side++) {
        for (;;) {
          const uint32_t cur = s.path[len - 1];
          uint32_t cand[3], dmin = 4, n = 0;
          for (uint32_t e = 0; e < 3; e++) {
            const int32_t j = s.adj[3 * cur + e];
            if (j < 0 || s.visited[j]) continue;
            const uint32_t d = free_deg((uint32_t)j);
            if (d < dmin) {
              dmin = d;
              n = 0;
            }
            if (d == dmin) cand[n++] = (uint32_t)j;
          }
          if (n) {
            const uint32_t j = cand[next() % n];
            s.pos[j] = (int32_t)len;
            s.path[len++] = j;
            s.visited[j] = 1;
            covered++;
            continue;
          }
          if (rotations == kRotations) break;
          uint32_t opt[3], m = 0;
          for (uint32_t e = 0; e < 3; e++) {
            const int32_t y = s.adj[3 * cur + e];
            if (y >= 0 && s.pos[y] >= 0 && (uint32_t)s.pos[y] + 2 < len) opt[m++] = (uint32_t)s.pos[y];
          }
          if (!m) break;
          reverse_from(opt[next() % m] + 1);
          rotations++;
        }
        reverse_from(0);
      }
      for (uint32_t i = 0; i < len; i++) {
        s.order[n_order++] = s.path[i];
        s.pos[s.path[i]] = -1;
      }
      s.lens[n_strips++] = len;
    }
    if (attempt == 0 || n_strips < best_strips) {
      best_strips = n_strips;
      std::copy(s.order.begin(), s.order.begin() + T, s.best_order.begin());
      std::copy(s.lens.begin(), s.lens.begin() + n_strips, s.best_lens.begin());
    }
  }

  // optionally, fewer strips by the search, started from the greedy count
  if (search_nodes && best_strips > 1) {
    s.eu.clear();
    s.ev.clear();
    s.rem.assign(T, 0);
    for (uint32_t t = 0; t < T; t++)
      for (uint32_t e = 0; e < 3; e++) {
        const int32_t j = s.adj[3 * t + e];
        if (j > (int32_t)t) {
          s.eu.push_back(t);
          s.ev.push_back((uint32_t)j);
          s.rem[t]++;
          s.rem[j]++;
        }
      }
    const uint32_t n_edges = (uint32_t)s.eu.size();
    s.deg.assign(T, 0);
    s.end_of.resize(T);
    for (uint32_t t = 0; t < T; t++) s.end_of[t] = t;
    s.sel.assign(n_edges, 0);
    s.best_sel.assign(n_edges, 0);
    CoverSearch cs{s, T, n_edges};
    cs.node_limit = search_nodes;
    cs.best = T - best_strips;
    cs.run(0);
    if (cs.improved) {
      const uint32_t n = chosen_paths(s, T, n_edges);
      if (n && n == T - cs.best) {
        best_strips = n;
        std::copy(s.order.begin(), s.order.begin() + T, s.best_order.begin());
        std::copy(s.lens.begin(), s.lens.begin() + n, s.best_lens.begin());
      }
    }
  }

  // emission: each path is one strip; restarts between strips
  out.stream.clear();
  out.flags.clear();
  out.order.assign(s.best_order.begin(), s.best_order.begin() + T);
  out.strips = best_strips;
  uint32_t at = 0;
  for (uint32_t k = 0; k < best_strips; k++) {
    const uint32_t *p = s.best_order.data() + at;
    const uint32_t plen = s.best_lens[k];
    at += plen;
    // entry edge of the first triangle: the first of its edges not leading to p[1]
    uint32_t rot = 0;
    if (plen > 1)
      while (rot < 3 && s.adj[3 * p[0] + rot] == (int32_t)p[1]) rot++;
    uint32_t a = vert(p[0], rot), b = vert(p[0], rot + 1), c = vert(p[0], rot + 2);
    if (k == 0) {
      out.stream.insert(out.stream.end(), {a, b, c});
      out.flags.push_back(0);
    } else {
      const uint32_t last = out.stream.back();
      out.stream.insert(out.stream.end(), {last, a, a, b, c});
      out.flags.insert(out.flags.end(), {0, 1, 1, 0, 0});
    }
    uint32_t cr = rot;
    for (uint32_t i = 0; i + 1 < plen; i++) {
      const uint32_t cur = p[i], nxt = p[i + 1];
      const uint32_t eR = (cr + 1) % 3, eL = (cr + 2) % 3;
      bool right;
      if (s.adj[3 * cur + eR] == (int32_t)nxt) right = true;
      else if (s.adj[3 * cur + eL] == (int32_t)nxt) right = false;
      else break;  // not reachable for a path of mutual neighbours
      const uint32_t e0 = right ? c : a, e1 = right ? b : c;
      uint32_t f = 0;
      while (f < 3 && !(vert(nxt, f) == e0 && vert(nxt, f + 1) == e1)) f++;
      if (f == 3) break;
      const uint32_t x = vert(nxt, f + 2);
      a = e0;
      b = e1;
      c = x;
      out.stream.push_back(x);
      out.flags.push_back(right ? 1 : 0);
      cr = f;
    }
  }
  out.tp = (uint32_t)out.flags.size();
}

}  // namespace mc
