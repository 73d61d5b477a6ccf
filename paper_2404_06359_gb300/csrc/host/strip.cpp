// Greedy generalized triangle strip of one meshlet (Sec. 2, 4.2).
//
// Strip rule: a strip enters triangle (a,b,c) through (a,b) and continues
// across the right edge (b,c) into (c,b,x) or across the left edge (c,a) into
// (a,c,x).  The optimal strips of Sec. 4.1 need a MILP solver; this builder
// is deterministic and greedy:
//   * a strip starts at the unvisited triangle with the fewest unvisited
//     neighbours (lowest list position on ties), rotated so that its entry
//     edge borders no unvisited neighbour (first such of the three rotations
//     of the input order, else the input order);
//   * it continues right or left into an unvisited neighbour, choosing the
//     one with fewer unvisited neighbours when both exist (right on ties);
//   * between strips, a restart is four degenerate triangles (Sec. 4.2):
//     entries (c, p, p, q) flagged (L, R, R, L), then r flagged L, which a
//     decoder walks as (a,c,c), (c,c,p), (p,c,p), (p,p,q), (p,q,r).
// Neighbours are found on directed edges: the triangle across edge x->y of a
// triangle is the one holding y->x (lowest list position if several).
#include <algorithm>

#include "host_internal.h"

namespace mc {

void build_strip(const uint32_t *tri, const uint32_t *ids, uint32_t T, StripScratch &s,
                 StripOut &out) {
  auto vert = [&](uint32_t t, uint32_t i) { return tri[3 * (size_t)ids[t] + (i % 3)]; };
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
  s.visited.assign(T, 0);
  auto free_nb = [&](uint32_t t, uint32_t e) {
    int32_t n = s.nb[3 * t + e];
    return n >= 0 && !s.visited[n];
  };
  auto unvisited_nb = [&](uint32_t t) {
    return (uint32_t)free_nb(t, 0) + free_nb(t, 1) + free_nb(t, 2);
  };

  out.stream.clear();
  out.flags.clear();
  out.order.clear();
  out.strips = 0;
  uint32_t count = 0;
  while (count < T) {
    uint32_t start = T, best = 4;
    for (uint32_t t = 0; t < T; t++) {
      if (s.visited[t]) continue;
      uint32_t u = unvisited_nb(t);
      if (u < best) {
        best = u;
        start = t;
        if (u == 0) break;
      }
    }
    uint32_t rot = 0;
    for (uint32_t r = 0; r < 3; r++)
      if (!free_nb(start, r)) {
        rot = r;
        break;
      }
    uint32_t a = vert(start, rot), b = vert(start, rot + 1), c = vert(start, rot + 2);
    if (out.strips == 0) {
      out.stream.insert(out.stream.end(), {a, b, c});
      out.flags.push_back(0);
    } else {
      uint32_t last = out.stream.back();
      out.stream.insert(out.stream.end(), {last, a, a, b, c});
      out.flags.insert(out.flags.end(), {0, 1, 1, 0, 0});
    }
    out.strips++;
    s.visited[start] = 1;
    out.order.push_back(start);
    count++;
    uint32_t cur = start, cr = rot;
    for (;;) {
      uint32_t eR = (cr + 1) % 3, eL = (cr + 2) % 3;
      int32_t tR = free_nb(cur, eR) ? s.nb[3 * cur + eR] : -1;
      int32_t tL = free_nb(cur, eL) ? s.nb[3 * cur + eL] : -1;
      if (tR < 0 && tL < 0) break;
      bool right = (tR >= 0 && tL >= 0) ? unvisited_nb((uint32_t)tR) <= unvisited_nb((uint32_t)tL)
                                        : tR >= 0;
      uint32_t nxt = (uint32_t)(right ? tR : tL);
      uint32_t e0 = right ? c : a, e1 = right ? b : c;
      uint32_t f = 0;
      while (f < 3 && !(vert(nxt, f) == e0 && vert(nxt, f + 1) == e1)) f++;
      uint32_t x = vert(nxt, f + 2);
      a = e0;
      b = e1;
      c = x;
      out.stream.push_back(x);
      out.flags.push_back(right ? 1 : 0);
      s.visited[nxt] = 1;
      out.order.push_back(nxt);
      count++;
      cur = nxt;
      cr = f;
    }
  }
  out.tp = (uint32_t)out.flags.size();
}

}  // namespace mc
