// Meshlet split (Sec. 3) and the re-split of over-long strips (Sec. 4.2).
//
// Greedy growth, deterministic:
//   * seed: the lowest-index unassigned triangle; its class fixes the limits
//     (V~, T~), and only triangles of that class join;
//   * frontier: unassigned triangles sharing an edge with the meshlet, each
//     numbered when it first joins (edges of an added triangle in the order
//     (v0,v1), (v1,v2), (v2,v0), the triangles on an edge by increasing id);
//   * pick: the frontier triangle adding the fewest vertices (0 or 1: a
//     frontier triangle adds at most one); among those, the one with the most
//     edges shared with an assigned triangle of its class (any meshlet, so a
//     triangle about to be enclosed by full meshlets goes first instead of
//     being left behind as a one-triangle meshlet); among those, the
//     lowest-numbered;
//   * stop when the pick would exceed V~ or T~.
// The frontier is a min-heap keyed by (vertices added, 3 - shared edges,
// number); both only fall while a meshlet grows, so a changed triangle is
// pushed again and outdated entries are skipped when they surface.  Classes never share triangles, so each class grows on its
// own thread and the meshlets are merged back in seed order.  A grown meshlet
// whose strip (restart degenerates included) exceeds T~ is split into the
// first ceil(T/2) triangles of its strip order and the rest, recursively.
#include <algorithm>
#include <cstring>
#include <queue>

#include "host_internal.h"

namespace mc {

uint32_t default_threads(uint32_t requested) {
  if (requested) return requested;
  unsigned h = std::thread::hardware_concurrency();
  return h ? h : 1;
}

void parallel_for(uint64_t n, uint32_t threads, const std::function<void(uint64_t)> &fn,
                  uint64_t chunk) {
  threads = default_threads(threads);
  if (n == 0) return;
  if (threads <= 1 || n <= chunk) {
    for (uint64_t i = 0; i < n; i++) fn(i);
    return;
  }
  std::atomic<uint64_t> next{0};
  auto work = [&]() {
    for (;;) {
      uint64_t b = next.fetch_add(chunk);
      if (b >= n) return;
      uint64_t e = std::min(n, b + chunk);
      for (uint64_t i = b; i < e; i++) fn(i);
    }
  };
  uint32_t nt = (uint32_t)std::min<uint64_t>(threads, (n + chunk - 1) / chunk);
  std::vector<std::thread> pool;
  for (uint32_t i = 1; i < nt; i++) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
}

namespace {

struct Grown {
  uint32_t seed;
  uint32_t cls;
  std::vector<uint32_t> tris;
};

struct Adjacency {
  std::vector<uint32_t> off;  // n_verts + 1
  std::vector<uint32_t> lst;  // incident triangles, ascending
};

void build_adjacency(const uint32_t *tri, uint32_t nt, uint32_t nv, uint32_t threads,
                     Adjacency &adj) {
  adj.off.assign((size_t)nv + 1, 0);
  for (size_t i = 0; i < (size_t)nt * 3; i++) adj.off[tri[i] + 1]++;
  for (uint32_t v = 0; v < nv; v++) adj.off[v + 1] += adj.off[v];
  adj.lst.resize((size_t)nt * 3);
  std::vector<uint32_t> cur(adj.off.begin(), adj.off.end() - 1);
  for (uint32_t t = 0; t < nt; t++)
    for (int i = 0; i < 3; i++) adj.lst[cur[tri[3 * (size_t)t + i]]++] = t;
  (void)threads;
}

struct Grower {
  const uint32_t *tri;
  const uint8_t *cls;
  const Adjacency *adj;
  // per-triangle state, shared between classes (each triangle is touched by
  // the thread of its own class only)
  uint8_t *assigned;
  uint32_t *fstamp;   // frontier membership (meshlet stamp)
  uint8_t *shared;    // edges shared with assigned same-class triangles (frontier only)
  uint32_t *seqof;    // frontier number
  // per-thread
  std::vector<uint32_t> vstamp;
  uint32_t stamp = 0;
  uint32_t cur_cls = 0;

  bool same_class(uint32_t t) const { return (cls ? cls[t] : 0) == cur_cls; }

  bool has(uint32_t t, uint32_t v) const {
    const uint32_t *p = tri + 3 * (size_t)t;
    return p[0] == v || p[1] == v || p[2] == v;
  }
  uint32_t cost(uint32_t t) const {
    const uint32_t *p = tri + 3 * (size_t)t;
    return (vstamp[p[0]] != stamp) + (vstamp[p[1]] != stamp) + (vstamp[p[2]] != stamp);
  }

  // edges of t that an assigned triangle of the current class shares
  uint32_t shared_edges(uint32_t t) const {
    const uint32_t *p = tri + 3 * (size_t)t;
    uint32_t n = 0;
    for (int e = 0; e < 3; e++) {
      const uint32_t u = p[e], w = p[(e + 1) % 3];
      for (uint32_t k = adj->off[u]; k < adj->off[u + 1]; k++) {
        const uint32_t t3 = adj->lst[k];
        if (t3 != t && same_class(t3) && assigned[t3] && has(t3, w)) {
          n++;
          break;
        }
      }
    }
    return n;
  }

  void grow_class(uint32_t c, uint32_t n_tris, uint32_t max_v, uint32_t max_t,
                  uint32_t stamp_base, std::vector<Grown> &out) {
    using Item = std::pair<uint64_t, uint32_t>;  // (key, triangle)
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    auto key = [&](uint32_t t2) {
      return ((uint64_t)cost(t2) << 40) | ((uint64_t)(3 - shared[t2]) << 32) | seqof[t2];
    };
    stamp = stamp_base;
    cur_cls = c;
    uint32_t scan = 0;
    for (;;) {
      while (scan < n_tris && (!same_class(scan) || assigned[scan])) scan++;
      if (scan == n_tris) break;
      stamp++;
      Grown g;
      g.seed = scan;
      g.cls = c;
      while (!heap.empty()) heap.pop();
      uint32_t seq = 0, nV = 0;
      uint32_t t = scan;
      for (;;) {
        assigned[t] = 1;
        g.tris.push_back(t);
        const uint32_t *p = tri + 3 * (size_t)t;
        for (int i = 0; i < 3; i++) {
          uint32_t v = p[i];
          if (vstamp[v] == stamp) continue;
          vstamp[v] = stamp;
          nV++;
          // frontier triangles on v now add one vertex fewer
          for (uint32_t k = adj->off[v]; k < adj->off[v + 1]; k++) {
            uint32_t t2 = adj->lst[k];
            if (same_class(t2) && fstamp[t2] == stamp && !assigned[t2]) heap.push({key(t2), t2});
          }
        }
        for (int e = 0; e < 3; e++) {
          uint32_t u = p[e], w = p[(e + 1) % 3];
          for (uint32_t k = adj->off[u]; k < adj->off[u + 1]; k++) {
            uint32_t t2 = adj->lst[k];
            if (t2 == t || !same_class(t2) || assigned[t2] || !has(t2, w)) continue;
            if (fstamp[t2] != stamp) {  // joins the frontier
              fstamp[t2] = stamp;
              seqof[t2] = seq++;
              shared[t2] = (uint8_t)shared_edges(t2);
              heap.push({key(t2), t2});
            } else {  // t now shares this edge
              const uint8_t n = (uint8_t)shared_edges(t2);
              if (n != shared[t2]) {
                shared[t2] = n;
                heap.push({key(t2), t2});
              }
            }
          }
        }
        // pick: the smallest current key (entries whose key has since fallen are stale)
        while (!heap.empty()) {
          const uint32_t t2 = heap.top().second;
          if (!assigned[t2] && heap.top().first == key(t2)) break;
          heap.pop();
        }
        if (heap.empty()) break;
        const uint32_t pick = heap.top().second;
        if (g.tris.size() + 1 > max_t || nV + cost(pick) > max_v) break;
        heap.pop();
        t = pick;
      }
      out.push_back(std::move(g));
    }
  }
};

// Strip + split of one grown meshlet into final meshlets (appended in order).
struct Final {
  std::vector<uint32_t> tris;
  StripOut strip;
};

void split_final(const uint32_t *tri, const uint32_t *ids, uint32_t T, uint32_t max_t,
                 StripScratch &s, std::vector<Final> &out) {
  Final f;
  build_strip(tri, ids, T, s, f.strip);
  if (f.strip.tp <= max_t) {
    f.tris.assign(ids, ids + T);
    out.push_back(std::move(f));
    return;
  }
  std::vector<uint32_t> sub(T);
  for (uint32_t i = 0; i < T; i++) sub[i] = ids[f.strip.order[i]];
  uint32_t h = (T + 1) / 2;
  split_final(tri, sub.data(), h, max_t, s, out);
  split_final(tri, sub.data() + h, T - h, max_t, s, out);
}

}  // namespace
}  // namespace mc

using namespace mc;

extern "C" mc_status mc_meshletize(const uint32_t *tri_idx, uint32_t n_tris, uint32_t n_verts,
                                   const uint8_t *tri_class, const mc_limits *limits,
                                   uint32_t n_classes, uint32_t n_threads, mc_meshlets **out) {
  if (!out) return MC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!tri_idx || !limits || n_classes == 0 || n_classes > 256 || n_verts == 0)
    return MC_ERR_INVALID_ARG;
  for (uint32_t c = 0; c < n_classes; c++)
    if (limits[c].max_verts < 3 || limits[c].max_verts > 256 || limits[c].max_tris < 1 ||
        limits[c].max_tris > 256)
      return MC_ERR_INVALID_ARG;
  uint32_t threads = default_threads(n_threads);
  std::atomic<int> bad{0};
  parallel_for(
      n_tris, threads,
      [&](uint64_t t) {
        const uint32_t *p = tri_idx + 3 * t;
        if (p[0] >= n_verts || p[1] >= n_verts || p[2] >= n_verts || p[0] == p[1] ||
            p[1] == p[2] || p[0] == p[2] || (tri_class && tri_class[t] >= n_classes))
          bad.store(1, std::memory_order_relaxed);
      },
      1 << 16);
  if (bad.load()) return MC_ERR_INVALID_ARG;

  mc_meshlets *m = new (std::nothrow) mc_meshlets();
  if (!m) return MC_ERR_OOM;
  try {
    m->n_tris = n_tris;
    m->n_verts = n_verts;
    Adjacency adj;
    build_adjacency(tri_idx, n_tris, n_verts, threads, adj);
    std::vector<uint8_t> assigned(n_tris, 0);
    std::vector<uint32_t> fstamp(n_tris, 0), seqof(n_tris, 0);
    std::vector<uint8_t> shared(n_tris, 0);
    // which classes occur
    std::vector<uint8_t> present(n_classes, 0);
    if (tri_class) {
      for (uint32_t t = 0; t < n_tris; t++) present[tri_class[t]] = 1;
    } else {
      present[0] = 1;
    }
    std::vector<uint32_t> cls_list;
    for (uint32_t c = 0; c < n_classes; c++)
      if (present[c]) cls_list.push_back(c);
    std::vector<std::vector<Grown>> grown(cls_list.size());
    parallel_for(cls_list.size(), threads, [&](uint64_t i) {
      Grower g;
      g.tri = tri_idx;
      g.cls = tri_class;
      g.adj = &adj;
      g.assigned = assigned.data();
      g.fstamp = fstamp.data();
      g.shared = shared.data();
      g.seqof = seqof.data();
      g.vstamp.assign(n_verts, 0);
      uint32_t c = cls_list[i];
      // stamps of different classes never meet on one triangle; vertex stamps
      // are per thread
      g.grow_class(c, n_tris, limits[c].max_verts, limits[c].max_tris, 0, grown[i]);
    });
    // merge in seed order
    std::vector<const Grown *> all;
    for (auto &v : grown)
      for (auto &g : v) all.push_back(&g);
    std::sort(all.begin(), all.end(), [](const Grown *a, const Grown *b) { return a->seed < b->seed; });
    m->n_grown = (uint32_t)all.size();
    std::vector<std::vector<Final>> finals(all.size());
    parallel_for(
        all.size(), threads,
        [&](uint64_t i) {
          thread_local StripScratch s;
          const Grown *g = all[i];
          split_final(tri_idx, g->tris.data(), (uint32_t)g->tris.size(), limits[g->cls].max_tris, s,
                      finals[i]);
        },
        64);
    size_t nm = 0, ns = 0;
    for (auto &v : finals)
      for (auto &f : v) {
        nm++;
        ns += f.strip.stream.size();
      }
    m->tri.reserve(n_tris);
    m->start.reserve(nm + 1);
    m->stream.reserve(ns);
    m->flags.reserve(ns);
    m->stream_start.reserve(nm + 1);
    m->tp.reserve(nm);
    m->strips.reserve(nm);
    for (auto &v : finals)
      for (auto &f : v) {
        m->start.push_back((uint32_t)m->tri.size());
        m->tri.insert(m->tri.end(), f.tris.begin(), f.tris.end());
        m->stream_start.push_back(m->stream.size());
        m->stream.insert(m->stream.end(), f.strip.stream.begin(), f.strip.stream.end());
        m->flags.insert(m->flags.end(), f.strip.flags.begin(), f.strip.flags.end());
        m->flags.push_back(0);  // keep flags aligned with stream (T' + 2 slots)
        m->flags.push_back(0);
        m->tp.push_back((uint16_t)f.strip.tp);
        m->strips.push_back((uint16_t)f.strip.strips);
      }
    m->start.push_back((uint32_t)m->tri.size());
    m->stream_start.push_back(m->stream.size());
    m->corners.resize(3 * (size_t)m->tri.size());
    for (size_t i = 0; i < m->tri.size(); i++)
      for (int c = 0; c < 3; c++) m->corners[3 * i + c] = tri_idx[3 * (size_t)m->tri[i] + c];
  } catch (const std::bad_alloc &) {
    delete m;
    return MC_ERR_OOM;
  }
  *out = m;
  return MC_OK;
}

extern "C" uint32_t mc_meshlets_count(const mc_meshlets *m) {
  return m ? (uint32_t)(m->start.empty() ? 0 : m->start.size() - 1) : 0;
}

extern "C" mc_status mc_meshlets_get(const mc_meshlets *m, uint32_t *out_tri, uint32_t *out_start) {
  if (!m) return MC_ERR_INVALID_ARG;
  if (out_tri) std::memcpy(out_tri, m->tri.data(), m->tri.size() * sizeof(uint32_t));
  if (out_start) std::memcpy(out_start, m->start.data(), m->start.size() * sizeof(uint32_t));
  return MC_OK;
}

extern "C" void mc_meshlets_free(mc_meshlets *m) { delete m; }
