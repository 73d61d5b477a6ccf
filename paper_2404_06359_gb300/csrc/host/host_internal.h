// Internal declarations of the host-side encoder (meshletize / stripify /
// encode).  Not part of the C ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <functional>
#include <thread>
#include <vector>

#include "meshlet_codec.h"

namespace mc {

// Runs fn(i) for i in [0, n) on up to `threads` workers, dynamic chunks.
void parallel_for(uint64_t n, uint32_t threads, const std::function<void(uint64_t)> &fn,
                  uint64_t chunk = 1);
uint32_t default_threads(uint32_t requested);

// One meshlet's generalized triangle strip (Sec. 2, 4.2).
struct StripOut {
  uint32_t tp = 0;      // T' (triangles incl. restart degenerates)
  uint32_t strips = 0;  // number of strips (restarts + 1)
  std::vector<uint32_t> stream;  // T'+2 global vertex ids
  std::vector<uint8_t> flags;    // T' flags, 1 = right
  std::vector<uint32_t> order;   // list positions in strip order
};

// Per-thread scratch of the strip builder.
struct StripScratch {
  std::vector<uint64_t> keys;
  std::vector<int32_t> nb, adj, pos;
  std::vector<uint8_t> visited;
  std::vector<uint32_t> path, order, lens, best_order, best_lens;
  // fewest-strips search
  std::vector<uint32_t> eu, ev, rem, end_of;
  std::vector<uint8_t> deg, sel, best_sel;
  std::vector<int32_t> chosen_nb;
};

// Strip over the triangles tri[ids[i]], i = list position (or, with
// list_corners, the triangle whose corners are list_corners[3i..3i+2]; ids
// then only seed the random choices): the best of the randomised greedy
// covers and, with search_nodes > 0, the fewest-strips cover a branch and
// bound finds within that many nodes when it has fewer strips.
void build_strip(const uint32_t *tri, const uint32_t *ids, uint32_t T, StripScratch &s,
                 StripOut &out, uint32_t search_nodes = 0, const uint32_t *list_corners = nullptr);

}  // namespace mc

// Final meshlets of one mesh: triangle grouping plus the strip of each.
struct mc_meshlets {
  uint32_t n_tris = 0, n_verts = 0;
  uint32_t n_grown = 0;
  std::vector<uint32_t> tri;          // triangle ids grouped by meshlet
  std::vector<uint32_t> corners;      // their 3 vertex ids each (input winding), same order
  std::vector<uint32_t> start;        // meshlet offsets into tri (count + 1)
  std::vector<uint64_t> stream_start; // meshlet offsets into stream (count + 1)
  std::vector<uint32_t> stream;       // strip entries (global vertex ids)
  std::vector<uint8_t> flags;         // one per strip triangle, same offsets - 2*m
  std::vector<uint16_t> tp;           // T' per meshlet
  std::vector<uint16_t> strips;       // strips per meshlet
};

struct mc_blob {
  std::vector<mc_desc> desc;
  std::vector<uint8_t> payload;
  std::vector<mc_grid> grids;
  std::vector<mc_mesh_info> meshes;
  std::vector<uint32_t> vmap;
  std::vector<mc_cone> cones;
  uint32_t n_attr = 0, attr_bits = 0;
  std::vector<mc_attr_desc> attr_desc;
  std::vector<mc_attr_grid> attr_grids;
  uint64_t total_tris = 0, total_verts = 0, input_tris = 0;
  uint64_t restarts = 0, split_meshlets = 0, conn_bits = 0, pos_bits_total = 0;
  uint32_t max_block_words = 0, max_tris = 0, max_verts = 0;
};
