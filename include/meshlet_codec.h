/*
 * meshlet_codec.h -- C ABI of the GB300 GTS-Reuse meshlet codec.
 *
 * Implements the data-parallel decode of Kuth et al., "Towards Practical
 * Meshlet Compression" (VMV 2024) on NVIDIA GB300 (sm_103a), plus the host
 * preprocessing that produces its input.
 *
 *   host    mc_meshletize  split a triangle mesh into meshlets (Sec. 3)
 *           mc_encode      generalized triangle strips with one L/R flag per
 *                          triangle (Sec. 2, 4.2), index reuse packing
 *                          (Sec. 4.3), crack-free fixed-point positions
 *                          (Sec. 4.4)
 *   device  mc_decode_*    parallel decode of many meshlets to u8 local and
 *                          u32 global triangle indices and FP32 positions
 *                          (Sec. 3, 4.2-4.4), optionally fused with culling.
 *
 * Conventions shared by every call:
 *   - Host objects (mc_meshlets, mc_blob) are created and freed by the
 *     library.  Device buffers are allocated by the caller and are never
 *     freed or reallocated by the library.
 *   - Device calls are asynchronous on the caller's CUDA stream (`stream` is
 *     a cudaStream_t; NULL = legacy default stream) and never synchronise.
 *   - Argument errors are returned synchronously (MC_ERR_INVALID_ARG,
 *     MC_ERR_LIMIT); launch failures as MC_ERR_CUDA.  Errors found by a
 *     kernel (corrupt stream, exceeded capacity) are OR-ed as bit masks
 *     (1u << mc_status) into the caller's device status word *d_status,
 *     which the caller reads after synchronising.  The kernels never trap.
 *   - No call falls back to a CPU implementation.
 *
 * Blob format (little-endian; the device reads it as is):
 *   descriptor, 32 bytes per meshlet (mc_desc below);
 *   payload block per meshlet, u32 words, bits LSB-first, 16-byte aligned:
 *     ceil(T'/32) L/R words     bit k = 1: triangle k is entered across the
 *                               right edge (b,c) of triangle k-1, 0: left edge
 *                               (c,a) (Sec. 2); bit 0 is 0
 *     ceil(T'/32) increment words  bit k = 1: the strip entry of triangle k is
 *                               a vertex not seen before (Sec. 4.3); bit 0 is 0
 *     ceil(R*w/32) reuse words  R = T' - V + 2 entries of w bits (Sec. 4.3)
 *     ceil(3*V*b/32) position words  vertex v channel c at bit (3v+c)*b
 *   plain GTS block (descriptor w = 0, Sec. 4.2 before the reuse packing):
 *     the L/R words, then ceil((T'-1)/4) words holding one byte per triangle
 *     k >= 1, its strip entry I[k+2] (byte k-1), then the position words
 *   grid entry, 32 bytes (mc_grid below): FP32 origin G and step Delta of
 *     the global quantisation grid of one mesh at one bit width (Sec. 4.4).
 *   normal cone, 32 bytes per meshlet (mc_cone below), optional input of the
 *     fused cull.
 */
#ifndef MESHLET_CODEC_H
#define MESHLET_CODEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MC_OK = 0,
  MC_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
  MC_ERR_LIMIT = 2,       /* a meshlet or grid coordinate exceeds the format */
  MC_ERR_CORRUPT = 3,     /* the bitstream contradicts itself */
  MC_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  MC_ERR_OOM = 5,         /* host allocation failed */
  MC_ERR_TIMEOUT = 6      /* a bounded device wait gave up */
} mc_status;

/* Human-readable name of a status code (static storage). */
const char *mc_status_string(mc_status s);

/* Library version string (static storage). */
const char *mc_version(void);

/* ------------------------------------------------------------------ format */

/* Per-meshlet descriptor, 32 bytes (Sec. 3: a meshlet stores the offset of
 * its vertex block and of its index data).  tri_base / vertex_base place the
 * meshlet's decoded triangles and vertices in the batch-wide outputs. */
typedef struct {
  uint32_t payload_off16; /* payload block offset, in 16-byte units */
  uint32_t vertex_base;   /* first decoded vertex; global index = base + local */
  uint32_t tri_base;      /* first decoded triangle (T' slots incl. degenerates) */
  uint16_t n_verts;       /* V, 3..256 */
  uint16_t n_tris;        /* T' = triangles incl. restart degenerates, 1..256 */
  uint8_t reuse_bits;     /* w, 1..8, 2^w >= V; 0 = plain GTS block */
  uint8_t pos_bits;       /* b, 1..32 */
  uint16_t grid;          /* index of the mc_grid entry */
  uint32_t L[3];          /* meshlet minimum on the global grid (Sec. 4.4);
                           * L[c] + 2^b - 1 < 2^32 (the whole quantisation box
                           * is representable), else the meshlet is corrupt */
} mc_desc;

/* Global quantisation grid (Sec. 4.4): x = G + g * Delta for grid coordinate
 * g = L + q, evaluated in FP32 as fmaf((float)g, Delta, G) when g < 2^24 and
 * as fmaf((float)(g & 0xFFF), Delta, fmaf((float)(g >> 12), 4096 Delta, G))
 * otherwise.  One entry per mesh and position bit width. */
typedef struct {
  float G[3];
  uint32_t pos_bits;
  float delta[3];
  uint32_t mesh_id;
} mc_grid;

/* Attribute channels beyond the position (Sec. 4.4: the attribute vector of
 * a vertex; every channel is quantised uniformly at attr_bits bits on its
 * own crack-free global grid, by the rules of the positions).  A blob with
 * n_attr channels stores, after the position words of each payload block,
 * ceil(n_attr * V * attr_bits / 32) attribute words (vertex v channel c at
 * bit (n_attr v + c) attr_bits), plus one record per meshlet and one grid
 * per mesh:
 *   mc_attr_desc (32 B): La[c] = the meshlet's minimum on the attribute grid
 *                        of channel c; grid = index of its mc_attr_grid;
 *   mc_attr_grid (48 B): origin G[c] and step delta[c] per channel, decoded
 *                        like the positions: a = fma((float)g, delta, G) for
 *                        g = La + q < 2^24, else the split form of mc_grid. */
typedef struct {
  uint32_t La[5];
  uint16_t grid;
  uint16_t reserved0;
  uint32_t reserved1[2];
} mc_attr_desc;

typedef struct {
  float G[5];
  float delta[5];
  uint32_t attr_bits;
  uint32_t mesh_id;
} mc_attr_grid;

/* Normal cone of a meshlet, 32 bytes: the per-meshlet cull data kept beside
 * the offsets (Sec. 3: the triangle normals of a meshlet form a cone, stored
 * as an axis and an opening angle; Sec. 5: 16 B of cull information per
 * meshlet in the paper's layout).  Here: a sphere holding the decoded
 * vertices and a cone holding every triangle normal, computed by mc_encode
 * in FP64 from the decoded FP32 positions:
 *   center  middle of the positions' bounding box (FP32, nearest);
 *   radius  largest distance of a position from center, times 1 + 2^-20,
 *           rounded up to FP32;
 *   axis    normalised sum of the unit normals (p1 - p0) x (p2 - p0) of the
 *           triangles with an area (FP32, nearest);
 *   s       sin of the cone's half angle + 2^-20, rounded up to FP32: with
 *           c = the smallest normal . axis, s = sqrt(1 - c^2) + 2^-20; 1 (no
 *           cone) when c <= 0, when no triangle has an area or when s >= 1.
 * A meshlet is back-facing as a whole for a camera at e when
 *   axis . (center - e) >= s |center - e| + radius
 * (every normal n within the cone and every point p within the sphere then
 * satisfy n . (p - e) >= 0). */
typedef struct {
  float center[3];
  float radius;
  float axis[3];
  float s;
} mc_cone;

/* -------------------------------------------------------------------- host */

typedef struct mc_meshlets mc_meshlets; /* opaque, library-owned */
typedef struct mc_blob mc_blob;         /* opaque, library-owned */

typedef struct {
  uint32_t max_verts; /* V~, 3..256 (Sec. 3) */
  uint32_t max_tris;  /* T~, 1..256; bounds T' including degenerates (Sec. 4.2) */
} mc_limits;

/* Split a triangle mesh into meshlets (Sec. 3) -- deterministic greedy growth
 * from the lowest-index unassigned triangle, preferring frontier triangles
 * that add no vertex, then the earliest to join the frontier -- and split
 * every meshlet whose strip, restart degenerates included, exceeds T~ into
 * the two halves of its strip order (Sec. 4.2).
 *   tri_idx   n_tris x 3 vertex indices (< n_verts), counter-clockwise
 *   tri_class optional n_tris class ids (< n_classes): meshlets never mix
 *             classes and use limits[class]; NULL = all class 0
 *   n_threads worker threads (0 = hardware concurrency)
 * Returns MC_ERR_INVALID_ARG for out-of-range or repeated vertex indices. */
mc_status mc_meshletize(const uint32_t *tri_idx, uint32_t n_tris, uint32_t n_verts,
                        const uint8_t *tri_class, const mc_limits *limits,
                        uint32_t n_classes, uint32_t n_threads, mc_meshlets **out);

/* Number of meshlets, and their triangle grouping: out_tri (n_tris ids, may
 * be NULL) grouped by meshlet, out_start (count + 1 offsets, may be NULL). */
uint32_t mc_meshlets_count(const mc_meshlets *m);
mc_status mc_meshlets_get(const mc_meshlets *m, uint32_t *out_tri, uint32_t *out_start);
void mc_meshlets_free(mc_meshlets *m);

typedef struct {
  uint32_t pos_bits;              /* b for every meshlet (1..32) ... */
  const uint8_t *pos_bits_per_meshlet; /* ... or one b per meshlet (may be NULL) */
  uint32_t reuse_mode;            /* 0: w = 8 (Sec. 3), 1: w = ceil(log2 V),
                                   * 2: plain GTS (Sec. 4.2: every stream entry
                                   * stored at 8 bits; descriptor w = 0) */
  const uint32_t *order;          /* optional: blob slot p holds meshlet order[p] */
  uint32_t mesh_id;               /* written into the grid entries */
  uint32_t n_threads;             /* 0 = hardware concurrency */
  const float *attrs;             /* optional: n_verts x n_attr extra attribute
                                   * channels per input vertex (e.g. normal,
                                   * texture coordinate; Sec. 4.4) */
  uint32_t n_attr;                /* 0..5 */
  uint32_t attr_bits;             /* b of every attribute channel (1..32) */
  uint32_t strip_search_nodes;    /* 0: the greedy strips; else per meshlet a
                                   * branch and bound for the fewest strips
                                   * (Sec. 4.1's objective: the most shared
                                   * edges used, no fork, no cycle) runs from
                                   * the greedy cover for at most this many
                                   * nodes, and its cover is used when it has
                                   * fewer strips (fewer restart degenerates) */
} mc_encode_params;

/* Encode the meshlets of one mesh (Sec. 4.2-4.4) into a blob.
 *   pos_xyz  n_verts x 3 FP32 positions
 * Per meshlet: greedy generalized triangle strip (restart = four degenerate
 * triangles), first-appearance vertex numbering, L/R + increment flags,
 * reuse entries; positions on the global grid with Delta = w/(2^b - 1)
 * rounded up to FP32 (w = largest meshlet extent at that b), grid coordinate
 * floor((x - G)/Delta + 1/2), stored relative to the meshlet minimum L.
 * MC_ERR_LIMIT if a grid coordinate exceeds 32 bits. */
mc_status mc_encode(const mc_meshlets *m, const float *pos_xyz, uint32_t n_verts,
                    const mc_encode_params *p, mc_blob **out);

/* Concatenate blobs into one batch: payload offsets, vertex/triangle bases
 * and grid ids are rebased; grid mesh ids become the blob's list position. */
mc_status mc_blob_concat(const mc_blob *const *blobs, uint32_t n, mc_blob **out);

typedef struct {
  uint32_t first_meshlet, n_meshlets; /* blob slots of this mesh */
  uint64_t tri_base, n_tris;          /* decoded triangle range (T') */
  uint64_t vertex_base, n_verts;      /* decoded vertex range */
  uint64_t input_tris;                /* triangles of the input mesh */
} mc_mesh_info;

/* Read-only view of a blob (pointers stay valid until mc_blob_free). */
typedef struct {
  const mc_desc *desc;       uint32_t n_meshlets;
  const uint8_t *payload;    uint64_t payload_bytes;
  const mc_grid *grids;      uint32_t n_grids;
  const mc_mesh_info *meshes; uint32_t n_meshes;
  const uint32_t *vertex_map; /* input vertex id of each decoded vertex */
  uint64_t total_tris;        /* sum of T' (decoded triangle slots) */
  uint64_t total_verts;       /* sum of V */
  uint64_t input_tris;        /* sum of input triangles */
  uint64_t restarts;          /* strip restarts (each = 4 degenerates) */
  uint64_t split_meshlets;    /* meshlets added by splitting */
  uint64_t conn_bits;         /* sum of 2 T' + w R (flags + reuse) */
  uint64_t pos_bits_total;    /* sum of 3 V b */
  uint32_t max_block_words;   /* largest payload block, u32 words */
  uint32_t max_tris;          /* largest T' */
  const mc_cone *cones;       /* normal cone per meshlet (n_meshlets) */
  uint32_t n_attr, attr_bits; /* extra attribute channels (0 = none) */
  const mc_attr_desc *attr_desc;  /* n_meshlets records (n_attr > 0) */
  const mc_attr_grid *attr_grids; /* n_attr_grids entries */
  uint32_t n_attr_grids;
  uint32_t max_verts;         /* largest V */
} mc_blob_view_t;

mc_status mc_blob_view(const mc_blob *b, mc_blob_view_t *v);
void mc_blob_free(mc_blob *b);

/* ------------------------------------------------------------------ device */

/* A batch resident in device memory (caller-owned): the three blob arrays. */
typedef struct {
  const mc_desc *desc;
  const uint8_t *payload;
  const mc_grid *grids;
  uint32_t n_meshlets;      /* at most 2^31 (the persistent kernels' 32-bit
                             * work counter needs headroom); more is
                             * MC_ERR_LIMIT from every device call */
  uint32_t n_grids;
  uint64_t payload_bytes;
  uint64_t total_tris;  /* capacity of the outputs, triangles (sum of T') */
  uint64_t total_verts; /* capacity of the outputs, vertices (sum of V) */
  uint32_t max_block_words; /* from mc_blob_view (sizes shared-memory staging) */
  uint32_t max_tris;        /* largest T' (from mc_blob_view); 0 = 256 */
  const mc_cone *cones;     /* optional device copy of the normal cones
                             * (n_meshlets, 16-byte aligned); NULL = the
                             * fused cull uses no cone test */
  uint32_t n_attr, attr_bits; /* the blob's attribute channels (0 = none);
                               * they size every payload block */
  const mc_attr_desc *attr_desc;  /* device copies (16-byte aligned), needed by */
  const mc_attr_grid *attr_grids; /* mc_decode_batch_vertices only */
  uint32_t n_attr_grids;
  uint32_t max_verts;       /* largest V (from mc_blob_view, sizes the fused
                             * culls' per-warp vertex buffers); 0 = max_tris
                             * + 2; a meshlet with more vertices is corrupt */
} mc_device_batch;

/* Launch shape; zero fields take the library defaults or the autotuned
 * values.  checked = 1 selects the kernel variant that validates every
 * stream entry (reuse index < vertices seen, flag/count consistency) and
 * reports MC_ERR_CORRUPT instead of decoding garbage. */
typedef struct {
  uint32_t warps_per_cta;     /* 1..32 */
  uint32_t ctas_per_sm;       /* persistent CTAs per SM */
  uint32_t meshlets_per_grab; /* work-queue granularity (persistent kernels,
                               * 1..16); a grab whose shared-memory buffers
                               * do not fit warps_per_cta warps on an SM is
                               * reduced until they do */
  uint32_t checked;
  uint32_t wait_cycles;       /* limit, in SM clock cycles, of each wait of a
                               * warp on another warp's result (the look-back
                               * of mc_decode_cull_ordered); 0 = 2^31 (about a
                               * second).  A wait that runs out sets
                               * MC_ERR_TIMEOUT in the status word.  The waits
                               * of a warp for its own bulk copies keep their
                               * fixed bound of 2^31 cycles. */
  uint32_t lanes_per_meshlet; /* sub-warp width of mc_decode_batch and its
                               * graph / host-buffer forms: 32 = one meshlet
                               * per warp, 16 = two meshlets per warp (one
                               * per half; grabs of at least 2 meshlets);
                               * 0 = the autotuned value, else 32.  Other
                               * calls use 32. */
} mc_tuning;

/* Bytes of device scratch the persistent kernels need (work-queue counters).
 * The scratch must be zero before its first use; every kernel that uses it
 * leaves it zeroed when it completes. */
size_t mc_scratch_bytes(void);

/* Plain decode: one launch over meshlets [first, first + count), one warp per
 * meshlet (the baseline; a per-mesh decode issues one call per mesh).
 * Outputs (any of d_local / d_global may be NULL, d_pos may not; d_local and
 * d_global must be 16-byte aligned):
 *   d_local  u8  [3 * total_tris]  local triangle indices, meshlet m at
 *            3 * tri_base(m); degenerates are kept (Sec. 4.2)
 *   d_global u32 [3 * total_tris]  vertex_base(m) + local
 *   d_pos    f32 [3 * total_verts] FP32 positions (Sec. 4.4)
 * Triangle k with flag R is (I[k+1], old, I[k+2]), with flag L
 * (old, I[k+1], I[k+2]), where I is the strip stream (I[0..2] = 0,1,2) and
 * old = I[j+1] for the last j < k whose flag differs from flag k (I[0] if
 * none) -- the bit scan of Sec. 4.2; I[k+2] is the inclusive add-scan of the
 * increment flags (+2) or reuse entry k+1-s (Sec. 4.3). */
mc_status mc_decode_plain(const mc_device_batch *b, uint32_t first, uint32_t count,
                          uint8_t *d_local, uint32_t *d_global, float *d_pos,
                          uint32_t *d_status, const mc_tuning *t, void *stream);

/* Batched decode: all meshlets of the batch in one persistent launch whose
 * warps pull meshlets from a device work queue in d_scratch
 * (mc_scratch_bytes(), zeroed before first use).  Same outputs as
 * mc_decode_plain over the whole batch.  t = NULL: autotuned shape (or the
 * default if mc_autotune has not run for this batch signature). */
mc_status mc_decode_batch(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                          float *d_pos, uint32_t *d_status, void *d_scratch,
                          const mc_tuning *t, void *stream);

/* Batched decode into full vertices: as mc_decode_batch, but each decoded
 * vertex is written as 8 FP32 (32 bytes, the vertex layout of Sec. 5):
 * x, y, z, the n_attr attribute channels (b->attr_desc / attr_grids), and
 * zeros up to 8.  d_vertex: f32 [8 * total_verts], 16-byte aligned.
 * MC_ERR_INVALID_ARG if the batch has no attribute channels or their
 * records / grids are missing. */
mc_status mc_decode_batch_vertices(const mc_device_batch *b, uint8_t *d_local,
                                   uint32_t *d_global, float *d_vertex, uint32_t *d_status,
                                   void *d_scratch, const mc_tuning *t, void *stream);

/* One decode request of a serving batch: a range of meshlets of a resident
 * pool batch (e.g. one mesh of it) and the request's own output buffers.
 * Its decoded triangles and vertices are numbered from the range's first
 * meshlet: global index = (vertex_base(m) - vertex_base) + local. */
typedef struct {
  uint32_t first_meshlet; /* range of the pool batch */
  uint32_t n_meshlets;
  uint32_t work_start;    /* sum of n_meshlets of the requests before this one */
  uint32_t reserved0;
  uint32_t tri_base;      /* tri_base / vertex_base of first_meshlet */
  uint32_t vertex_base;
  uint32_t tri_count;     /* output capacity: sum of T' / V over the range */
  uint32_t vert_count;
  uint8_t *d_local;       /* u8 [3 tri_count] or NULL, 16-byte aligned */
  uint32_t *d_global;     /* u32 [3 tri_count] or NULL, 16-byte aligned */
  float *d_pos;           /* f32 [3 vert_count] */
  void *reserved1;
} mc_request;

/* Continuous-batching decode: the meshlet ranges of n_reqs requests (a device
 * array, work_start ascending, total_work = sum of n_meshlets) in one
 * persistent launch whose warps pull meshlets from the work queue in
 * d_scratch, each written to its request's buffers.  The decoded bits are
 * those of mc_decode_batch on the same meshlets (Sec. 4.2-4.4), only renumbered
 * per request, so a request decodes the same alone or in any mix. */
mc_status mc_decode_requests(const mc_device_batch *pool, const mc_request *d_reqs,
                             uint32_t n_reqs, uint32_t total_work, uint32_t *d_status,
                             void *d_scratch, const mc_tuning *t, void *stream);

/* Allocation-free form of mc_decode_batch (no counterpart in the paper: it
 * only changes where the decoder's scratch lives).  Some callers cannot hand
 * the library a scratch buffer: hosts that own every device allocation and
 * forbid libraries from allocating, or render loops where a cudaMalloc would
 * implicitly synchronise the device mid-frame.  This call takes no d_scratch;
 * the work-queue counters live in a 256-byte file-scope device array of the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The call allocates nothing (no cudaMalloc / cudaFree): it clears
 * the counters with cudaMemsetAsync on `stream` and launches the same kernel
 * with the same outputs and launch shapes as mc_decode_batch.
 *   - The first call on a device looks up the array's device address for
 *     that device (with that device current); make that first call before
 *     any stream capture.
 *   - All calls on a device share the array: calls whose kernels overlap on
 *     the GPU (e.g. on two streams) race and give wrong results; serialise
 *     them.
 *   - MC_ERR_LIMIT if the batch has more than 2^31 meshlets (the 32-bit
 *     counters need headroom) or the device ordinal is 64 or more.
 *   - The looked-up address is kept for the life of the process: after a
 *     cudaDeviceReset (or anything else that unloads the library's device
 *     code on that device) it is stale, and this call must not be used on
 *     that device again. */
mc_status mc_decode_batch_noalloc(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                                  float *d_pos, uint32_t *d_status, const mc_tuning *t,
                                  void *stream);

/* Fused decode + cull + compaction in one persistent launch: the decode of
 * mc_decode_batch (Sec. 4.2-4.4) with per-meshlet culling (Sec. 3: meshlets
 * are culled whole, by their bounds and normal cone, before their triangles)
 * and a per-triangle back-face test.
 *   d_view_proj  16 FP32, row-major clip matrix: clip = M [x y z 1]^T
 *   d_tri_out    u32 [3 * total_tris]: surviving triangles as global index
 *                triples, compacted in unspecified order
 *   d_tri_count  u32, receives the number of surviving triangles (the
 *                running count lives in d_scratch during the launch)
 *   d_pos        f32 [3 * total_verts], written for meshlets that pass the
 *                meshlet tests only
 * A meshlet is skipped when all 8 corners of its quantisation box
 * [L, L + 2^b - 1] lie outside one clip plane (-w <= x, y, z <= w), or --
 * when b->cones is set and the matrix has a camera position -- when its
 * normal cone faces away from that camera (mc_cone).  The camera position is
 * the point whose clip x, y and w are zero: rows r_i = M[i][0..2] and
 * b_i = -M[i][3] of rows 0, 1, 3 give, in FP64,
 *   e = (b0 (r1 x r3) + b1 (r3 x r0) + b3 (r0 x r1)) / (r0 . (r1 x r3)),
 * rounded to FP32 (none when the determinant is 0 or not finite); the cone
 * test is evaluated in FP32 as v = center - e, d = fma(a_z, v_z, fma(a_y,
 * v_y, a_x v_x)), l = sqrt(fma(v_z, v_z, fma(v_y, v_y, v_x v_x))), skip iff
 * s < 1 and d >= fma(s, l, radius).  A triangle is dropped when two of its
 * indices coincide (restart degenerates) or when all three clip w are
 * positive and the determinant of its (x, y, w) clip rows is not positive
 * (back-facing, counter-clockwise front faces).  Decoded indices never leave
 * the chip except as survivors. */
mc_status mc_decode_cull(const mc_device_batch *b, const float *d_view_proj,
                         uint32_t *d_tri_out, uint32_t *d_tri_count, float *d_pos,
                         uint32_t *d_status, void *d_scratch, const mc_tuning *t,
                         void *stream);

/* The fused cull (as mc_decode_cull, Sec. 3 and 4.2-4.4) against several
 * views in one persistent launch: each
 * meshlet is staged, dequantised and strip-walked once, then tested, culled
 * and compacted once per view whose meshlet tests it passes.
 *   d_view_projs  n_views x 16 FP32 row-major clip matrices, 1 <= n_views <= 8
 *   d_tri_out     u32; view v's survivors (global index triples, unspecified
 *                 order) at d_tri_out + v * tri_stride
 *   tri_stride    u32 elements per view region, >= 3 * total_tris
 *   d_tri_counts  u32 [n_views]: survivors per view
 *   d_pos         f32 [3 * total_verts], written for meshlets that pass the
 *                 meshlet tests of at least one view
 * Per view, the tests and their FP32 evaluation are mc_decode_cull's, so view
 * v's survivors are the ones mc_decode_cull returns for matrix v (as a set).
 * Uses d_scratch words 8-15 for the per-view counts; grabs hold at most 4
 * meshlets.  MC_ERR_INVALID_ARG for n_views outside 1..8 or a short stride. */
mc_status mc_decode_cull_views(const mc_device_batch *b, const float *d_view_projs,
                               uint32_t n_views, uint32_t *d_tri_out, uint64_t tri_stride,
                               uint32_t *d_tri_counts, float *d_pos, uint32_t *d_status,
                               void *d_scratch, const mc_tuning *t, void *stream);

/* The fused cull (as mc_decode_cull, Sec. 3 and 4.2-4.4) with the survivors
 * in a fixed order: meshlet order, then
 * triangle order within a meshlet -- the order of a sequential decode and
 * cull.  Same arguments and results as mc_decode_cull otherwise, plus
 *   d_order  device buffer of mc_cull_order_bytes(b) bytes, 8-byte aligned,
 *            library-owned for the duration of the call (cleared by it)
 * The order comes from a decoupled look-back over the work-queue grabs
 * (each warp publishes its grab's survivor count as soon as the grab is
 * decoded, and after its next grab sums the counts of the first grab's
 * predecessors back to the nearest published prefix); grabs hold at most 3
 * meshlets in this mode.  Every wait is bounded: a wait that gives up sets
 * MC_ERR_TIMEOUT in the status word.  Calls that overlap on the GPU must not
 * share d_order or d_scratch. */
size_t mc_cull_order_bytes(const mc_device_batch *b);
mc_status mc_decode_cull_ordered(const mc_device_batch *b, const float *d_view_proj,
                                 uint32_t *d_tri_out, uint32_t *d_tri_count, float *d_pos,
                                 uint32_t *d_status, void *d_scratch, void *d_order,
                                 const mc_tuning *t, void *stream);

/* ------------------------------------------------------------------ runtime */

/* Time candidate launch shapes of mc_decode_batch on this batch (the outputs
 * are overwritten) -- warps per CTA {4, 8, 16} x meshlets per grab {1, 2, 4,
 * 8, 16} x CTAs per SM {the occupancy limit, half of it} x lanes per meshlet
 * {32, 16} -- and remember the fastest for batches with the same
 * signature (meshlet count, payload size, largest block) on this device.
 * Each shape runs four times, each run after the positions have been
 * rewritten (which evicts the input from L2 when it is larger than L2, as
 * between frames); the best of the last three counts.  Synchronises
 * `stream`.  best (may be NULL) receives the chosen shape, best_ms (may be
 * NULL) its time. */
mc_status mc_autotune(const mc_device_batch *b, uint8_t *d_local, uint32_t *d_global,
                      float *d_pos, uint32_t *d_status, void *d_scratch, void *stream,
                      mc_tuning *best, float *best_ms);

/* CUDA-graph wrapper: mc_graph_capture_batch records one mc_decode_batch
 * launch (with fixed pointers) into an executable graph; mc_graph_launch
 * replays it on a stream. */
typedef struct mc_graph mc_graph;
mc_status mc_graph_capture_batch(const mc_device_batch *b, uint8_t *d_local,
                                 uint32_t *d_global, float *d_pos, uint32_t *d_status,
                                 void *d_scratch, const mc_tuning *t, void *stream,
                                 mc_graph **out);
/* Same for the fused culling kernel: the graph holds one launch per matrix in
 * d_view_projs (n_views x 16 FP32); launch i writes d_tri_count[i] (n_views
 * entries) and overwrites the same d_tri_out / d_pos. */
mc_status mc_graph_capture_cull(const mc_device_batch *b, const float *d_view_projs,
                                uint32_t n_views, uint32_t *d_tri_out, uint32_t *d_tri_count,
                                float *d_pos, uint32_t *d_status, void *d_scratch,
                                const mc_tuning *t, void *stream, mc_graph **out);
/* Same for the multi-view cull: ceil(n_views / 8) launches of
 * mc_decode_cull_views, launch i covering views 8 i .. 8 i + 7 (any n_views >=
 * 1); view v writes d_tri_counts[v] and region v mod 8 of d_tri_out (so
 * d_tri_out holds min(n_views, 8) regions of tri_stride words, which later
 * launches overwrite). */
mc_status mc_graph_capture_cull_views(const mc_device_batch *b, const float *d_view_projs,
                                      uint32_t n_views, uint32_t *d_tri_out, uint64_t tri_stride,
                                      uint32_t *d_tri_counts, float *d_pos, uint32_t *d_status,
                                      void *d_scratch, const mc_tuning *t, void *stream,
                                      mc_graph **out);
mc_status mc_graph_launch(mc_graph *g, void *stream);
void mc_graph_free(mc_graph *g);

/* Host-buffer decode (end to end): copies the host blob arrays of `v` into
 * the caller's device buffers d_desc / d_payload / d_grids, decodes them as
 * mc_decode_batch does and copies the outputs back into h_local / h_global /
 * h_pos (NULL = not copied).  The batch is cut into up to 8 chunks of
 * consecutive meshlets whose input copies, decodes and output copies run on
 * three library-owned streams (one set per device), so that chunk i's decode
 * overlaps chunk i+1's input and chunk i-1's output copies; the call is
 * ordered after earlier work on `stream` and later work on `stream` waits
 * for all of it.  Host buffers (the view's arrays included) should be pinned
 * for the copies to be asynchronous.  Concurrent calls from several host
 * threads enqueue one after another.  MC_ERR_CORRUPT if the host
 * descriptors' payload offsets, triangle or vertex bases are not
 * non-decreasing.  Asynchronous on `stream`. */
mc_status mc_decode_batch_host(const mc_blob_view_t *v, mc_desc *d_desc, uint8_t *d_payload,
                               mc_grid *d_grids, uint8_t *d_local, uint32_t *d_global,
                               float *d_pos, uint32_t *d_status, void *d_scratch,
                               uint8_t *h_local, uint32_t *h_global, float *h_pos,
                               const mc_tuning *t, void *stream);

/* Kernel launches this library has issued since load (all entry points). */
uint64_t mc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MESHLET_CODEC_H */
