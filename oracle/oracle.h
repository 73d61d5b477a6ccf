/*
 * CPU oracle for GTS-Reuse meshlet compression
 * (Kuth et al., "Towards Practical Meshlet Compression", VMV 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential restatement of
 * the method used to check the library.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or constant with the library: every format constant below is
 * restated here on purpose.
 *
 * Pipeline (all host memory, plain C99, compiled with -ffp-contract=off):
 *   orc_meshletize   greedy meshlet growth under (V~, T~) limits (Sec. 3),
 *                    plus the split of meshlets whose strip, restarts
 *                    included, exceeds T~ (Sec. 4.2, last paragraph).
 *   orc_stripify     greedy generalized triangle strip of one meshlet with
 *                    one L/R flag per triangle (Sec. 2) and restarts emulated
 *                    by four degenerate triangles (Sec. 4.2).
 *   orc_encode       first-appearance relabelling, increment flags and reuse
 *                    buffer (Sec. 4.3), crack-free global-grid fixed-point
 *                    positions (Sec. 4.4), packed into the blob format.
 *   orc_decode_*     sequential strip walk (Sec. 2) -- deliberately NOT the
 *                    parallel closed form the GPU uses (Sec. 4.2/4.3) -- and
 *                    dequantisation to FP32 and FP64 (Sec. 4.4).
 *   orc_decode_cull  the same decode followed by a frustum test per meshlet
 *                    and a back-face/degenerate test per triangle.
 *
 * Blob format (little-endian):
 *   descriptor, 32 B per meshlet:
 *     u32 payload offset in 16-byte units, u32 vertex_base, u32 tri_base,
 *     u16 V, u16 T' (triangles incl. degenerates), u8 reuse width w
 *     (0 = plain GTS, below),
 *     u8 position bits b, u16 grid id, u32 L[3] (meshlet minimum on the grid)
 *   payload block per meshlet, u32 words, bits LSB-first, padded to 16 B:
 *     ceil(T'/32) L/R words (bit k = 1: triangle k entered across the right
 *     edge), ceil(T'/32) increment words (bit k = 1: new vertex),
 *     ceil(R*w/32) reuse words, ceil(3*V*b/32) position words
 *     (vertex v channel c at bit (3v+c)*b).  Bit 0 of both flag words is 0.
 *     Plain GTS (Sec. 4.2, w = 0): the L/R words, then one byte per
 *     triangle k >= 1 holding its stream entry I[k+2] (ceil((T'-1)/4)
 *     words), then the position words.
 *   grid entry, 32 B: f32 G[3], u32 b, f32 Delta[3], u32 mesh id.
 *   attribute words (blobs with n_attr extra channels): after the position
 *     words, ceil(n_attr*V*attr_bits/32) words, vertex v channel c at bit
 *     (n_attr*v + c)*attr_bits; attribute record, 32 B per meshlet: u32 La[5]
 *     (meshlet minimum on the attribute grid), u16 attribute grid id;
 *     attribute grid, 48 B: f32 G[5], f32 Delta[5], u32 attr_bits, u32 mesh id.
 *   normal cone, 32 B per meshlet (blob order), the per-meshlet cull data
 *   the paper keeps beside the offsets (Sec. 3, Sec. 5 "cull information"):
 *     f32 center[3], f32 radius   a sphere holding the decoded vertices,
 *     f32 axis[3], f32 s          unit axis of the cone holding every
 *                                 triangle normal and s = sine of its half
 *                                 angle plus 2^-20 (1 = no cone).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stddef.h>
#include <stdint.h>

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_LIMIT = 2,
  ORC_ERR_CORRUPT = 3,
  ORC_ERR_NOMEM = 5
};

/* Greedy meshletization.  Triangles are grouped into meshlets of at most
 * limits[2c] vertices and limits[2c+1] triangles for class c = tri_class[t]
 * (tri_class may be NULL: one class).  out_tri receives all triangle ids
 * grouped by meshlet, out_start (n_tris + 1 entries) the group starts.
 * Meshlets whose strip needs more than limits[2c+1] triangles once restart
 * degenerates are added are split in halves of their strip order.
 * *out_n_grown = meshlets before splitting. */
int orc_meshletize(uint32_t n_verts, const uint32_t *tris, uint32_t n_tris,
                   const uint8_t *tri_class, const uint32_t *limits,
                   uint32_t n_classes, uint32_t *out_tri, uint32_t *out_start,
                   uint32_t *out_n_meshlets, uint32_t *out_n_grown);

/* Greedy strip of the T triangles tris[ids[i]] (i = list position).
 * stream: T' + 2 global vertex ids; flags: T' entries (0 = L, 1 = R; entry 0
 * is 0); strip_order: the T list positions in strip order.
 * search_nodes > 0: the branch and bound of orc_min_strips then runs from the
 * greedy cover with that node budget, and the fewest-strips cover it finds is
 * taken when it has fewer strips than the greedy one; its strips are emitted
 * from each path end in list order that is not yet emitted, walking the path.
 * Capacity needed: stream 5*T, flags 5*T. */
int orc_stripify(const uint32_t *tris, const uint32_t *ids, uint32_t T, uint32_t search_nodes,
                 uint32_t *stream, uint8_t *flags, uint32_t *strip_order,
                 uint32_t *out_tp, uint32_t *out_strips);

/* Fewest strips (path cover of the triangles' adjacency graph) of the
 * triangles ids[0..T), by exhaustive branch and bound starting from the
 * greedy count greedy_strips (Sec. 4.1 maximises the used adjacency edges
 * under the same no-fork / no-cycle conditions).  *out_min = the minimum, or
 * 0 when the search needed more than max_nodes nodes (max_nodes = 0: not
 * searched); *out_lower = a lower bound valid at any size (each connected
 * part needs max(1, ceil(e / 2)) strips, e = its triangles with at most one
 * neighbour); *out_best (may be NULL) = the fewest strips the search found
 * within max_nodes nodes, proven minimal or not. */
int orc_min_strips(const uint32_t *tris, const uint32_t *ids, uint32_t T, uint32_t greedy_strips,
                   uint32_t max_nodes, uint32_t *out_min, uint32_t *out_lower, uint32_t *out_best);


typedef struct {
  uint32_t n_meshlets;
  uint32_t n_grids;
  uint64_t payload_bytes;
  uint64_t total_tris;  /* sum of T' */
  uint64_t total_verts; /* sum of V  */
  uint64_t restarts;
  uint64_t degenerates;
  uint64_t conn_bits;   /* sum of 2 T' + w R */
  uint64_t reuse_entries;
  uint8_t *desc;
  uint8_t *payload;
  uint8_t *grids;
  uint32_t *vmap; /* input vertex id of every decoded vertex (total_verts) */
  uint8_t *cones; /* 32 B normal cone per meshlet (blob order) */
  uint32_t n_attr, attr_bits; /* extra attribute channels (0..5) and their bits */
  uint8_t *adesc; /* 32 B attribute record per meshlet (blob order) */
  uint8_t *agrids; /* one 48 B attribute grid */
} orc_blob;

/* Encode the meshlets (mtri/mstart as produced by orc_meshletize) of one mesh.
 * bits[m]: position bits of meshlet m (1..32).  reuse_mode 0: w = 8,
 * reuse_mode 1: w = ceil(log2 V), reuse_mode 2: plain GTS (every stream
 * entry stored at 8 bits, no increment flags).  perm (may be NULL): blob slot p holds
 * meshlet perm[p].  mesh_id is written into the grid entries.  attrs (may be
 * NULL with n_attr = 0): n_attr (<= 5) extra attribute channels per input
 * vertex (attrs[n_attr v + c]), quantised crack-free at attr_bits bits on one
 * grid for the mesh, by the rules of the positions (Sec. 4.4).
 * strip_search_nodes: the node budget of the fewest-strips search per
 * meshlet (orc_stripify; 0 = the greedy strips). */
int orc_encode(const float *pos, uint32_t n_verts, const uint32_t *tris,
               const uint32_t *mtri, const uint32_t *mstart,
               uint32_t n_meshlets, const uint8_t *bits, uint32_t reuse_mode,
               const uint32_t *perm, uint32_t mesh_id, const float *attrs,
               uint32_t n_attr, uint32_t attr_bits, uint32_t strip_search_nodes, orc_blob **out);
void orc_blob_free(orc_blob *b);

/* FP32 dequantisation of a grid coordinate g (Sec. 4.4):
 *   g < 2^24:  x = fmaf((float)g, D, G)
 *   otherwise: x = fmaf((float)(g & 0xFFF), D, fmaf((float)(g >> 12), D * 4096, G)). */
float orc_dequant32(uint32_t g, float G, float D);

/* Sequential decode of one meshlet (descriptor desc32) into
 * local[3*T'] u8 indices, pos[3*V] FP32 and pos64[3*V] FP64 (may be NULL). */
int orc_decode_meshlet(const uint8_t *desc32, const uint8_t *payload,
                       uint64_t payload_bytes, const uint8_t *grids,
                       uint32_t n_grids, uint8_t *local, float *pos,
                       double *pos64);

/* Decode meshlets [first, first + count) into whole-batch outputs placed at
 * each meshlet's tri_base / vertex_base (any output may be NULL). */
int orc_decode(const uint8_t *desc, uint32_t n_meshlets, const uint8_t *payload,
               uint64_t payload_bytes, const uint8_t *grids, uint32_t n_grids,
               uint32_t first, uint32_t count, uint8_t *local, uint32_t *global,
               float *pos, double *pos64);

/* Decode + cull meshlets [first, first + count).  vp: row-major 4x4 clip
 * matrix.  Surviving triangles are appended to tri_out as global u32 triples
 * (meshlet order, then triangle order); *count_io is the running count in
 * triangles.  cones (may be NULL: no cone test): the blob's cone records; a
 * meshlet is then also dropped whole when the matrix has a camera position
 * (orc_view_eye) and orc_cone_test rejects it.  Positions are written only
 * for meshlets that pass both tests; pass_out[m] (may be NULL) receives 1
 * for those. */
int orc_decode_cull(const uint8_t *desc, uint32_t n_meshlets,
                    const uint8_t *payload, uint64_t payload_bytes,
                    const uint8_t *grids, uint32_t n_grids, uint32_t first,
                    uint32_t count, const float *vp, const uint8_t *cones,
                    uint32_t *tri_out, uint64_t *count_io, float *pos,
                    uint8_t *pass_out);

/* Decode the attribute channels of meshlets [first, first + count) of a blob
 * with n_attr channels at attr_bits bits (adesc / agrids: its attribute
 * records and grids): attr[n_attr * (vertex_base + v) + c] = FP32
 * dequantisation of La_c + q (the position formula, Sec. 4.4). */
int orc_decode_attrs(const uint8_t *desc, const uint8_t *adesc, uint32_t n_meshlets,
                     const uint8_t *payload, uint64_t payload_bytes, const uint8_t *agrids,
                     uint32_t n_agrids, uint32_t n_attr, uint32_t attr_bits, uint32_t first,
                     uint32_t count, float *attr);

/* Camera position of a clip matrix: the point whose clip x, y and w are all
 * zero (rows 0, 1, 3), solved in FP64 by the cross-product inverse
 *   e = (b0 (r1 x r3) + b1 (r3 x r0) + b3 (r0 x r1)) / (r0 . (r1 x r3)),
 * r_i = (M[i][0..2]), b_i = -M[i][3], and rounded to FP32.  Returns 0 (no
 * camera position: an affine projection) when the determinant is 0 or not
 * finite. */
int orc_view_eye(const float *vp, float eye[3]);

/* Normal-cone test of one meshlet (cone record cone32) for a camera at eye:
 * 1 when every triangle is back-facing, by the sufficient condition
 *   axis . (center - eye) >= s |center - eye| + radius,
 * evaluated in FP32 as d = fma(a_z, v_z, fma(a_y, v_y, a_x v_x)),
 * l = sqrt(fma(v_z, v_z, fma(v_y, v_y, v_x v_x))), reject iff s < 1 and
 * d >= fma(s, l, radius), with v = center - eye componentwise. */
int orc_cone_test(const uint8_t *cone32, const float eye[3]);

#endif
