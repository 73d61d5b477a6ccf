// Device helpers shared by the fused cull kernels: clip-space rows, the
// camera position of a clip matrix and the normal-cone test.
#pragma once

#include "decode_warp.cuh"

namespace mcdev {

__device__ __forceinline__ float clip_row(const float *M, int r, float x, float y, float z) {
  return __fmaf_rn(M[4 * r + 2], z, __fmaf_rn(M[4 * r + 1], y, __fmaf_rn(M[4 * r + 0], x, M[4 * r + 3])));
}

// Rows 0, 1 and 3 of a clip matrix in registers (clip x, y and w), so that a
// loop whose shared-memory stores could alias the matrix does not reload it.
struct ClipRows {
  float m[12];
};
__device__ __forceinline__ ClipRows clip_rows(const float *M) {
  ClipRows c;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    c.m[i] = M[i];
    c.m[4 + i] = M[4 + i];
    c.m[8 + i] = M[12 + i];
  }
  return c;
}
// clip_row's operation order; r = 0, 1, 2 for rows 0, 1, 3
__device__ __forceinline__ float clip_dot(const ClipRows &c, int r, float x, float y, float z) {
  return __fmaf_rn(c.m[4 * r + 2], z,
                   __fmaf_rn(c.m[4 * r + 1], y, __fmaf_rn(c.m[4 * r + 0], x, c.m[4 * r + 3])));
}

// Camera position of a clip matrix M (row-major, in shared memory): the point
// whose clip x, y and w are zero, from rows r0, r1, r3 and b_i = -M[i][3] by
// the cross-product inverse in FP64,
//   e = (b0 (r1 x r3) + b1 (r3 x r0) + b3 (r0 x r1)) / (r0 . (r1 x r3)),
// rounded to FP32.  Returns false (no camera: affine projection) when the
// determinant is 0 or not finite, or a coordinate is not finite.
__device__ inline bool view_eye(const float *M, float *eye) {
  double r0[3], r1[3], r3[3];
  for (int c = 0; c < 3; c++) {
    r0[c] = M[c];
    r1[c] = M[4 + c];
    r3[c] = M[12 + c];
  }
  const double b0 = -(double)M[3], b1 = -(double)M[7], b3 = -(double)M[15];
  auto cross = [](const double *u, const double *v, double *w) {
    w[0] = __dsub_rn(__dmul_rn(u[1], v[2]), __dmul_rn(u[2], v[1]));
    w[1] = __dsub_rn(__dmul_rn(u[2], v[0]), __dmul_rn(u[0], v[2]));
    w[2] = __dsub_rn(__dmul_rn(u[0], v[1]), __dmul_rn(u[1], v[0]));
  };
  double k0[3], k1[3], k3[3];
  cross(r1, r3, k0);
  cross(r3, r0, k1);
  cross(r0, r1, k3);
  const double det =
      __dadd_rn(__dadd_rn(__dmul_rn(r0[0], k0[0]), __dmul_rn(r0[1], k0[1])), __dmul_rn(r0[2], k0[2]));
  if (!(det != 0.0) || !isfinite(det)) return false;
  for (int c = 0; c < 3; c++) {
    const double num =
        __dadd_rn(__dadd_rn(__dmul_rn(b0, k0[c]), __dmul_rn(b1, k1[c])), __dmul_rn(b3, k3[c]));
    const double e = __ddiv_rn(num, det);
    if (!isfinite(e)) return false;
    eye[c] = __double2float_rn(e);
  }
  return true;
}

// Normal-cone test (mc_cone) of one meshlet for a camera at eye: true when
// axis . v >= s |v| + radius with v = center - eye, in FP32 with a fixed
// operation order.
__device__ __forceinline__ bool cone_record_faces_away(const float4 c0, const float4 c1,
                                                       const float *eye) {
  const float vx = __fsub_rn(c0.x, eye[0]), vy = __fsub_rn(c0.y, eye[1]), vz = __fsub_rn(c0.z, eye[2]);
  const float d = __fmaf_rn(c1.z, vz, __fmaf_rn(c1.y, vy, __fmul_rn(c1.x, vx)));
  const float l = __fsqrt_rn(__fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx))));
  return (c1.w < 1.0f) & (d >= __fmaf_rn(c1.w, l, c0.w));
}
__device__ __forceinline__ bool cone_faces_away(const mc_cone *cone, const float *eye) {
  const float4 *p = reinterpret_cast<const float4 *>(cone);
  return cone_record_faces_away(__ldg(p), __ldg(p + 1), eye);  // center, radius / axis, s
}

__device__ __forceinline__ void sts_u32_if(uint32_t a, uint32_t x, bool p) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.shared.u32 [%0], %1;\n}" ::"r"(a),
               "r"(x), "r"((uint32_t)p)
               : "memory");
}

}  // namespace mcdev
