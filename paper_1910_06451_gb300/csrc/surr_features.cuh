// Feature row of the learned surrogate (not part of the paper), shared by the
// training-path feature kernel and the fused inference kernel.
#pragma once

#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace fk {

// Per control point m < min(M, D + 1) (frame j = cj[m]): its position, then
// sin/cos of the joint values q_j and q_{j+1} (q_0 = q_{D+1} = 0): 7 values
// per point, zero-padded to kSurrIn, rounded to BF16.  Points beyond the
// first D + 1 (on the chains here: link midpoints, averages of two frame
// origins) add no information and are left out.  q: the D joint values of
// one query, or null for a row of zeros.
__device__ __forceinline__ void surr_feature_row(const ChainF &c, const float *q, bf16 (&h)[kSurrIn]) {
  float f[kSurrIn];
#pragma unroll
  for (int i = 0; i < kSurrIn; ++i) f[i] = 0.f;
  if (q) {
    float qv[FK_MAX_DOF + 2];
    qv[0] = 0.f;
    for (int i = 0; i < c.D; ++i) qv[i + 1] = q[i];
    qv[c.D + 1] = 0.f;
    PoseF P;
    pose_base(c, P);
    for (int fr = 0; fr <= c.D; ++fr) {
      if (fr > 0) pose_step(c, fr - 1, qv[fr], P);
      for (int m = 0; m < c.M && m <= c.D; ++m)
        if (c.cj[m] == fr) {
          float o[3];
          pose_point(P, c.ct[m], o);
          float s0, c0, s1, c1;
          sincosf(qv[fr], &s0, &c0);
          sincosf(qv[fr + 1], &s1, &c1);
          const int b = 7 * m;
          f[b + 0] = o[0];
          f[b + 1] = o[1];
          f[b + 2] = o[2];
          f[b + 3] = s0;
          f[b + 4] = c0;
          f[b + 5] = s1;
          f[b + 6] = c1;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < kSurrIn; ++i) h[i] = __float2bfloat16_rn(f[i]);
}

}  // namespace fk
