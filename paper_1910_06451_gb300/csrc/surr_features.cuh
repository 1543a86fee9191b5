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
//
// Every loop has a compile-time bound, so the row stays in registers: DC > 0
// is a chain of exactly DC joints, DC = 0 any chain up to FK_MAX_DOF joints
// (longer unrolled code).  Both give the same values.
template <int DC>
__device__ __forceinline__ void surr_feature_row_t(const ChainF &c, const float *q, bf16 (&h)[kSurrIn]) {
  constexpr int DMAX = DC > 0 ? DC : FK_MAX_DOF;
  const int D = DC > 0 ? DC : c.D;
  const bf16 zero = __float2bfloat16_rn(0.f);
#pragma unroll
  for (int i = 0; i < kSurrIn; ++i) h[i] = zero;
  if (q) {
    // sin/cos of q_0 .. q_{D+1}, each computed once (q_0 = q_{D+1} = 0)
    float sq[DMAX + 2], cq[DMAX + 2];
#pragma unroll
    for (int i = 0; i < DMAX + 2; ++i) {
      sq[i] = 0.f;
      cq[i] = 1.f;
      if (i >= 1 && i <= D) sincosf(q[i - 1], &sq[i], &cq[i]);
    }
    PoseF P;
    pose_base(c, P);
#pragma unroll
    for (int fr = 0; fr <= DMAX; ++fr) {
      if (fr > D) break;
      if (fr > 0) pose_step(c, fr - 1, q[fr - 1], P);
#pragma unroll
      for (int m = 0; m <= DMAX && 7 * m + 6 < kSurrIn; ++m)
        if (m <= D && m < c.M && c.cj[m] == fr) {
          float o[3];
          pose_point(P, c.ct[m], o);
          h[7 * m + 0] = __float2bfloat16_rn(o[0]);
          h[7 * m + 1] = __float2bfloat16_rn(o[1]);
          h[7 * m + 2] = __float2bfloat16_rn(o[2]);
          h[7 * m + 3] = __float2bfloat16_rn(sq[fr]);
          h[7 * m + 4] = __float2bfloat16_rn(cq[fr]);
          h[7 * m + 5] = __float2bfloat16_rn(sq[fr + 1]);
          h[7 * m + 6] = __float2bfloat16_rn(cq[fr + 1]);
        }
    }
  }
}

__device__ __forceinline__ void surr_feature_row(const ChainF &c, const float *q, bf16 (&h)[kSurrIn]) {
  switch (c.D) {
    case 7: surr_feature_row_t<7>(c, q, h); break;
    case 3: surr_feature_row_t<3>(c, q, h); break;
    default: surr_feature_row_t<0>(c, q, h); break;
  }
}

}  // namespace fk
