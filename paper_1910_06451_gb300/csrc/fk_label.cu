// Ground-truth collision labels on the GPU: sphere-swept links against
// axis-aligned boxes, in FP64.  Link i is the segment between the origins of
// frames i-1 and i.  The squared segment-to-box distance g(t) is convex and
// quadratic between the parameters where a coordinate crosses a slab face;
// each piece is minimised in closed form and g is evaluated at the clamped
// minimiser and at both ends.  A configuration collides (+1) when some link
// comes within the radius of some box (touching counts), else it is free (-1).
#include "fk_internal.h"

namespace fk {

__device__ __forceinline__ double point_box_d2(const double p[3], const double *lo, const double *hi) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double e = 0.0;
    if (p[c] < lo[c])
      e = __dsub_rn(lo[c], p[c]);
    else if (p[c] > hi[c])
      e = __dsub_rn(p[c], hi[c]);
    s = __dadd_rn(s, __dmul_rn(e, e));
  }
  return s;
}

__device__ double seg_box_d2(const double p0[3], const double p1[3], const double *lo, const double *hi) {
  const double dp[3] = {__dsub_rn(p1[0], p0[0]), __dsub_rn(p1[1], p0[1]), __dsub_rn(p1[2], p0[2])};
  double ts[8];
  int nt = 0;
  ts[nt++] = 0.0;
  ts[nt++] = 1.0;
  for (int c = 0; c < 3; ++c) {
    if (dp[c] == 0.0) continue;
    const double bnd[2] = {lo[c], hi[c]};
    for (int b = 0; b < 2; ++b) {
      const double t = __ddiv_rn(__dsub_rn(bnd[b], p0[c]), dp[c]);
      if (t > 0.0 && t < 1.0) ts[nt++] = t;
    }
  }
  for (int x = 1; x < nt; ++x)
    for (int y = x; y > 0 && ts[y - 1] > ts[y]; --y) {
      const double tmp = ts[y];
      ts[y] = ts[y - 1];
      ts[y - 1] = tmp;
    }
  double best = INFINITY;
  for (int k = 0; k + 1 < nt; ++k) {
    const double ta = ts[k], tb = ts[k + 1];
    const double tm = __dmul_rn(0.5, __dadd_rn(ta, tb));
    double sab = 0.0, sbb = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double x = __dadd_rn(p0[c], __dmul_rn(tm, dp[c]));
      double bound;
      if (x < lo[c])
        bound = lo[c];
      else if (x > hi[c])
        bound = hi[c];
      else
        continue;
      const double A = __dsub_rn(p0[c], bound), B = dp[c];
      sab = __dadd_rn(sab, __dmul_rn(A, B));
      sbb = __dadd_rn(sbb, __dmul_rn(B, B));
    }
    double t = ta;
    if (sbb > 0.0) {
      t = __ddiv_rn(-sab, sbb);
      if (t < ta) t = ta;
      if (t > tb) t = tb;
    }
    const double p[3] = {__dadd_rn(p0[0], __dmul_rn(t, dp[0])), __dadd_rn(p0[1], __dmul_rn(t, dp[1])),
                         __dadd_rn(p0[2], __dmul_rn(t, dp[2]))};
    const double g = point_box_d2(p, lo, hi);
    if (g < best) best = g;
  }
  const double g0 = point_box_d2(p0, lo, hi), g1 = point_box_d2(p1, lo, hi);
  if (g0 < best) best = g0;
  if (g1 < best) best = g1;
  return best;
}

// One warp per configuration: lane 0 runs the FP64 chain and leaves the D+1
// frame origins in shared memory, then the lanes split the D x nb (link, box)
// pairs and a ballot gives the label.
constexpr int kLabelWarps = 8;

__global__ void __launch_bounds__(kLabelWarps * 32) label_kernel(const ChainD c, const Boxes bx,
                                                                  const float *__restrict__ q, int64_t n,
                                                                  int8_t *__restrict__ y) {
  __shared__ double org[kLabelWarps][FK_MAX_DOF + 1][3];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t k = blockIdx.x * (int64_t)kLabelWarps + wl;
  if (k >= n) return;  // whole warp
  if (lane == 0) {
    PoseD P;
    pose_base(c, P);
    org[wl][0][0] = P.T[3];
    org[wl][0][1] = P.T[7];
    org[wl][0][2] = P.T[11];
    for (int i = 0; i < c.D; ++i) {
      pose_step(c, i, (double)q[k * c.D + i], P);
      org[wl][i + 1][0] = P.T[3];
      org[wl][i + 1][1] = P.T[7];
      org[wl][i + 1][2] = P.T[11];
    }
  }
  __syncwarp();
  bool hit = false;
  const int pairs = c.D * bx.nb;
  for (int e = lane; e < pairs && !hit; e += 32) {
    const int i = e / bx.nb, b = e % bx.nb;
    hit = seg_box_d2(org[wl][i], org[wl][i + 1], bx.b[b], bx.b[b] + 3) <= bx.r2;
  }
  const unsigned any = __ballot_sync(0xffffffffu, hit);
  if (lane == 0) y[k] = any ? 1 : -1;
}

cudaError_t launch_label(const ChainD &c, const Boxes &bx, const float *q, int64_t n, int8_t *y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  label_kernel<<<(unsigned)((n + kLabelWarps - 1) / kLabelWarps), kLabelWarps * 32, 0, s>>>(c, bx, q, n, y);
  return cudaGetLastError();
}

}  // namespace fk
