// Ground-truth collision labels on the GPU: sphere-swept links against
// axis-aligned boxes, decided as in FP64.  Link i is the segment between the origins of
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

// FP32 version of the same distance (used as a filter, see below).
__device__ float seg_box_d2_f32(const float p0[3], const float p1[3], const float *lo, const float *hi) {
  const float dp[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
  float ts[8];
  int nt = 0;
  ts[nt++] = 0.f;
  ts[nt++] = 1.f;
  for (int c = 0; c < 3; ++c) {
    if (dp[c] == 0.f) continue;
    const float bnd[2] = {lo[c], hi[c]};
    for (int b = 0; b < 2; ++b) {
      const float t = (bnd[b] - p0[c]) / dp[c];
      if (t > 0.f && t < 1.f) ts[nt++] = t;
    }
  }
  for (int x = 1; x < nt; ++x)
    for (int y = x; y > 0 && ts[y - 1] > ts[y]; --y) {
      const float tmp = ts[y];
      ts[y] = ts[y - 1];
      ts[y - 1] = tmp;
    }
  auto pb = [&](const float p[3]) {
    float s2 = 0.f;
    for (int c = 0; c < 3; ++c) {
      const float e = p[c] < lo[c] ? lo[c] - p[c] : (p[c] > hi[c] ? p[c] - hi[c] : 0.f);
      s2 = fmaf(e, e, s2);
    }
    return s2;
  };
  float best = fminf(pb(p0), pb(p1));
  for (int k = 0; k + 1 < nt; ++k) {
    const float ta = ts[k], tb = ts[k + 1], tm = 0.5f * (ta + tb);
    float sab = 0.f, sbb = 0.f;
    for (int c = 0; c < 3; ++c) {
      const float x = fmaf(tm, dp[c], p0[c]);
      float bound;
      if (x < lo[c])
        bound = lo[c];
      else if (x > hi[c])
        bound = hi[c];
      else
        continue;
      sab = fmaf(p0[c] - bound, dp[c], sab);
      sbb = fmaf(dp[c], dp[c], sbb);
    }
    float t = ta;
    if (sbb > 0.f) t = fminf(fmaxf(-sab / sbb, ta), tb);
    const float p[3] = {fmaf(t, dp[0], p0[0]), fmaf(t, dp[1], p0[1]), fmaf(t, dp[2], p0[2])};
    best = fminf(best, pb(p));
  }
  return best;
}

// One warp per configuration.  The lanes first decide every (link, box) pair
// in FP32: frame origins from the FP32 chain (error below 1e-6 m), distances
// from the FP32 version of the algorithm.  A pair whose FP32 distance is more
// than kLabelBand from the radius is decided by it; if any pair is decided as
// a hit the configuration collides.  Otherwise, if some pair was too close to
// call, the configuration is decided again entirely in FP64 exactly as
// before: lane 0 runs the FP64 chain and the lanes split the pairs.
constexpr int kLabelWarps = 8;
constexpr float kLabelBand = 1e-5f;  // metres, about ten times the FP32 position error

__global__ void __launch_bounds__(kLabelWarps * 32) label_kernel(const ChainF cf, const ChainD c, const Boxes bx,
                                                                  const float *__restrict__ q, int64_t n,
                                                                  int8_t *__restrict__ y) {
  __shared__ double org[kLabelWarps][FK_MAX_DOF + 1][3];
  __shared__ float orgf[kLabelWarps][FK_MAX_DOF + 1][3];
  __shared__ float boxf[kMaxBoxes][6];
  for (int e = threadIdx.x; e < bx.nb * 6; e += blockDim.x) boxf[e / 6][e % 6] = (float)bx.b[e / 6][e % 6];
  __syncthreads();
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t k = blockIdx.x * (int64_t)kLabelWarps + wl;
  if (k >= n) return;  // whole warp
  if (lane == 0) {
    PoseF P;
    pose_base(cf, P);
    orgf[wl][0][0] = P.p[0];
    orgf[wl][0][1] = P.p[1];
    orgf[wl][0][2] = P.p[2];
    for (int i = 0; i < cf.D; ++i) {
      pose_step(cf, i, q[k * cf.D + i], P);
      orgf[wl][i + 1][0] = P.p[0];
      orgf[wl][i + 1][1] = P.p[1];
      orgf[wl][i + 1][2] = P.p[2];
    }
  }
  __syncwarp();
  const float r = sqrtf((float)bx.r2);
  const float r_in = (r - kLabelBand) * (r - kLabelBand), r_out = (r + kLabelBand) * (r + kLabelBand);
  bool hit = false, unsure = false;
  const int pairs = c.D * bx.nb;
  for (int e = lane; e < pairs; e += 32) {
    const int i = e / bx.nb, b = e % bx.nb;
    const float d2 = seg_box_d2_f32(orgf[wl][i], orgf[wl][i + 1], boxf[b], boxf[b] + 3);
    if (d2 <= r_in && r > kLabelBand)
      hit = true;
    else if (!(d2 > r_out))
      unsure = true;
  }
  const unsigned any_hit = __ballot_sync(0xffffffffu, hit);
  const unsigned any_unsure = __ballot_sync(0xffffffffu, unsure);
  if (any_hit || !any_unsure) {
    if (lane == 0) y[k] = any_hit ? 1 : -1;
    return;
  }
  // too close to call in FP32: decide in FP64
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
  bool hit64 = false;
  for (int e = lane; e < pairs && !hit64; e += 32) {
    const int i = e / bx.nb, b = e % bx.nb;
    hit64 = seg_box_d2(org[wl][i], org[wl][i + 1], bx.b[b], bx.b[b] + 3) <= bx.r2;
  }
  const unsigned any64 = __ballot_sync(0xffffffffu, hit64);
  if (lane == 0) y[k] = any64 ? 1 : -1;
}

cudaError_t launch_label(const ChainF &cf, const ChainD &c, const Boxes &bx, const float *q, int64_t n, int8_t *y,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  label_kernel<<<(unsigned)((n + kLabelWarps - 1) / kLabelWarps), kLabelWarps * 32, 0, s>>>(cf, c, bx, q, n, y);
  return cudaGetLastError();
}

}  // namespace fk
