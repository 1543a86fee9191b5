// Device-side building blocks shared by the fkfast kernels: chain parameters
// passed by value to every kernel, and forward kinematics in FP32 and FP64
// (Das and Yip, arXiv 1910.06451, Sec. II-A, Eqs. 1-2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fkfast.h"

namespace fk {

// Error bits a kernel may raise in the workspace error word.
enum : int { kErrTimeout = 1, kErrCapacity = 2, kErrIndex = 4 };

// Kinematic chain in the form the FP32 kernels use.  Control points fixed to
// frame 0 (the base) have the same position for every configuration, so
// their RQ summand is exactly 1; they are counted in n_const and the FP32
// score kernels evaluate only the Mv configuration-dependent points.
struct ChainF {
  int D, M, Mv, n_const;
  int type[FK_MAX_DOF];
  float a[FK_MAX_DOF], ca[FK_MAX_DOF], sa[FK_MAX_DOF], d[FK_MAX_DOF], th0[FK_MAX_DOF];
  float R0[9], p0[3];           // base rotation (row-major) and translation
  int vj[FK_MAX_CP];            // frame of each configuration-dependent point
  float vt[FK_MAX_CP][3];       // its offset in that frame
  int vidx[FK_MAX_CP];          // its index among all M points
  int cj[FK_MAX_CP];            // frame of every point (fk_forward output order)
  float ct[FK_MAX_CP][3];
  int summand;  // FK_SUMMAND_RQ or FK_SUMMAND_GAUSS
  // Low parts of the FP64 parameters (value = float field + low part, about
  // 48 bits), for the pair-arithmetic kinematics of the score kernels.
  float a_l[FK_MAX_DOF], ca_l[FK_MAX_DOF], sa_l[FK_MAX_DOF], d_l[FK_MAX_DOF], th0_l[FK_MAX_DOF];
  float R0_l[9], p0_l[3];
  float vt_l[FK_MAX_CP][3];
  int vt_nz[FK_MAX_CP];         // offset of configuration-dependent point v is not zero
  // Twist near +-pi/2: the high word of sin(alpha) is +-1 and |cos(alpha)| <
  // 2^-20, so Rx(alpha) is a signed swap of the y and z columns plus FP32
  // corrections (fk_dfk.cuh).
  int quarter[FK_MAX_DOF];
  int rot_last;                 // a configuration-dependent point on frame D has an offset
  float reach;                  // sum over links of |a| + |d| + |theta0 or d offset| bound, plus
                                // |p0| and the largest offset (metres): bounds every lever arm
  int circ;                     // configuration-dependent point 0 sits on frame 1 of a revolute
                                // joint 1, so it moves on a circle about that joint's axis
};

// The same chain for the FP64 kernels.  cos/sin of the link twists are taken
// on the host once.  The FP64 code evaluates Eq. 1 and the product of Eq. 2
// with separately rounded products and sums in a fixed order (no fused
// multiply-add), so that its rounding is that of the plain 4x4 product.
struct ChainD {
  int D, M, Mv, n_const;
  int vidx[FK_MAX_CP];          // indices of the configuration-dependent points
  int type[FK_MAX_DOF];
  double a[FK_MAX_DOF], ca[FK_MAX_DOF], sa[FK_MAX_DOF], d[FK_MAX_DOF], th0[FK_MAX_DOF];
  double T0[12];                // rows 0..2 of the base transform
  int cj[FK_MAX_CP];
  double ct[FK_MAX_CP][3];
  int summand;  // FK_SUMMAND_RQ or FK_SUMMAND_GAUSS
  int circ;           // as ChainF::circ
  double circ_rho;    // radius of that circle (metres): the distance of point 0
                      // from joint 1's axis
};

// ------------------------------------------------------------------ FP32 --
// Pose of the current frame: rotation columns x, y, z and origin p.
struct PoseF {
  float x[3], y[3], z[3], p[3];
};

__device__ __forceinline__ void pose_base(const ChainF &c, PoseF &P) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    P.x[r] = c.R0[3 * r + 0];
    P.y[r] = c.R0[3 * r + 1];
    P.z[r] = c.R0[3 * r + 2];
    P.p[r] = c.p0[r];
  }
}

// Advance the pose by link i: R <- R Rz(theta) Rx(alpha), p <- p + R (a c, a s, d).
__device__ __forceinline__ void pose_step(const ChainF &c, int i, float qi, PoseF &P) {
  float theta = c.th0[i], dd = c.d[i];
  if (c.type[i] == FK_REVOLUTE)
    theta += qi;
  else
    dd += qi;
  float s, co;
  sincosf(theta, &s, &co);
  const float ca = c.ca[i], sa = c.sa[i], a = c.a[i];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float xn = co * P.x[r] + s * P.y[r];
    float yn = co * P.y[r] - s * P.x[r];
    P.p[r] += a * xn + dd * P.z[r];
    float zn = ca * P.z[r] - sa * yn;
    P.y[r] = ca * yn + sa * P.z[r];
    P.z[r] = zn;
    P.x[r] = xn;
  }
}

__device__ __forceinline__ void pose_point(const PoseF &P, const float t[3], float out[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) out[r] = P.p[r] + P.x[r] * t[0] + P.y[r] * t[1] + P.z[r] * t[2];
}

// Configuration-dependent control points of one configuration (FP32).
template <int MV>
__device__ __forceinline__ void fk_points_f32(const ChainF &c, const float *q, float (&cp)[MV][3]) {
  PoseF P;
  pose_base(c, P);
#pragma unroll
  for (int m = 0; m < MV; ++m)
    if (c.vj[m] == 0) pose_point(P, c.vt[m], cp[m]);
  for (int i = 0; i < c.D; ++i) {
    pose_step(c, i, q[i], P);
#pragma unroll
    for (int m = 0; m < MV; ++m)
      if (c.vj[m] == i + 1) pose_point(P, c.vt[m], cp[m]);
  }
}

// ------------------------------------------------------------------ FP64 --
// Rows 0..2 of the frame transform; row 3 is (0, 0, 0, 1).
struct PoseD {
  double T[12];
};

__device__ __forceinline__ void pose_base(const ChainD &c, PoseD &P) {
#pragma unroll
  for (int k = 0; k < 12; ++k) P.T[k] = c.T0[k];
}

// T <- T * A_i with A_i of Eq. 1.  Each entry is the sum over k of
// T[r][k] A[k][c] taken in ascending k with every product rounded; terms with
// an exact zero factor in A are left out (adding an exact zero is exact).
__device__ __forceinline__ void pose_step(const ChainD &c, int i, double qi, PoseD &P) {
  double theta = c.th0[i], dd = c.d[i];
  if (c.type[i] == FK_REVOLUTE)
    theta = __dadd_rn(theta, qi);
  else
    dd = __dadd_rn(dd, qi);
  double st, ct;
  sincos(theta, &st, &ct);
  const double ca = c.ca[i], sa = c.sa[i], a = c.a[i];
  const double A01 = __dmul_rn(-ca, st), A11 = __dmul_rn(ca, ct);
  const double A02 = __dmul_rn(sa, st), A12 = __dmul_rn(-sa, ct);
  const double A03 = __dmul_rn(a, ct), A13 = __dmul_rn(a, st);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double t0 = P.T[4 * r + 0], t1 = P.T[4 * r + 1], t2 = P.T[4 * r + 2], t3 = P.T[4 * r + 3];
    P.T[4 * r + 0] = __dadd_rn(__dmul_rn(t0, ct), __dmul_rn(t1, st));
    P.T[4 * r + 1] = __dadd_rn(__dadd_rn(__dmul_rn(t0, A01), __dmul_rn(t1, A11)), __dmul_rn(t2, sa));
    P.T[4 * r + 2] = __dadd_rn(__dadd_rn(__dmul_rn(t0, A02), __dmul_rn(t1, A12)), __dmul_rn(t2, ca));
    P.T[4 * r + 3] =
        __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(t0, A03), __dmul_rn(t1, A13)), __dmul_rn(t2, dd)), t3);
  }
}

// pos(T * Trans(t)) with the products and sums in ascending order.
__device__ __forceinline__ void pose_point(const PoseD &P, const double t[3], double out[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    out[r] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(P.T[4 * r + 0], t[0]), __dmul_rn(P.T[4 * r + 1], t[1])),
                                 __dmul_rn(P.T[4 * r + 2], t[2])),
                       P.T[4 * r + 3]);
}

// FP64 reciprocal of x in [1, 2^100]: an FP32 MUFU estimate (relative error
// about 2^-23) refined by two Newton-Raphson steps y <- y + y (1 - x y),
// each of which squares the relative error; the result is within an ulp or
// so of 1/x.  It replaces the IEEE division, which is a long instruction
// sequence on a part whose FP64 rate is 1/64 of its FP32 rate.
__device__ __forceinline__ double rcp_f64(double x) {
  float xf = __double2float_rn(x), yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
  double y = (double)yf;
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// RQ summand of Eq. 3 in FP64: (1 + (gamma/2) |x - x'|^2)^-2.
__device__ __forceinline__ double k_rq_f64(double hg, const double *x, const double *xp) {
  const double d0 = x[0] - xp[0], d1 = x[1] - xp[1], d2 = x[2] - xp[2];
  const double t = fma(hg, fma(d0, d0, fma(d1, d1, d2 * d2)), 1.0);
  return rcp_f64(t * t);
}

// The non-paper Gaussian summand in FP64: exp(-(gamma/2) |x - x'|^2).
__device__ __forceinline__ double k_gauss_f64(double hg, const double *x, const double *xp) {
  const double d0 = x[0] - xp[0], d1 = x[1] - xp[1], d2 = x[2] - xp[2];
  return exp(-hg * fma(d0, d0, fma(d1, d1, d2 * d2)));
}

// The chain's summand in FP64 (hg = gamma / 2).
__device__ __forceinline__ double k_sum_f64(int summand, double hg, const double *x, const double *xp) {
  return summand == FK_SUMMAND_GAUSS ? k_gauss_f64(hg, x, xp) : k_rq_f64(hg, x, xp);
}

}  // namespace fk
