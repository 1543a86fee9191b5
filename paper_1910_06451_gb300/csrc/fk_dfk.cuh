// Forward kinematics (Sec. II-A, Eqs. 1-2) of one configuration in pair
// ("double-float") arithmetic, for the score kernels.
//
// Why: the FP32 score decides a label from f(q) alone whenever
// |f| > eps(q) B(q), so eps(q) must bound the whole FP32 error, the
// kinematics included.  An FP32 chain accumulates the rounding of every
// rotation product and the 1-2 ulp error of every sine and cosine along the
// lever arms of the joints after it; a worst-case bound for seven joints is
// several hundred units of roundoff in the control points, far above the
// rest of the error budget.  Computed here, the only error of a control
// point that matters is its final rounding to FP32.
//
// Values are unevaluated sums h + l of two FP32 numbers, combined with the
// error-free transformations two-sum (Knuth, TAOCP vol. 2, 4.2.2) and
// two-product by FMA (Dekker, Numer. Math. 18, 1971).  The pairs are kept
// unnormalised between operations ("sloppy" pair arithmetic): the low part
// may exceed half an ulp of the high part, but every quantity of the chain is
// bounded (rotation entries by 1, positions by the reach), so each operation
// adds an ABSOLUTE error of a few u^2 times the magnitudes it combines
// (u = 2^-24).  Over a chain of D joints that stays below 2^-36 of the
// reach, which is what the error bound of the score needs.
//
// Sine and cosine: theta = k pi/2 + r with k = rint(theta 2/pi) and r formed
// exactly enough by subtracting k times a three-float split of pi/2 (Cody and
// Waite, "Software Manual for the Elementary Functions", 1980), |r| <= pi/4;
// sin r and cos r by their Taylor series to the r^15 and r^16 terms (the
// first omitted terms are below 2^-55): the leading five coefficients of each
// in pair Horner steps, the small tail in FP32; the quadrant swaps and
// negates.  The coefficients are 1/n! and pi/2 from FP64, whose 53 bits
// cover what the pairs hold.  Valid for |theta| < 2^16.
#pragma once

#include <cstdint>

#include "fk_device.cuh"

namespace fk {

struct dd {
  float h, l;
};

__device__ __forceinline__ dd dd_of(float x) { return {x, 0.f}; }
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.h, -a.l}; }

// a b: the product of the high parts exactly (FMA), the cross terms added,
// a.l b.l dropped (below u^2 |a b| for normalised inputs)
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return {p, e};
}

// a + b: two-sum of the high parts, the low parts added (not renormalised)
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

// renormalise so that |l| <= ulp(h)/2
__device__ __forceinline__ dd dd_norm(dd a) {
  const float s = __fadd_rn(a.h, a.l);
  return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

// the pair rounded to the nearest FP32 value (one rounding of h + l)
__device__ __forceinline__ float dd_round(dd a) { return __fadd_rn(a.h, a.l); }

// Coefficients of the Taylor series of sin r / r and cos r in r^2, as pairs:
// kSinC[j] = (-1)^j / (2j + 1)!, kCosC[j] = (-1)^j / (2j)!, j = 0..8.
struct TrigCoef {
  float sh[9], sl[9], ch[9], cl[9];
  float p0, p1, p2;  // pi/2 = p0 + p1 + p2 (to FP64's 53 bits)
};
constexpr TrigCoef make_trig_coef() {
  TrigCoef c{};
  double f = 1.0;  // (n)! as n runs 0, 1, 2, ...
  for (int n = 0; n <= 17; ++n) {
    if (n > 0) f *= (double)n;
    const double v = ((n / 2) % 2 ? -1.0 : 1.0) / f;
    if (n % 2 == 0 && n / 2 <= 8) {
      c.ch[n / 2] = (float)v;
      c.cl[n / 2] = (float)(v - (double)(float)v);
    }
    if (n % 2 == 1 && n / 2 <= 8) {
      c.sh[n / 2] = (float)v;
      c.sl[n / 2] = (float)(v - (double)(float)v);
    }
  }
  const double pio2 = 1.57079632679489661923;
  c.p0 = (float)pio2;
  c.p1 = (float)(pio2 - (double)c.p0);
  c.p2 = (float)(pio2 - (double)c.p0 - (double)c.p1);
  return c;
}
__constant__ constexpr TrigCoef kTrig = make_trig_coef();

// sin and cos of theta (a pair), |theta| < 2^16.  Absolute error about 2^-44
// (checked exhaustively over the FP32 angles of [-8, 8] against FP64).
__device__ __forceinline__ void dd_sincos(dd th, dd &sn, dd &cs) {
  const float k = rintf(th.h * 0.636619772f);  // the nearest multiple of pi/2; |r| <= pi/4 + 2^-10
  // r = theta - k pi/2: k p0 and k p1 as exact products, k p2 rounded
  const float kp0 = __fmul_rn(k, kTrig.p0), kp0e = fmaf(k, kTrig.p0, -kp0);
  const float kp1 = __fmul_rn(k, kTrig.p1), kp1e = fmaf(k, kTrig.p1, -kp1);
  dd r = dd_add(th, dd{-kp0, -kp0e});
  r = dd_add(r, dd{-kp1, -kp1e});
  r.l = __fsub_rn(r.l, __fmul_rn(k, kTrig.p2));
  r = dd_norm(r);
  dd r2 = dd_norm(dd_mul(r, r));
  // tails in FP32: the terms from r^11 (sine) and r^10 (cosine) on are below
  // 2^-24 in magnitude, so their own rounding stays below 2^-48
  float ys = fmaf(fmaf(kTrig.sh[7], r2.h, kTrig.sh[6]), r2.h, kTrig.sh[5]);
  float yc = fmaf(fmaf(fmaf(kTrig.ch[8], r2.h, kTrig.ch[7]), r2.h, kTrig.ch[6]), r2.h, kTrig.ch[5]);
  dd S = dd_of(ys), C = dd_of(yc);
#pragma unroll
  for (int j = 4; j >= 0; --j) {
    S = dd_add(dd_mul(S, r2), dd{kTrig.sh[j], kTrig.sl[j]});
    C = dd_add(dd_mul(C, r2), dd{kTrig.ch[j], kTrig.cl[j]});
  }
  const dd s0 = dd_norm(dd_mul(r, dd_norm(S)));
  const dd c0 = dd_norm(C);
  const int q = ((int)k) & 3;
  const dd a = (q & 1) ? c0 : s0;   // sin of theta up to sign
  const dd b = (q & 1) ? s0 : c0;   // cos of theta up to sign
  sn = (q & 2) ? dd_neg(a) : a;
  cs = ((q + 1) & 2) ? dd_neg(b) : b;
}

// Frame pose in pairs: rotation columns x, y, z and origin p.
struct PoseDD {
  dd x[3], y[3], z[3], p[3];
};

__device__ __forceinline__ void pose_base(const ChainF &c, PoseDD &P) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    P.x[r] = dd{c.R0[3 * r + 0], c.R0_l[3 * r + 0]};
    P.y[r] = dd{c.R0[3 * r + 1], c.R0_l[3 * r + 1]};
    P.z[r] = dd{c.R0[3 * r + 2], c.R0_l[3 * r + 2]};
    P.p[r] = dd{c.p0[r], c.p0_l[r]};
  }
}

// Link i: R <- R Rz(theta) Rx(alpha), p <- p + R Rz(theta) (a, 0, d), the
// product of Eq. 1 taken column by column.  A twist near +-pi/2
// (ChainF::quarter: the high word of sin(alpha) is +-1 and |cos(alpha)| <
// 2^-20) is a signed swap of the y and z columns plus small corrections
// formed in FP32 (the cosine times the other column's high word, the low word
// of the sine times the column's high word): the terms dropped are below
// 2^-40 of a unit entry.
// rot = false: only the origin is needed after this link (the rotation is
// left as it was).  The pairs are not renormalised: each step adds at most a
// few u^2 of absolute error to entries bounded by 1 (rotation) or the reach.
__device__ __forceinline__ void pose_step(const ChainF &c, int i, float qi, PoseDD &P, bool rot = true) {
  dd theta{c.th0[i], c.th0_l[i]}, dlen{c.d[i], c.d_l[i]};
  if (c.type[i] == FK_REVOLUTE)
    theta = dd_add(theta, dd_of(qi));
  else
    dlen = dd_add(dlen, dd_of(qi));
  dd s, co;
  dd_sincos(theta, s, co);
  const dd a{c.a[i], c.a_l[i]};
  const dd ca{c.ca[i], c.ca_l[i]}, sa{c.sa[i], c.sa_l[i]};
  const bool quarter = c.quarter[i] != 0;
  const float sgn = c.sa[i];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const dd xn = dd_add(dd_mul(co, P.x[r]), dd_mul(s, P.y[r]));
    P.p[r] = dd_add(P.p[r], dd_add(dd_mul(a, xn), dd_mul(dlen, P.z[r])));
    if (!rot) continue;
    const dd yn = dd_add(dd_mul(co, P.y[r]), dd_mul(dd_neg(s), P.x[r]));
    dd zn, yy;
    if (quarter) {
      // zn = ca z - sa yn, yy = ca yn + sa z with sa = sgn + sa.l, sgn = +-1
      zn = dd{-sgn * yn.h, fmaf(ca.h, P.z[r].h, fmaf(-sa.l, yn.h, -sgn * yn.l))};
      yy = dd{sgn * P.z[r].h, fmaf(ca.h, yn.h, fmaf(sa.l, P.z[r].h, sgn * P.z[r].l))};
    } else {
      zn = dd_add(dd_mul(ca, P.z[r]), dd_mul(dd_neg(sa), yn));
      yy = dd_add(dd_mul(ca, yn), dd_mul(sa, P.z[r]));
    }
    P.x[r] = xn;
    P.y[r] = yy;
    P.z[r] = zn;
  }
}

// Configuration-dependent control point v: pos(pose * Trans(t_v)) (Eq. 2)
// times the coordinate scale g = gh + gl, rounded once to FP32.
__device__ __forceinline__ void pose_point_scaled(const ChainF &c, const PoseDD &P, int v, dd g, float out[3]) {
  const dd t0{c.vt[v][0], c.vt_l[v][0]}, t1{c.vt[v][1], c.vt_l[v][1]}, t2{c.vt[v][2], c.vt_l[v][2]};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    dd w = P.p[r];
    if (c.vt_nz[v]) w = dd_add(w, dd_add(dd_mul(P.x[r], t0), dd_add(dd_mul(P.y[r], t1), dd_mul(P.z[r], t2))));
    out[r] = dd_round(dd_mul(g, dd_norm(w)));
  }
}

// The configuration-dependent control points of configuration q, scaled by
// g and rounded to FP32: cp[v] = fl(g FK_v(q)) up to the pair error.
template <int MV>
__device__ __forceinline__ void fk_points_dd(const ChainF &c, const float *q, dd g, float (&cp)[MV][3]) {
  PoseDD P;
  pose_base(c, P);
#pragma unroll
  for (int m = 0; m < MV; ++m)
    if (c.vj[m] == 0) pose_point_scaled(c, P, m, g, cp[m]);
  for (int i = 0; i < c.D; ++i) {
    pose_step(c, i, q[i], P, i + 1 < c.D || c.rot_last);
#pragma unroll
    for (int m = 0; m < MV; ++m)
      if (c.vj[m] == i + 1) pose_point_scaled(c, P, m, g, cp[m]);
  }
}

}  // namespace fk
