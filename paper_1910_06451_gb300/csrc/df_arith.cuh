// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32
// numbers (about 48 significant bits), manipulated with the error-free
// transformations two-sum (Knuth, TAOCP vol. 2, 4.2.2) and two-product by
// FMA (Dekker, Numer. Math. 18, 1971, with the splitting replaced by the
// fused product), so FP64-class accuracy comes from the FP32 pipes.  The
// sums and the products whose rounding error is recovered are written with
// the round-to-nearest intrinsics, which the compiler never fuses into an
// FMA (a fused product would no longer be the value the error term assumes).
#pragma once

#include "fk_ptx.cuh"

namespace fk {

struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
// a - b, accurate when the two cancel
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) {
  dfl s = two_sum(a.h, -b.h);
  s.l += a.l - b.l;
  return quick_two_sum(s.h, s.l);
}
// (h + l)^2 = h^2 + 2 h l (l^2 is below the precision); h^2 exactly by FMA
__device__ __forceinline__ dfl df_sqr(dfl a) {
  const float p = __fmul_rn(a.h, a.h);
  const float e = fmaf(a.h, a.h, -p);
  return quick_two_sum(p, fmaf(2.f * a.h, a.l, e));
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.h, -p);
  return quick_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
// sum of two non-negative values (no cancellation)
__device__ __forceinline__ dfl df_add_pos(dfl a, dfl b) {
  dfl s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return quick_two_sum(s.h, s.l);
}
// 1 / a for a >= 1: y = rcp(a.h) with relative error about 2^-23, then
// y + y (1 - a y) with the residual 1 - a y formed exactly (a.h y = p + pe by
// FMA, 1 - p exact since p is within a factor 2 of 1): error about 2^-46
__device__ __forceinline__ dfl df_rcp(dfl a) {
  const float y = rcp_approx(a.h);
  const float p = __fmul_rn(a.h, y);
  const float pe = fmaf(a.h, y, -p);
  const float e = ((1.f - p) - pe) - a.l * y;
  return quick_two_sum(y, __fmul_rn(y, e));
}


// One summand t^-2 of the FK kernel in pair arithmetic, t = 1 + |q - s|^2 in
// coordinates scaled by sqrt(gamma/2); q = qh + ql and s = (s[0] + s[1],
// s[2] + s[3], s[4] + s[5]) per axis.  Every step keeps its rounding error:
//   d = q - s      (dh, e) = two_sum(qh, -sh), dl = e + (ql - sl)
//   d^2            p = dh^2, e' = fma(dh, dh, -p) + dl (2 dh + dl)
//   t              th + tl = 1 + p_x + p_y + p_z (three two-sums) + sum of e'
//   t^2            uh = th^2, ul = fma(th, th, -uh) + 2 th tl
//   t^-2           y = rcp(uh), r = y + y (1 - uh y - ul y)
// Returns the unnormalised pair (y, y res); relative error ~1e-13 (the
// neglected square of the Newton residual is 2^-44).
__device__ __forceinline__ void df_rq_term(const float qh[3], const float ql[3], const float *s, float &rh,
                                           float &rl) {
  float p[3], ep[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const dfl d = two_sum(qh[r], -s[2 * r]);
    const float dl = d.l + (ql[r] - s[2 * r + 1]);
    p[r] = __fmul_rn(d.h, d.h);
    ep[r] = fmaf(dl, fmaf(2.f, d.h, dl), fmaf(d.h, d.h, -p[r]));
  }
  const dfl t1 = two_sum(1.f, p[0]);
  const dfl t2 = two_sum(t1.h, p[1]);
  const dfl t3 = two_sum(t2.h, p[2]);
  const float th = t3.h;
  const float tl = ((t1.l + t2.l) + t3.l) + ((ep[0] + ep[1]) + ep[2]);
  const float uh = __fmul_rn(th, th);
  const float ul = fmaf(2.f * th, tl, fmaf(th, th, -uh));
  const float y = rcp_approx(uh);
  const float res = fmaf(-ul, y, fmaf(-uh, y, 1.f));
  rh = y;
  rl = y * res;
}

// a + b for pairs of any signs
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return quick_two_sum(s.h, s.l);
}

// 1/k! for k = 0..12 as pairs, from FP64 (whose 53 bits cover the pair's 48)
struct InvFact {
  float h[13], l[13];
};
constexpr InvFact make_inv_fact() {
  InvFact c{};
  double v = 1.0;
  for (int k = 0; k <= 12; ++k) {
    if (k > 0) v /= (double)k;
    c.h[k] = (float)v;
    c.l[k] = (float)(v - (double)c.h[k]);
  }
  return c;
}
__constant__ constexpr InvFact kInvFact = make_inv_fact();
constexpr double kLn2 = 0.69314718055994530942;

// One Gaussian summand 2^(-t) (the non-paper summand, coordinates scaled by
// sqrt(gamma/2 log2 e)) in pair arithmetic, t = |q - s|^2 formed as in
// df_rq_term without the 1.  t = n + r with n = rint(t_h), r = (t_h - n) + t_l
// (the first difference is exact), 2^(-r) = e^(-r ln 2) by its Taylor series
// to the 12th power in pair Horner steps (|r ln 2| <= 0.347: the first
// neglected term is below 2e-16), then scaled by 2^(-n) exactly.  t_h > 125
// gives 0 (below 2^-125 of the largest summand).  Relative error about 1e-13
// plus ln 2 t times the relative error of t (2^-46).
__device__ __forceinline__ void df_gauss_term(const float qh[3], const float ql[3], const float *s, float &rh,
                                              float &rl) {
  float p[3], ep[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const dfl d = two_sum(qh[r], -s[2 * r]);
    const float dl = d.l + (ql[r] - s[2 * r + 1]);
    p[r] = __fmul_rn(d.h, d.h);
    ep[r] = fmaf(dl, fmaf(2.f, d.h, dl), fmaf(d.h, d.h, -p[r]));
  }
  const dfl t1 = two_sum(p[0], p[1]);
  const dfl t2 = two_sum(t1.h, p[2]);
  const float th = t2.h;
  const float tl = (t1.l + t2.l) + ((ep[0] + ep[1]) + ep[2]);
  if (th > 125.f) {
    rh = rl = 0.f;
    return;
  }
  const float n = rintf(th);
  const dfl r = two_sum(th - n, tl);
  const dfl ln2{(float)kLn2, (float)(kLn2 - (double)(float)kLn2)};
  const dfl mx = df_mul(dfl{-r.h, -r.l}, ln2);  // -r ln 2
  dfl y{kInvFact.h[12], kInvFact.l[12]};
#pragma unroll
  for (int k = 11; k >= 0; --k) y = df_add(df_mul(y, mx), dfl{kInvFact.h[k], kInvFact.l[k]});
  const float scale = __int_as_float((127 - (int)n) << 23);  // 2^(-n), n in [0, 125]
  rh = y.h * scale;
  rl = y.l * scale;
}

}  // namespace fk
