// The FP32 score of one block of queries against a whole support set, shared
// by the per-call kernel (score_f32_kernel) and the persistent multi-scene
// kernel.  See fk_score.cu for the arithmetic.
#pragma once

#include <cuda_fp16.h>

#include "fk_dfk.cuh"
#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace fk {

// Packed FP32x2 arithmetic: each 64-bit register holds the same quantity for
// the two support points of a pair.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 rcp2(f2 x) {
  float lo, hi;
  upk(x, lo, hi);
  return pk(rcp_approx(lo), rcp_approx(hi));
}

__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// 2^(-t) for t >= 0 (the Gaussian summand with the coordinates scaled by
// sqrt(gamma/2 log2 e)) on the MUFU unit, both halves.
__device__ __forceinline__ float ex2_neg(float t) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-t));
  return r;
}
__device__ __forceinline__ f2 ex2_neg2(f2 t) {
  float lo, hi;
  upk(t, lo, hi);
  return pk(ex2_neg(lo), ex2_neg(hi));
}

// 2^(-t) for t >= 0 on the FP32 pipe, both halves: t is clamped to 125 (the
// value is then below 2^-124, negligible beside the summand of 1 at t = 0),
// split as t = n + r with n = rint(t) (the 1.5 * 2^23 rounding constant puts n
// in the low bits of j) and r in [-1/2, 1/2]; 2^(-r) is a degree-5
// polynomial fitted to the relative error on [-1/2, 1/2] by iteratively
// reweighted least squares on Chebyshev nodes (7.5e-8 in exact arithmetic,
// 2.3e-7 with FP32 Horner steps), and 2^(-n) is applied by subtracting n from
// the exponent field: (bits(j) << 23) is n << 23 because the constant's own
// bits vanish in the shift.
__device__ __forceinline__ f2 ex2_neg2_poly(f2 t) {
  float t0, t1;
  upk(t, t0, t1);
  const f2 tc = pk(fminf(t0, 125.f), fminf(t1, 125.f));
  const f2 magic = pk(12582912.f, 12582912.f);
  const f2 j = add2(tc, magic);
  const f2 r = sub2(tc, sub2(j, magic));
  f2 p = pk(-1.327647129073739e-3f, -1.327647129073739e-3f);
  p = fma2(p, r, pk(9.675541892647743e-3f, 9.675541892647743e-3f));
  p = fma2(p, r, pk(-5.550713092088699e-2f, -5.550713092088699e-2f));
  p = fma2(p, r, pk(2.4022120237350464e-1f, 2.4022120237350464e-1f));
  p = fma2(p, r, pk(-6.931469440460205e-1f, -6.931469440460205e-1f));
  p = fma2(p, r, pk(1.0000001192092896f, 1.0000001192092896f));
  float p0, p1, j0, j1;
  upk(p, p0, p1);
  upk(j, j0, j1);
  return pk(__uint_as_float(__float_as_uint(p0) - (__float_as_uint(j0) << 23)),
            __uint_as_float(__float_as_uint(p1) - (__float_as_uint(j1) << 23)));
}

constexpr uint32_t kDrainLimit = 1u << 22;  // polls while draining copies after a timeout

// Number of control-point pairs that share one reciprocal: the rest take one
// MUFU reciprocal each.  A shared pair costs 3 more packed FP32 operations
// and 2 fewer reciprocals than two singles.  Per support pair and query a
// warp needs about 2 (7 Mv + 3 NP + 2) FP32-pipe cycles (packed operations
// take two) against 8 (2 Mv - 2 NP) MUFU cycles (4 lanes per sub-partition),
// plus the kinematics and folds on the FP32 pipe: NP = 0 balances the two
// at 7 points, NP = 1 at 11 and 12 (measured: 7 points 5.82 -> 5.78 ms,
// 11 points 121.0 -> 119.5 ms against the previous rule (Mv + 3) / 7).
template <int MV>
struct RcpPlan {
  static constexpr int NP = (MV + 5) / 14;
};

// (H, L) += x exactly up to the rounding of L: Knuth's two-sum on both
// halves of the packed registers.
__device__ __forceinline__ void fold2(f2 &H, f2 &L, f2 x) {
  const f2 s = add2(H, x);
  const f2 bb = sub2(s, H);
  const f2 e = add2(sub2(H, sub2(s, bb)), sub2(x, bb));
  H = s;
  L = add2(L, e);
}

struct BlockOut {
  float *f;            // [n] or null
  int8_t *label;       // [n]
  float eps0, eps1;    // band: |f| <= (eps0 + eps1 (|p(q)| + |s|max)) B(q)
  int32_t *band_idx;   // or null: no band list
  int32_t *band_scene; // or null: scene id of each band entry
  int32_t scene;
  int64_t idx_base;    // added to the local index in band_idx
  int32_t *band_cnt;
  int32_t *err;
  uint32_t wait_limit;
  const int32_t *npair_pos;  // [0] positive-weight pairs, which lead the records;
                             // [1] float bits of |s|max, the largest scaled support-point norm
  float cnorm;               // CIRC: the band takes max(|p(q)| + |s|max, cnorm)
};

// Scores queries q0 .. q0 + NTHR*Q - 1 (those below n) of the query array q
// (n x D) against the support records rec (ns points, (ns+1)/2 pair records,
// the o.npair_pos[0] positive-weight pairs first) with chain c.  tiles:
// 2 * TP * rec_len(MV) float4 of shared memory; bar: two mbarriers.  Every
// thread of the CTA must call it.  Returns false (in every thread) if a tile
// wait gave up; the caller must then stop using the CTA's barriers.
//
// Kinematics: each query's control points in pair arithmetic (fk_dfk.cuh),
// scaled by g = sqrt(gamma/2) (RQ) and rounded once to FP32, so a control
// point is off by at most u |p| (u = 2^-24).
// HALF = true: the differences and t = 1 + |d|^2 are computed in packed
// FP16 (HSUB2/HFMA2, query and support coordinates rounded to half), then
// widened to FP32 for the reciprocals and the accumulation.  HALF = false:
// all FP32.
// GAUSS = true: the non-paper Gaussian summand.  Coordinates come scaled by
// sqrt(gamma/2 log2 e), so the summand is 2^(-t) with t = |p - s|^2 (no
// "1 +"): on the MUFU unit (ex2.approx) for the first MV - POLY points of
// every support point and on the FP32 pipe (ex2_neg2_poly) for the last POLY;
// with HALF, t in packed FP16 and 2^(-t) by ex2.approx.f16x2 (two halves per
// MUFU operation), widened to FP32 for the sums.  No reciprocal sharing.
// CIRC = true (RQ in FP32 only): point 0, on the circle of a revolute
// joint 1 (ChainF::circ), takes t = 1 + D^2 with D = sin(theta/2) C -
// cos(theta/2) S from the record's circle entry (C, S) = 2 rho g (cos, sin)
// (theta_s / 2): one product and two FMAs in place of three differences and
// three FMAs.  D is 2 rho g sin((theta - theta_s) / 2), the scaled distance of
// the two points up to sign; sin and cos of theta / 2 come from pair
// arithmetic rounded once.  Its error is covered by the band term
// eps1 cnorm, cnorm = 6 rho g (section on the band in fkfast_api.cu).
// Accumulation: each pair adds w * acc into the sum of its sign (positive
// part P of f first, then the negative part N), kFoldPairs at a time in
// FP32, each partial folded into a pair accumulator (compensated summation:
// the accumulation error of f is then at most kFoldPairs + 3 units of
// roundoff of B(q), whatever the size of the support set); f = P + N and the
// bound B(q) = P - N = sum_s |w_s| sum_m K(s_m, q_m).
template <int MV, int Q, int TP, int NTHR, bool HALF = false, bool GAUSS = false, int POLY = 0, bool CIRC = false>
__device__ __forceinline__ bool score_block(const ChainF &c, const float4 *__restrict__ rec, int64_t ns, dd g,
                                            const float *__restrict__ q, int64_t n, int64_t q0, const BlockOut &o,
                                            float4 *tiles, uint64_t *bar) {
  static_assert(POLY >= 0 && POLY <= MV && (POLY == 0 || (GAUSS && !HALF)), "polynomial points: FP32 Gaussian only");
  static_assert(!CIRC || (!HALF && !GAUSS), "circle form: FP32 RQ only");
  constexpr int REC = rec_len(MV);
  constexpr int NP = RcpPlan<MV>::NP;

  const int tid = threadIdx.x;
  const int64_t npair = (ns + 1) / 2;
  const int ntiles = (int)((npair + TP - 1) / TP);
  const int64_t npp = (int64_t)o.npair_pos[0];  // pairs of the positive part
  const float smax = __int_as_float(o.npair_pos[1]);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int64_t p0 = (int64_t)t * TP;
    const int64_t cnt = npair - p0 < TP ? npair - p0 : TP;
    const uint32_t bytes = (uint32_t)(cnt * REC * sizeof(float4));
    uint64_t *b = &bar[t & 1];
    mbar_arrive_expect_tx(b, bytes);
    tma_bulk_load(tiles + (size_t)(t & 1) * TP * REC, rec + p0 * REC, bytes, b);
  };
  if (tid == 0) {
    if (ntiles > 0) issue(0);
    if (ntiles > 1) issue(1);
  }

  // forward kinematics of this thread's queries in pair arithmetic, scaled
  // so that t = 1 + |p - s|^2, rounded to FP32 and duplicated into both
  // halves of a packed register; s_eps: the query's band eps0 + eps1 (|p| + |s|max)
  const int64_t qbase = q0 + tid;
  f2 P[Q][MV][3];
  __half2 Ph[HALF ? Q : 1][HALF ? MV : 1][3];
  // per thread and query, outside the register file (touched once per
  // kFoldPairs pairs): the pair accumulator (AH, AL) of the current sign,
  // the finished positive part PF, and the query's band eps(q)
  __shared__ f2 s_acc[3][Q][NTHR];
  __shared__ float s_eps[Q][NTHR];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t qi = qbase + k * NTHR;
    float qv[FK_MAX_DOF];
    for (int i = 0; i < c.D; ++i) qv[i] = qi < n ? q[qi * c.D + i] : 0.f;
    float cp[MV][3];
    fk_points_dd<MV>(c, qv, g, cp);
    float pn = 0.f;
#pragma unroll
    for (int m = 0; m < MV; ++m) {
      pn = fmaxf(pn, sqrtf(fmaf(cp[m][0], cp[m][0], fmaf(cp[m][1], cp[m][1], cp[m][2] * cp[m][2]))));
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float v = cp[m][r];
        if (HALF)
          Ph[HALF ? k : 0][HALF ? m : 0][r] = __float2half2_rn(v);
        else
          P[k][m][r] = pk(v, v);
      }
    }
    if (CIRC) {
      // point 0: sin and cos of half the joint-1 angle (pair arithmetic,
      // rounded once), the cosine negated for the kernel's product
      dd th = dd_add(dd{c.th0[0], c.th0_l[0]}, dd_of(qv[0]));
      th.h *= 0.5f;
      th.l *= 0.5f;
      dd sh, ch;
      dd_sincos(th, sh, ch);
      const float sg = dd_round(sh), cg = dd_round(ch);
      P[k][0][0] = pk(sg, sg);
      P[k][0][1] = pk(-cg, -cg);
    }
    s_eps[k][tid] = fmaf(o.eps1, CIRC ? fmaxf(pn + smax, o.cnorm) : pn + smax, o.eps0);
    s_acc[0][k][tid] = s_acc[1][k][tid] = s_acc[2][k][tid] = pk(0.f, 0.f);
  }
  const __half2 one_h = __float2half2_rn(1.f);
  const f2 one2 = pk(1.f, 1.f);
  const f2 zero2 = pk(0.f, 0.f);
  const float nc = (float)c.n_const;
  const f2 nc2 = pk(nc, nc);

  // s_acc[0] + s_acc[1]: the pair accumulator of the current sign (P, then
  // N); s_acc[2]: P once it is complete
  bool neg = npp <= 0;  // accumulating the negative part (uniform over the CTA)
  int t_fail = -1;
  for (int t = 0; t < ntiles; ++t) {
    const bool got = mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, o.wait_limit);
    if (!__syncthreads_and(got)) {
      t_fail = t;
      break;
    }
    const float4 *tile = tiles + (size_t)(t & 1) * TP * REC;
    const int64_t p0 = (int64_t)t * TP;
    const int cnt = (int)(npair - p0 < TP ? npair - p0 : TP);
    // the summands of one support pair for this thread's queries
    auto pair_sums = [&](const float4 *r, f2 (&acc)[Q]) {
#pragma unroll
        for (int k = 0; k < Q; ++k) acc[k] = nc2;
        f2 tv[Q][MV];
#pragma unroll
        for (int m = 0; m < MV; ++m) {
          const float4 xy = r[m];
          const float4 zz = r[MV + m / 2];
          if (HALF) {
            const __half2 hx = __floats2half2_rn(xy.x, xy.y), hy = __floats2half2_rn(xy.z, xy.w);
            const __half2 hz = (m & 1) ? __floats2half2_rn(zz.z, zz.w) : __floats2half2_rn(zz.x, zz.y);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
              const int kk = HALF ? k : 0, mm = HALF ? m : 0;
              const __half2 dx = __hsub2(Ph[kk][mm][0], hx), dy = __hsub2(Ph[kk][mm][1], hy),
                            dz = __hsub2(Ph[kk][mm][2], hz);
              if (GAUSS) {
                // the summand itself: 2^(-t) for both support points in one MUFU operation
                const __half2 nt = __hneg2(__hfma2(dx, dx, __hfma2(dy, dy, __hmul2(dz, dz))));
                uint32_t e;
                asm("ex2.approx.f16x2 %0, %1;" : "=r"(e) : "r"(*reinterpret_cast<const uint32_t *>(&nt)));
                const float2 ef = __half22float2(*reinterpret_cast<const __half2 *>(&e));
                tv[k][m] = pk(ef.x, ef.y);
              } else {
                const float2 tf = __half22float2(__hfma2(dx, dx, __hfma2(dy, dy, __hfma2(dz, dz, one_h))));
                tv[k][m] = pk(tf.x, tf.y);
              }
            }
          } else if (CIRC && m == 0) {
            const float4 cs = r[REC - 2];
            const f2 C = pk(cs.x, cs.y), S = pk(cs.z, cs.w);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
              const f2 D = fma2(P[k][0][0], C, mul2(P[k][0][1], S));
              tv[k][0] = fma2(D, D, one2);
            }
          } else {
            const f2 sx = pk(xy.x, xy.y), sy = pk(xy.z, xy.w);
            const f2 sz = (m & 1) ? pk(zz.z, zz.w) : pk(zz.x, zz.y);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
              const f2 dx = sub2(P[k][m][0], sx), dy = sub2(P[k][m][1], sy), dz = sub2(P[k][m][2], sz);
              tv[k][m] = GAUSS ? fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))) : fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, one2)));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          if constexpr (GAUSS) {
#pragma unroll
            for (int m = 0; m < MV; ++m)
              acc[k] = add2(acc[k], HALF ? tv[k][m] : (m < MV - POLY ? ex2_neg2(tv[k][m]) : ex2_neg2_poly(tv[k][m])));
          } else {
            // pairs: 1/t1^2 + 1/t2^2 = (t1^2 + t2^2) / (t1 t2)^2
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
              const f2 t1 = tv[k][2 * pp], t2 = tv[k][2 * pp + 1];
              const f2 pr = mul2(t1, t2);
              const f2 num = fma2(t1, t1, mul2(t2, t2));
              acc[k] = fma2(num, rcp2(mul2(pr, pr)), acc[k]);
            }
#pragma unroll
            for (int m = 2 * NP; m < MV; ++m) {
              const f2 rr = rcp2(tv[k][m]);
              acc[k] = fma2(rr, rr, acc[k]);
            }
          }
        }
    };
    // eight support pairs per loop trip (four for more than 8 points, which
    // would spill otherwise): fewer loop and address instructions on a kernel
    // bound by instruction dispatch
    constexpr int UNR = MV > 8 ? 4 : 8;
    // pairs [0, js) of this tile belong to the positive part, [js, cnt) to the negative
    int64_t js64 = npp - p0;
    const int js = (int)(js64 < 0 ? 0 : (js64 > cnt ? cnt : js64));
    for (int j0 = 0; j0 < cnt;) {
      if (j0 >= js && !neg) {  // the positive part is complete
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          s_acc[2][k][tid] = add2(s_acc[0][k][tid], s_acc[1][k][tid]);
          s_acc[0][k][tid] = s_acc[1][k][tid] = zero2;
        }
        neg = true;
      }
      const int seg = j0 < js ? js : cnt;
      f2 part[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) part[k] = zero2;
      auto pair_step = [&](const float4 *r) {
        f2 acc[Q];
        pair_sums(r, acc);
        const float4 W = r[REC - 1];
        const f2 w = pk(W.x, W.y);
#pragma unroll
        for (int k = 0; k < Q; ++k) part[k] = fma2(w, acc[k], part[k]);
      };
      int j1;
      if (seg - j0 >= kFoldPairs) {  // a full partial: a loop of fixed length
        const float4 *r0 = tile + j0 * REC;
#pragma unroll UNR
        for (int jj = 0; jj < kFoldPairs; ++jj) pair_step(r0 + jj * REC);
        j1 = j0 + kFoldPairs;
      } else {
#pragma unroll 2
        for (int j = j0; j < seg; ++j) pair_step(tile + j * REC);
        j1 = seg;
      }
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        f2 H = s_acc[0][k][tid], L = s_acc[1][k][tid];
        fold2(H, L, part[k]);
        s_acc[0][k][tid] = H;
        s_acc[1][k][tid] = L;
      }
      j0 = j1;
    }
    __syncthreads();  // every thread is done with this buffer
    if (tid == 0 && t + 2 < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + 2);
    }
  }
  if (t_fail >= 0) {
    // give the copies still in flight (tiles t_fail and t_fail + 1) a
    // bounded chance to land before the CTA exits, then report
    if (tid == 0) {
      for (int t = t_fail; t < ntiles && t < t_fail + 2; ++t)
        mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, kDrainLimit);
      atomicOr(o.err, kErrTimeout);
    }
    return false;
  }
  if (!neg) {
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      s_acc[2][k][tid] = add2(s_acc[0][k][tid], s_acc[1][k][tid]);
      s_acc[0][k][tid] = s_acc[1][k][tid] = zero2;
    }
  }

  const unsigned lane = tid & 31;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    float p0v, p1v, n0v, n1v;
    upk(s_acc[2][k][tid], p0v, p1v);
    upk(add2(s_acc[0][k][tid], s_acc[1][k][tid]), n0v, n1v);
    const float pp = __fadd_rn(p0v, p1v), nn = __fadd_rn(n0v, n1v);
    const float f = __fadd_rn(pp, nn);
    const float bq = __fsub_rn(pp, nn);
    const int64_t qi = qbase + k * NTHR;
    const bool valid = qi < n;
    if (valid) {
      if (o.f) o.f[qi] = f;
      o.label[qi] = f >= 0.f ? 1 : -1;
    }
    if (o.band_idx) {
      const bool flag = valid && !(fabsf(f) > s_eps[k][tid] * bq);
      const unsigned bal = __ballot_sync(0xffffffffu, flag);
      if (bal) {
        int base = 0;
        if (lane == 0) base = atomicAdd(o.band_cnt, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (flag) {
          const int pos = base + __popc(bal & ((1u << lane) - 1u));
          o.band_idx[pos] = (int32_t)(o.idx_base + qi);
          if (o.band_scene) o.band_scene[pos] = o.scene;
        }
      }
    }
  }
  return true;
}

}  // namespace fk
