// The FP32 score of one block of queries against a whole support set, shared
// by the per-call kernel (score_f32_kernel) and the persistent multi-scene
// kernel.  See fk_score.cu for the arithmetic.
#pragma once

#include <cuda_fp16.h>

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
// MUFU reciprocal each.  About a sixth of the points paired balances the FP32
// pipe (128 lanes/clk/SM) against the MUFU pipe (16 lanes/clk/SM).
template <int MV>
struct RcpPlan {
  static constexpr int NP = (MV + 3) / 7;
};

struct BlockOut {
  float *f;            // [n] or null
  int8_t *label;       // [n]
  float eps;           // band: |f| <= eps B(q)
  int32_t *band_idx;   // or null: no band list
  int32_t *band_scene; // or null: scene id of each band entry
  int32_t scene;
  int64_t idx_base;    // added to the local index in band_idx
  int32_t *band_cnt;
  int32_t *err;
  uint32_t wait_limit;
  const int32_t *npair_pos;  // SPLIT kernels: positive-weight pairs, which lead the records
};

// HALF = true: the differences and t = 1 + |d|^2 are computed in packed
// FP16 (HSUB2/HFMA2, query coordinates and the support pair's coordinates
// rounded to half), then widened to FP32 for the reciprocals and the
// accumulation.  HALF = false: all FP32.
// CP1 = true (FP32 only): record entry 0 holds (U_a, U_b, V_a, V_b) of the
// circle form of the first point (ChainF::cp1), t = A - U cos theta_q -
// V sin theta_q with A = 1 + k: two FMAs instead of three differences and
// three FMAs.  Its FP32 error for A < 8 stays within that of the direct
// form on the points farther out.
// GAUSS = true: the non-paper Gaussian summand.  Coordinates come scaled by
// sqrt(gamma/2 log2 e), so the summand is 2^(-t) with t = |p - s|^2 (no
// "1 +"): on the MUFU unit (ex2.approx) for the first MV - POLY points of
// every support point and on the FP32 pipe (ex2_neg2_poly) for the last POLY;
// with HALF, t in packed FP16 and 2^(-t) by ex2.approx.f16x2 (two halves per
// MUFU operation), widened to FP32 for the sums.  No reciprocal sharing, no
// circle form.
// Scores queries q0 .. q0 + NTHR*Q - 1 (those below n) of the query array q
// (n x D) against the support records rec (ns points, (ns+1)/2 pair records)
// with chain c.  tiles: 2 * TP * rec_len(MV) float4 of shared memory; bar: two
// mbarriers.  Every thread of the CTA must call it.  Returns false (in every
// thread) if a tile wait gave up; the caller must then stop using the CTA's
// barriers.
// SPLIT = true: the records hold the positive-weight pairs first
// (o.npair_pos of them, see rec_pairs), so each pair adds w * acc into one of
// two accumulators, the positive part P or the negative part N; f = P + N and
// B(q) = P - N, one packed FMA per pair and query instead of two.
template <int MV, int Q, int TP, int NTHR, bool HALF = false, bool CP1 = false, bool GAUSS = false, int POLY = 0,
          bool SPLIT = false>
__device__ __forceinline__ bool score_block(const ChainF &c, const float4 *__restrict__ rec, int64_t ns, float gs,
                                            const float *__restrict__ q, int64_t n, int64_t q0, const BlockOut &o,
                                            float4 *tiles, uint64_t *bar, float cp1_A = 0.f) {
  static_assert(!(HALF && CP1), "the circle form is an FP32 path");
  static_assert(!(GAUSS && CP1), "the circle form is an RQ path");
  static_assert(POLY >= 0 && POLY <= MV && (POLY == 0 || (GAUSS && !HALF)), "polynomial points: FP32 Gaussian only");
  constexpr int REC = MV + (MV + 1) / 2 + 1;
  constexpr int NP = RcpPlan<MV>::NP;

  const int tid = threadIdx.x;
  const int64_t npair = (ns + 1) / 2;
  const int ntiles = (int)((npair + TP - 1) / TP);
  const int64_t npp = SPLIT ? (int64_t)*o.npair_pos : 0;  // pairs of the positive part
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

  // forward kinematics of this thread's queries, scaled by sqrt(gamma/2) so
  // that t = 1 + |p - s|^2, duplicated into both halves of a packed register
  const int64_t qbase = q0 + tid;
  f2 P[Q][MV][3];
  __half2 Ph[HALF ? Q : 1][HALF ? MV : 1][3];
  f2 ncq[CP1 ? Q : 1], nsq[CP1 ? Q : 1];  // -cos theta_q, -sin theta_q of joint 1
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int64_t qi = qbase + k * NTHR;
    float qv[FK_MAX_DOF];
    for (int i = 0; i < c.D; ++i) qv[i] = qi < n ? q[qi * c.D + i] : 0.f;
    if (CP1) {
      float sn, cs;
      sincosf(qv[0] + c.th0[0], &sn, &cs);
      ncq[CP1 ? k : 0] = pk(-cs, -cs);
      nsq[CP1 ? k : 0] = pk(-sn, -sn);
    }
    float cp[MV][3];
    fk_points_f32<MV>(c, qv, cp);
#pragma unroll
    for (int m = 0; m < MV; ++m)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float v = gs * cp[m][r];
        if (HALF)
          Ph[HALF ? k : 0][HALF ? m : 0][r] = __float2half2_rn(v);
        else
          P[k][m][r] = pk(v, v);
      }
  }
  const __half2 one_h = __float2half2_rn(1.f);
  const f2 one2 = pk(1.f, 1.f);
  const f2 A2 = pk(cp1_A, cp1_A);
  const float nc = (float)c.n_const;
  const f2 nc2 = pk(nc, nc);

  f2 F[Q], B[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) F[k] = B[k] = pk(0.f, 0.f);
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
          if (CP1 && m == 0) {
            const f2 u = pk(xy.x, xy.y), v = pk(xy.z, xy.w);
#pragma unroll
            for (int k = 0; k < Q; ++k) tv[k][0] = fma2(u, ncq[CP1 ? k : 0], fma2(v, nsq[CP1 ? k : 0], A2));
          } else if (HALF) {
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
    // bound by instruction dispatch (4M 7-DOF queries: 5.25 ms one pair per
    // trip, 5.11 ms four, 5.06 ms eight), within 128 registers for two CTAs
    // per SM
    constexpr int UNR = MV > 8 ? 4 : 8;
    if constexpr (SPLIT) {
      int64_t js = npp - p0;
      js = js < 0 ? 0 : (js > cnt ? cnt : js);
#pragma unroll UNR
      for (int j = 0; j < (int)js; ++j) {
        const float4 *r = tile + j * REC;
        f2 acc[Q];
        pair_sums(r, acc);
        const float4 W = r[REC - 1];
        const f2 w = pk(W.x, W.y);
#pragma unroll
        for (int k = 0; k < Q; ++k) F[k] = fma2(w, acc[k], F[k]);
      }
#pragma unroll UNR
      for (int j = (int)js; j < cnt; ++j) {
        const float4 *r = tile + j * REC;
        f2 acc[Q];
        pair_sums(r, acc);
        const float4 W = r[REC - 1];
        const f2 w = pk(W.x, W.y);
#pragma unroll
        for (int k = 0; k < Q; ++k) B[k] = fma2(w, acc[k], B[k]);
      }
    } else {
#pragma unroll UNR
      for (int j = 0; j < cnt; ++j) {
        const float4 *r = tile + j * REC;
        f2 acc[Q];
        pair_sums(r, acc);
        const float4 W = r[REC - 1];
        const f2 w = pk(W.x, W.y), aw = pk(W.z, W.w);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          F[k] = fma2(w, acc[k], F[k]);
          B[k] = fma2(aw, acc[k], B[k]);
        }
      }
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

  const unsigned lane = tid & 31;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    float f0, f1, b0, b1;
    upk(F[k], f0, f1);
    upk(B[k], b0, b1);
    // SPLIT: F holds the positive part, B the negative part of f
    const float f = SPLIT ? (f0 + f1) + (b0 + b1) : f0 + f1;
    const float bq = SPLIT ? (f0 + f1) - (b0 + b1) : b0 + b1;
    const int64_t qi = qbase + k * NTHR;
    const bool valid = qi < n;
    if (valid) {
      if (o.f) o.f[qi] = f;
      o.label[qi] = f >= 0.f ? 1 : -1;
    }
    if (o.band_idx) {
      const bool flag = valid && fabsf(f) <= o.eps * bq;
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
