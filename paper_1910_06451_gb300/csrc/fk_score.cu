// Proxy collision check: the Fastron model value f(q) = sum_s alpha_s
// K_FK(S_s, q) with the FK kernel of Eq. 4 and its sign (Sec. III-B).
//
// Three kernels:
//   pack     support set -> per support point s one record of Mv + 1 float4:
//            for each configuration-dependent control point m,
//            (-gamma s_m, 1 + gamma/2 |s_m|^2), then (w_s, |w_s|, 0, 0) with
//            w_s = alpha_s / M; plus the FP64 control points for re-scoring.
//            All from FP64 kinematics, rounded to FP32 once.
//   score    FP32.  One thread scores two queries: FK in registers, then the
//            support records stream through shared memory by tile (1-D TMA
//            bulk copies, double-buffered, mbarrier completion) and every
//            thread reads each record as a broadcast.  Per (s, m):
//              t = (c_sm + gamma/2 |p_m|^2) + s'_m . p_m  = 1 + gamma/2 |p_m - s_m|^2
//            and two summands share one reciprocal:
//              1/t1^2 + 1/t2^2 = (t1^2 + t2^2) / (t1 t2)^2.
//            Beside f the kernel accumulates B(q) = sum_s |w_s| sum_m t^-2,
//            which bounds |f| and scales the FP32 error; queries with
//            |f| <= eps B(q) are appended to a band list.
//   rescore  FP64, one warp per band query: FK and Eq. 3/4 in FP64 with the
//            operation order of the plain definition, lanes splitting the
//            support set, a fixed-order warp sum; f and the label are replaced.
#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace fk {

// ---------------------------------------------------------------- pack ---
// One thread per pair of support points (2j, 2j+1); an odd count is padded
// with a point of weight 0.
__global__ void pack_kernel(const ChainF cf, const ChainD cd, const PackArgs a) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t npair = (a.ns + 1) / 2;
  if (j >= npair) return;
  const int MV = cf.Mv;
  const int REC = rec_len(MV);
  float4 *rec = a.rec + j * REC;
  const double gs = sqrt(0.5 * a.gamma);
  float cpv[2][FK_MAX_CP][3];
  float w[2], aw[2];
  for (int h = 0; h < 2; ++h) {
    const int64_t s = 2 * j + h;
    if (s >= a.ns) {
      for (int v = 0; v < MV; ++v) cpv[h][v][0] = cpv[h][v][1] = cpv[h][v][2] = 0.f;
      w[h] = aw[h] = 0.f;
      continue;
    }
    const int64_t src = a.idx ? (int64_t)a.idx[s] : s;
    const double *x = a.X + src * cd.D;
    double cp[FK_MAX_CP][3];
    PoseD P;
    pose_base(cd, P);
    for (int m = 0; m < cd.M; ++m)
      if (cd.cj[m] == 0) pose_point(P, cd.ct[m], cp[m]);
    for (int i = 0; i < cd.D; ++i) {
      a.q_out[s * cd.D + i] = x[i];
      pose_step(cd, i, x[i], P);
      for (int m = 0; m < cd.M; ++m)
        if (cd.cj[m] == i + 1) pose_point(P, cd.ct[m], cp[m]);
    }
    for (int m = 0; m < cd.M; ++m)
      for (int r = 0; r < 3; ++r) a.cp64[(m * 3 + r) * a.ns + s] = cp[m][r];
    const double al = a.alpha[s];
    a.alpha_out[s] = al;
    for (int v = 0; v < MV; ++v)
      for (int r = 0; r < 3; ++r) cpv[h][v][r] = (float)(gs * cp[cf.vidx[v]][r]);
    const double wd = al / cd.M;
    w[h] = (float)wd;
    aw[h] = (float)fabs(wd);
  }
  for (int v = 0; v < MV; ++v) rec[v] = make_float4(cpv[0][v][0], cpv[1][v][0], cpv[0][v][1], cpv[1][v][1]);
  for (int v = 0; v < MV; v += 2) {
    const bool two = v + 1 < MV;
    rec[MV + v / 2] = make_float4(cpv[0][v][2], cpv[1][v][2], two ? cpv[0][v + 1][2] : 0.f,
                                  two ? cpv[1][v + 1][2] : 0.f);
  }
  rec[REC - 1] = make_float4(w[0], w[1], aw[0], aw[1]);
}

cudaError_t launch_pack_support(const ChainF &cf, const ChainD &cd, const PackArgs &a, cudaStream_t s) {
  if (a.ns <= 0) return cudaSuccess;
  const int64_t npair = (a.ns + 1) / 2;
  pack_kernel<<<(unsigned)((npair + 127) / 128), 128, 0, s>>>(cf, cd, a);
  return cudaGetLastError();
}

// --------------------------------------------------------------- score ---
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

constexpr int kScoreThreads = 256;
constexpr int kQ = 2;                          // queries per thread
constexpr int kQueriesPerCta = kScoreThreads * kQ;
constexpr int kTilePairs = 64;                 // support pairs per shared-memory tile
constexpr uint32_t kDrainLimit = 1u << 22;     // polls while draining copies after a timeout

// Number of control-point pairs that share one reciprocal: the rest take one
// MUFU reciprocal each.  About a sixth of the points paired balances the FP32
// pipe (128 lanes/clk/SM) against the MUFU pipe (16 lanes/clk/SM).
template <int MV>
struct RcpPlan {
  static constexpr int NP = (MV + 3) / 7;
};

template <int MV>
__global__ void __launch_bounds__(kScoreThreads, 2) score_f32_kernel(const ChainF c, const ScoreArgs a) {
  extern __shared__ __align__(128) float4 tiles[];  // [2][kTilePairs][REC]
  __shared__ __align__(8) uint64_t bar[2];
  constexpr int REC = MV + (MV + 1) / 2 + 1;
  constexpr int NP = RcpPlan<MV>::NP;

  const int tid = threadIdx.x;
  const int64_t npair = (a.ns + 1) / 2;
  const int ntiles = (int)((npair + kTilePairs - 1) / kTilePairs);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int64_t p0 = (int64_t)t * kTilePairs;
    const int64_t cnt = npair - p0 < kTilePairs ? npair - p0 : kTilePairs;
    const uint32_t bytes = (uint32_t)(cnt * REC * sizeof(float4));
    uint64_t *b = &bar[t & 1];
    mbar_arrive_expect_tx(b, bytes);
    tma_bulk_load(tiles + (size_t)(t & 1) * kTilePairs * REC, a.rec + p0 * REC, bytes, b);
  };
  if (tid == 0) {
    if (ntiles > 0) issue(0);
    if (ntiles > 1) issue(1);
  }

  // forward kinematics of this thread's queries, scaled by sqrt(gamma/2) so
  // that t = 1 + |p - s|^2, duplicated into both halves of a packed register
  const int64_t qbase = (int64_t)blockIdx.x * kQueriesPerCta + tid;
  f2 P[kQ][MV][3];
#pragma unroll
  for (int k = 0; k < kQ; ++k) {
    const int64_t qi = qbase + k * kScoreThreads;
    float qv[FK_MAX_DOF];
    for (int i = 0; i < c.D; ++i) qv[i] = qi < a.n ? a.q[qi * c.D + i] : 0.f;
    float cp[MV][3];
    fk_points_f32<MV>(c, qv, cp);
#pragma unroll
    for (int m = 0; m < MV; ++m)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float v = a.gs * cp[m][r];
        P[k][m][r] = pk(v, v);
      }
  }
  const f2 one2 = pk(1.f, 1.f);
  const float nc = (float)c.n_const;
  const f2 nc2 = pk(nc, nc);

  f2 F[kQ], B[kQ];
#pragma unroll
  for (int k = 0; k < kQ; ++k) F[k] = B[k] = pk(0.f, 0.f);
  int t_fail = -1;
  for (int t = 0; t < ntiles; ++t) {
    const bool got = mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, a.wait_limit);
    if (!__syncthreads_and(got)) {
      t_fail = t;
      break;
    }
    const float4 *tile = tiles + (size_t)(t & 1) * kTilePairs * REC;
    const int64_t p0 = (int64_t)t * kTilePairs;
    const int cnt = (int)(npair - p0 < kTilePairs ? npair - p0 : kTilePairs);
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
      const float4 *r = tile + j * REC;
      f2 acc[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) acc[k] = nc2;
      f2 tv[kQ][MV];
#pragma unroll
      for (int m = 0; m < MV; ++m) {
        const float4 xy = r[m];
        const float4 zz = r[MV + m / 2];
        const f2 sx = pk(xy.x, xy.y), sy = pk(xy.z, xy.w);
        const f2 sz = (m & 1) ? pk(zz.z, zz.w) : pk(zz.x, zz.y);
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
          const f2 dx = sub2(P[k][m][0], sx), dy = sub2(P[k][m][1], sy), dz = sub2(P[k][m][2], sz);
          tv[k][m] = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, one2)));
        }
      }
#pragma unroll
      for (int k = 0; k < kQ; ++k) {
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
      const float4 W = r[REC - 1];
      const f2 w = pk(W.x, W.y), aw = pk(W.z, W.w);
#pragma unroll
      for (int k = 0; k < kQ; ++k) {
        F[k] = fma2(w, acc[k], F[k]);
        B[k] = fma2(aw, acc[k], B[k]);
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
      atomicOr(a.err, kErrTimeout);
    }
    return;
  }

  const unsigned lane = tid & 31;
#pragma unroll
  for (int k = 0; k < kQ; ++k) {
    float f0, f1, b0, b1;
    upk(F[k], f0, f1);
    upk(B[k], b0, b1);
    const float f = f0 + f1, bq = b0 + b1;
    const int64_t qi = qbase + k * kScoreThreads;
    const bool valid = qi < a.n;
    if (valid) {
      if (a.f) a.f[qi] = f;
      a.label[qi] = f >= 0.f ? 1 : -1;
    }
    if (a.band_idx) {
      const bool flag = valid && fabsf(f) <= a.eps * bq;
      const unsigned bal = __ballot_sync(0xffffffffu, flag);
      if (bal) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.band_cnt, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (flag) a.band_idx[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)qi;
      }
    }
  }
}

}  // namespace fk

namespace fk {

template <int MV>
static cudaError_t launch_score_mv(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  constexpr int REC = MV + (MV + 1) / 2 + 1;
  const size_t smem = 2 * (size_t)kTilePairs * REC * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(score_f32_kernel<MV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.n + kQueriesPerCta - 1) / kQueriesPerCta);
  score_f32_kernel<MV><<<grid, kScoreThreads, smem, s>>>(c, a);
  return cudaGetLastError();
}

// Shapes with a compiled score kernel: the number of configuration-dependent
// control points.
bool score_supported(int mv) {
  switch (mv) {
    case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 11: case 12:
      return true;
    default:
      return false;
  }
}

cudaError_t launch_score_f32(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  switch (c.Mv) {
    case 1: return launch_score_mv<1>(c, a, s);
    case 2: return launch_score_mv<2>(c, a, s);
    case 3: return launch_score_mv<3>(c, a, s);
    case 4: return launch_score_mv<4>(c, a, s);
    case 5: return launch_score_mv<5>(c, a, s);
    case 6: return launch_score_mv<6>(c, a, s);
    case 7: return launch_score_mv<7>(c, a, s);
    case 8: return launch_score_mv<8>(c, a, s);
    case 11: return launch_score_mv<11>(c, a, s);
    case 12: return launch_score_mv<12>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------- rescore ---
constexpr int kRescoreWarps = 8;

__global__ void __launch_bounds__(kRescoreWarps * 32) rescore_f64_kernel(const ChainD c, const RescoreArgs a) {
  __shared__ double qcp[kRescoreWarps][FK_MAX_CP][3];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t gw = blockIdx.x * (int64_t)kRescoreWarps + wl;
  const int64_t nw = (int64_t)gridDim.x * kRescoreWarps;
  const int64_t cnt = *a.band_cnt;
  const double hg = 0.5 * a.gamma;
  for (int64_t e = gw; e < cnt; e += nw) {
    const int64_t k = a.band_idx[e];
    if (lane == 0) {
      PoseD P;
      pose_base(c, P);
      for (int m = 0; m < c.M; ++m)
        if (c.cj[m] == 0) pose_point(P, c.ct[m], qcp[wl][m]);
      for (int i = 0; i < c.D; ++i) {
        pose_step(c, i, (double)a.q[k * c.D + i], P);
        for (int m = 0; m < c.M; ++m)
          if (c.cj[m] == i + 1) pose_point(P, c.ct[m], qcp[wl][m]);
      }
    }
    __syncwarp();
    double f = 0.0;
    const double invM = 1.0 / c.M;
    for (int64_t s = lane; s < a.ns; s += 32) {
      double ks = (double)c.n_const;
      for (int v = 0; v < c.Mv; ++v) {
        const int m = c.vidx[v];
        const double sp[3] = {a.cp64[(m * 3 + 0) * a.ns + s], a.cp64[(m * 3 + 1) * a.ns + s],
                              a.cp64[(m * 3 + 2) * a.ns + s]};
        ks += k_rq_f64(hg, sp, qcp[wl][m]);
      }
      f = fma(a.alpha[s] * invM, ks, f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) {
      if (a.f) a.f[k] = (float)f;
      a.label[k] = f >= 0.0 ? 1 : -1;
    }
    __syncwarp();
  }
}

cudaError_t launch_rescore_f64(const ChainD &c, const RescoreArgs &a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  rescore_f64_kernel<<<(unsigned)(sms > 0 ? 2 * sms : 304), kRescoreWarps * 32, 0, s>>>(c, a);
  return cudaGetLastError();
}

}  // namespace fk
