// Proxy collision check: the Fastron model value f(q) = sum_s alpha_s
// K_FK(S_s, q) with the FK kernel of Eq. 4 and its sign (Sec. III-B).
//
// Kernels:
//   pack     support set -> pair records (see fk_internal.h: scaled FP32
//            coordinates of two support points, their weights w = alpha/M),
//            the positive-weight pairs first; double-float records and FP64
//            control points for the re-score; the largest norm of a scaled
//            support control point.  All from FP64 kinematics, rounded once.
//   score    FP32.  One thread scores two queries: FK in pair arithmetic,
//            rounded to FP32, in registers; the support records stream
//            through shared memory by tile (1-D TMA bulk copies,
//            double-buffered, mbarrier completion) and every thread reads each
//            record as a broadcast.  Per (s, m): t = 1 + |p_m - s_m|^2 in
//            scaled coordinates (three differences, three FMAs), and two
//            summands share one reciprocal: 1/t1^2 + 1/t2^2 = (t1^2 + t2^2) /
//            (t1 t2)^2.  Beside f the kernel forms B(q) = sum_s |w_s| sum_m
//            t^-2 and appends the queries with |f| <= eps(q) B(q) to a band
//            list; eps(q) bounds the kernel's whole error (the derivation is
//            at the host's score_band).
//   gauss    the non-paper Gaussian summand 2^(-|d|^2) (coordinates scaled
//            by sqrt(gamma/2 log2 e)) on MUFU ex2, optionally partly on an
//            FMA polynomial, or in packed half with ex2.f16x2.
//   rescore  FP64, one warp per band query: FK and Eq. 3/4 in FP64 with the
//            operation order of the plain definition, lanes splitting the
//            support set, a fixed-order warp sum; f and the label are replaced.
#include "df_arith.cuh"
#include "fk_internal.h"
#include "fk_ptx.cuh"
#include "score_core.cuh"

namespace fk {

// ---------------------------------------------------------------- pack ---
// Record slot of every support point: the points with alpha > 0 in ascending
// order from slot 0, those with alpha < 0 in ascending order from the first
// even slot after them (the odd slot between stays a zero-weight pad).  One
// CTA ranks the points chunk by chunk with warp ballots; it also writes the
// number of positive-weight pairs.
constexpr int kSlotThreads = 1024;

__global__ void __launch_bounds__(kSlotThreads) sign_slots_kernel(const double *__restrict__ alpha, int64_t ns,
                                                                  int32_t *__restrict__ slot,
                                                                  int32_t *__restrict__ npair_pos) {
  __shared__ int wsum[2][kSlotThreads / 32];
  __shared__ int total;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int cnt = 0;
  for (int64_t s = tid; s < ns; s += kSlotThreads) cnt += alpha[s] > 0.0;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) wsum[0][wid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int w = 0; w < kSlotThreads / 32; ++w) t += wsum[0][w];
    total = t;
  }
  __syncthreads();
  const int npos = total;
  const int neg0 = 2 * ((npos + 1) / 2);
  int run_pos = 0, run_neg = 0;  // points of each sign in earlier chunks
  for (int64_t c0 = 0; c0 < ns; c0 += kSlotThreads) {
    __syncthreads();  // wsum of the previous chunk has been read
    const int64_t s = c0 + tid;
    const bool in = s < ns;
    const bool pos = in && alpha[s] > 0.0, neg = in && !pos;
    const unsigned bp = __ballot_sync(0xffffffffu, pos), bn = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) {
      wsum[0][wid] = __popc(bp);
      wsum[1][wid] = __popc(bn);
    }
    __syncthreads();
    int before_p = 0, before_n = 0, chunk_p = 0, chunk_n = 0;
    for (int w = 0; w < kSlotThreads / 32; ++w) {
      if (w < wid) {
        before_p += wsum[0][w];
        before_n += wsum[1][w];
      }
      chunk_p += wsum[0][w];
      chunk_n += wsum[1][w];
    }
    const unsigned lt = (1u << lane) - 1u;
    if (pos) slot[s] = run_pos + before_p + __popc(bp & lt);
    if (neg) slot[s] = neg0 + run_neg + before_n + __popc(bn & lt);
    run_pos += chunk_p;
    run_neg += chunk_n;
  }
  if (tid == 0) *npair_pos = (npos + 1) / 2;
}

// One thread per support point s, writing its half h = slot & 1 of the pair
// record slot >> 1 (components h and 2 + h of each float4); the records are
// zero-filled first, so pads carry weight 0.  The FP64 kinematics run at 1/64
// of the FP32 rate, so the CTAs are small (32 threads) and spread over as many
// SMs as there are support points / 32.
constexpr int kPackThreads = 32;

__global__ void __launch_bounds__(kPackThreads) pack_kernel(const ChainF cf, const ChainD cd, const PackArgs a) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= a.ns) return;
  const int MV = cf.Mv;
  const int REC = rec_len(MV);
  const int64_t j = a.slot[s] >> 1;
  const int h = a.slot[s] & 1;
  float *rec = reinterpret_cast<float *>(a.rec + j * REC);
  auto put = [&](int e, int c, float v) { rec[4 * e + c] = v; };  // component c (0..3) of record entry e
  const double gs = a.scale;
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
  const double wd = al / cd.M;
  // FP32 record: (x_a, x_b, y_a, y_b) per point, z two points at a time, weights
  for (int v = 0; v < MV; ++v) {
    const int m = cf.vidx[v];
    put(v, h, (float)(gs * cp[m][0]));
    put(v, 2 + h, (float)(gs * cp[m][1]));
    put(MV + v / 2, 2 * (v & 1) + h, (float)(gs * cp[m][2]));
  }
  if (MV & 1) put(MV + MV / 2, 2 + h, 0.f);  // unused z slot of the last entry
  if (cd.circ) {
    // point 0 on its circle: with C = 2 rho g cos(theta_s / 2), S = 2 rho g
    // sin(theta_s / 2), the kernel's sin(theta / 2) C - cos(theta / 2) S is
    // 2 rho g sin((theta - theta_s) / 2), the scaled distance |p - s| up to sign
    double sh, ch;
    sincos(0.5 * (cd.th0[0] + x[0]), &sh, &ch);
    const double r2 = 2.0 * cd.circ_rho * gs;
    put(REC - 2, h, (float)(r2 * ch));
    put(REC - 2, 2 + h, (float)(r2 * sh));
  }
  put(REC - 1, h, (float)wd);
  put(REC - 1, 2 + h, (float)fabs(wd));
  // largest norm of a scaled configuration-dependent control point, rounded
  // up to FP32 (non-negative floats order like their bit patterns)
  double nmax = 0.0;
  for (int v = 0; v < MV; ++v) {
    const double *p = cp[cf.vidx[v]];
    nmax = fmax(nmax, gs * sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]));
  }
  atomicMax(a.npair_pos + 1, __float_as_int(__double2float_ru(nmax * (1.0 + 1e-12))));
  if (a.sdf) {
    float *r = a.sdf + s * rec_df_len(MV);
    for (int v = 0; v < MV; ++v)
      for (int c3 = 0; c3 < 3; ++c3) {
        const dfl xv = df_from_double(gs * cp[cf.vidx[v]][c3]);
        r[v * 6 + 2 * c3] = xv.h;
        r[v * 6 + 2 * c3 + 1] = xv.l;
      }
    const dfl wp = df_from_double(wd);
    r[6 * MV] = wp.h;
    r[6 * MV + 1] = wp.l;
    r[6 * MV + 2] = (float)fabs(wd);
    for (int i = 6 * MV + 3; i < rec_df_len(MV); ++i) r[i] = 0.f;
  }
}

cudaError_t launch_pack_support(const ChainF &cf, const ChainD &cd, const PackArgs &a, cudaStream_t s) {
  const size_t rec_bytes = sizeof(float4) * (size_t)rec_pairs(a.ns) * rec_len(cf.Mv);
  cudaError_t e = cudaMemsetAsync(a.rec, 0, rec_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.npair_pos + 1, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  sign_slots_kernel<<<1, kSlotThreads, 0, s>>>(a.alpha, a.ns, a.slot, a.npair_pos);
  if (a.ns > 0) pack_kernel<<<(unsigned)((a.ns + kPackThreads - 1) / kPackThreads), kPackThreads, 0, s>>>(cf, cd, a);
  return cudaGetLastError();
}

// --------------------------------------------------------------- score ---
constexpr int kScoreThreads = 256;
// queries per thread: two share every shared-memory read of a support pair;
// above 8 points their packed coordinates (2 x 3 x Mv 64-bit registers)
// would not fit in the 128 registers of two CTAs per SM, so one
template <int MV>
__host__ __device__ constexpr int queries_per_thread() {
  return MV > 8 ? 1 : 2;
}
template <int MV>
__host__ __device__ constexpr int queries_per_cta() {
  return kScoreThreads * queries_per_thread<MV>();
}
// The FP32 score kernel's own shape: from 7 points up one query per thread,
// with more resident CTAs to hide the MUFU and FMA latencies (4 per SM at 7
// and 8 points, 3 above); below, two queries per thread at 2 CTAs (4 would
// spill).  Measured on 4M queries: 7 points 5.77 -> 5.48 ms (two queries per
// thread at 2 CTAs against one at 4), 11 points 119.3 -> 118.1 ms (3 CTAs).
template <int MV>
__host__ __device__ constexpr int f32_queries_per_thread() {
  return MV > 6 ? 1 : 2;
}
template <int MV>
__host__ __device__ constexpr int f32_ctas_per_sm() {
  return MV > 8 ? 3 : (MV > 6 ? 4 : 2);
}
template <int MV>
__host__ __device__ constexpr int f32_queries_per_cta() {
  return kScoreThreads * f32_queries_per_thread<MV>();
}
constexpr int kTilePairs = 64;                 // support pairs per shared-memory tile

__device__ __forceinline__ dd pair_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

// CIRC: point 0 in the circle form (ScoreArgs::cnorm > 0).
template <int MV, bool CIRC>
__global__ void __launch_bounds__(kScoreThreads, f32_ctas_per_sm<MV>()) score_f32_kernel(const ChainF c,
                                                                                          const ScoreArgs a) {
  extern __shared__ __align__(128) float4 tiles[];  // [2][kTilePairs][rec_len(MV)]
  __shared__ __align__(8) uint64_t bar[2];
  const BlockOut o{a.f, a.label, a.eps0, a.eps1, a.band_idx, nullptr, 0, 0, a.band_cnt, a.err, a.wait_limit,
                   a.npair_pos, a.cnorm};
  score_block<MV, f32_queries_per_thread<MV>(), kTilePairs, kScoreThreads, false, false, 0, CIRC>(
      c, a.rec, a.ns, pair_of(a.gs), a.q, a.n, (int64_t)blockIdx.x * f32_queries_per_cta<MV>(), o, tiles, bar);
}

// The non-paper Gaussian summand (FP32 with POLY points per support point on
// the FMA polynomial, or packed half), otherwise the same block.
template <int MV, bool HALF, int POLY>
__global__ void __launch_bounds__(kScoreThreads, 2) score_gauss_kernel(const ChainF c, const ScoreArgs a) {
  extern __shared__ __align__(128) float4 tiles[];
  __shared__ __align__(8) uint64_t bar[2];
  const BlockOut o{a.f, a.label, a.eps0, a.eps1, a.band_idx, nullptr, 0, 0, a.band_cnt, a.err, a.wait_limit,
                   a.npair_pos};
  score_block<MV, queries_per_thread<MV>(), kTilePairs, kScoreThreads, HALF, true, POLY>(
      c, a.rec, a.ns, pair_of(a.gs), a.q, a.n, (int64_t)blockIdx.x * queries_per_cta<MV>(), o, tiles, bar);
}

// The packed-half variant of the same block (differences and t in FP16).
template <int MV>
__global__ void __launch_bounds__(kScoreThreads, 2) score_f16_kernel(const ChainF c, const ScoreArgs a) {
  extern __shared__ __align__(128) float4 tiles[];
  __shared__ __align__(8) uint64_t bar[2];
  const BlockOut o{a.f, a.label, a.eps0, a.eps1, a.band_idx, nullptr, 0, 0, a.band_cnt, a.err, a.wait_limit,
                   a.npair_pos};
  score_block<MV, queries_per_thread<MV>(), kTilePairs, kScoreThreads, true>(
      c, a.rec, a.ns, pair_of(a.gs), a.q, a.n, (int64_t)blockIdx.x * queries_per_cta<MV>(), o, tiles, bar);
}

}  // namespace fk

namespace fk {

template <int MV>
static cudaError_t launch_score_h_mv(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  constexpr int REC = rec_len(MV);
  const size_t smem = 2 * (size_t)kTilePairs * REC * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(score_f16_kernel<MV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.n + queries_per_cta<MV>() - 1) / queries_per_cta<MV>());
  score_f16_kernel<MV><<<grid, kScoreThreads, smem, s>>>(c, a);
  return cudaGetLastError();
}

template <int MV, bool HALF, int POLY>
static cudaError_t launch_gauss_mv(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  constexpr int REC = rec_len(MV);
  const size_t smem = 2 * (size_t)kTilePairs * REC * sizeof(float4);
  auto kern = score_gauss_kernel<MV, HALF, POLY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.n + queries_per_cta<MV>() - 1) / queries_per_cta<MV>());
  kern<<<grid, kScoreThreads, smem, s>>>(c, a);
  return cudaGetLastError();
}

// Shapes with compiled Gaussian-summand kernels (the 3-, 7- and 12-point
// arms); the FMA-polynomial split is compiled for 7 points.
bool score_gauss_supported(int mv) { return mv == 3 || mv == 7 || mv == 11; }

static cudaError_t launch_score_gauss(const ChainF &c, const ScoreArgs &a, bool half, cudaStream_t s) {
  if (half) {
    switch (c.Mv) {
      case 3: return launch_gauss_mv<3, true, 0>(c, a, s);
      case 7: return launch_gauss_mv<7, true, 0>(c, a, s);
      case 11: return launch_gauss_mv<11, true, 0>(c, a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (c.Mv) {
    case 3: return launch_gauss_mv<3, false, 0>(c, a, s);
    case 7:
      switch (a.poly) {
        case 1: return launch_gauss_mv<7, false, 1>(c, a, s);
        case 2: return launch_gauss_mv<7, false, 2>(c, a, s);
        default: return launch_gauss_mv<7, false, 0>(c, a, s);
      }
    case 11: return launch_gauss_mv<11, false, 0>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

bool score_f16_supported(int mv) { return mv == 3 || mv == 7 || mv == 11; }

cudaError_t launch_score_f16(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (c.summand == FK_SUMMAND_GAUSS) return launch_score_gauss(c, a, true, s);
  switch (c.Mv) {
    case 3: return launch_score_h_mv<3>(c, a, s);
    case 7: return launch_score_h_mv<7>(c, a, s);
    case 11: return launch_score_h_mv<11>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MV>
static cudaError_t launch_score_mv(const ChainF &c, const ScoreArgs &a, cudaStream_t s) {
  constexpr int REC = rec_len(MV);
  const size_t smem = 2 * (size_t)kTilePairs * REC * sizeof(float4);
  auto kern = a.cnorm > 0.f ? score_f32_kernel<MV, true> : score_f32_kernel<MV, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.n + f32_queries_per_cta<MV>() - 1) / f32_queries_per_cta<MV>());
  kern<<<grid, kScoreThreads, smem, s>>>(c, a);
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
  if (c.summand == FK_SUMMAND_GAUSS) return launch_score_gauss(c, a, false, s);
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
        ks += k_sum_f64(c.summand, hg, sp, qcp[wl][m]);
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
