// Double-float re-score of the FP32 band (Sec. III-B's model value f(q),
// evaluated again for the queries whose FP32 sign is not certain).
//
// The FP32 pass hands over every query with |f32| <= eps B(q).  Those are
// evaluated here with about 46 significant bits on the FP32 pipes:
//   band_fk     FP64 kinematics of each band query (Eqs. 1-2), control points
//               scaled by sqrt(gamma/2) (Gaussian summand: sqrt(gamma/2 log2 e))
//               in FP64 and split into FP32 pairs;
//   df          per (query, support point, control point) the summand
//               t^-2, t = 1 + |p - s|^2 in scaled coordinates, from pair
//               arithmetic (df_rq_term), summed per support point, weighted by
//               alpha_s / M and summed over a chunk of the support set;
//               the support set is cut into chunks when the band is small,
//               so that every SM has work;
//   finish      the chunk partials of each query are added in chunk order;
//               |f| > eps2 B(q) decides the label (the double-float error is
//               far below eps2 B(q)); the rest go to the FP64 re-score.
//
// Summand arithmetic: df_rq_term, or df_gauss_term for the non-paper
// Gaussian summand (df_arith.cuh).
// Error budget per query: coordinates 2^-48 relative (the pair split),
// summands ~1e-13 relative (the neglected square of the Newton residual is
// 2^-44), the unnormalised low words of the sums n 2^-48 of B(q) for n
// support points: below 1e-10 B(q) for n <= 20,000, against eps2 = 1e-9.
#include "df_arith.cuh"
#include "fk_internal.h"

namespace fk {

constexpr int kDfThreads = 128;
constexpr int kDfTile = 32;  // support points per shared-memory tile

// --------------------------------------------------------- band FK ---
__global__ void __launch_bounds__(32) band_fk_kernel(const ChainD c, const float *__restrict__ q,
                                                     const int32_t *__restrict__ band_idx, int64_t nb, double gs,
                                                     float2 *__restrict__ qdf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nb) return;
  const int64_t k = band_idx[e];
  double cp[FK_MAX_CP][3];
  PoseD P;
  pose_base(c, P);
  for (int m = 0; m < c.M; ++m)
    if (c.cj[m] == 0) pose_point(P, c.ct[m], cp[m]);
  for (int i = 0; i < c.D; ++i) {
    pose_step(c, i, (double)q[k * c.D + i], P);
    for (int m = 0; m < c.M; ++m)
      if (c.cj[m] == i + 1) pose_point(P, c.ct[m], cp[m]);
  }
  for (int v = 0; v < c.Mv; ++v)
    for (int r = 0; r < 3; ++r) {
      const dfl x = df_from_double(gs * cp[c.vidx[v]][r]);
      qdf[(v * 3 + r) * nb + e] = make_float2(x.h, x.l);
    }
}

// ------------------------------------------------------ df summands ---
template <int MV, bool GAUSS>
__global__ void __launch_bounds__(kDfThreads) rescore_df_kernel(const DfRescoreArgs a) {
  constexpr int RL = rec_df_len(MV);
  __shared__ __align__(16) float tile[kDfTile * RL];
  const int64_t e = blockIdx.x * (int64_t)kDfThreads + threadIdx.x;
  const bool live = e < a.nb;
  float qh[MV][3], ql[MV][3];
#pragma unroll
  for (int v = 0; v < MV; ++v)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 x = live ? a.qdf[(v * 3 + r) * a.nb + e] : make_float2(0.f, 0.f);
      qh[v][r] = x.x;
      ql[v][r] = x.y;
    }
  const int64_t s0 = (int64_t)blockIdx.y * a.chunk_len;
  const int64_t s1 = s0 + a.chunk_len < a.ns ? s0 + a.chunk_len : a.ns;
  const float n_const = (float)a.n_const;
  float fh = 0.f, fl = 0.f, B = 0.f;
  for (int64_t t0 = s0; t0 < s1; t0 += kDfTile) {
    const int cnt = (int)(s1 - t0 < kDfTile ? s1 - t0 : kDfTile);
    __syncthreads();  // the previous tile is consumed
    const float4 *src = reinterpret_cast<const float4 *>(a.sdf + t0 * RL);
    float4 *dst = reinterpret_cast<float4 *>(tile);
    for (int i = threadIdx.x; i < cnt * RL / 4; i += kDfThreads) dst[i] = src[i];
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float *S = tile + j * RL;
      float kh = n_const, kl = 0.f;
#pragma unroll
      for (int v = 0; v < MV; ++v) {
        float rh, rl;
        if (GAUSS)
          df_gauss_term(qh[v], ql[v], S + v * 6, rh, rl);
        else
          df_rq_term(qh[v], ql[v], S + v * 6, rh, rl);
        const dfl ks = two_sum(kh, rh);
        kh = ks.h;
        kl += ks.l + rl;
      }
      // f += w_s * ks, with w_s = alpha_s / M as a pair
      const float wh = S[6 * MV], wl = S[6 * MV + 1];
      const float ph = wh * kh;
      const float pe = fmaf(wh, kl, fmaf(wl, kh, fmaf(wh, kh, -ph)));
      const dfl fs = two_sum(fh, ph);
      fh = fs.h;
      fl += fs.l + pe;
      B = fmaf(S[6 * MV + 2], kh, B);
    }
  }
  if (live) a.part[(int64_t)blockIdx.y * a.nb + e] = make_float4(fh, fl, B, 0.f);
}

// ----------------------------------------------------------- finish ---
__global__ void __launch_bounds__(256) rescore_df_finish_kernel(const DfRescoreArgs a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.nb) return;
  float fh = 0.f, fl = 0.f, B = 0.f;
  for (int c = 0; c < a.chunks; ++c) {
    const float4 p = a.part[(int64_t)c * a.nb + e];
    const dfl s = two_sum(fh, p.x);
    fh = s.h;
    fl += s.l + p.y;
    B += p.z;
  }
  const double f = (double)fh + (double)fl;
  const int64_t k = a.band_idx[e];
  if (fabs(f) > a.eps2 * (double)B) {
    if (a.f) a.f[k] = (float)f;
    a.label[k] = f >= 0.0 ? 1 : -1;
  } else {
    a.band2_idx[atomicAdd(a.band2_cnt, 1)] = (int32_t)k;
  }
}

template <int MV>
static cudaError_t launch_df_mv(const DfRescoreArgs &a, bool gauss, unsigned qblocks, cudaStream_t s) {
  if (gauss)
    rescore_df_kernel<MV, true><<<dim3(qblocks, (unsigned)a.chunks), kDfThreads, 0, s>>>(a);
  else
    rescore_df_kernel<MV, false><<<dim3(qblocks, (unsigned)a.chunks), kDfThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int rescore_df_chunks(int64_t nb, int64_t ns, int sms) {
  const int64_t qblocks = (nb + kDfThreads - 1) / kDfThreads;
  if (qblocks <= 0 || ns <= 0) return 1;
  int64_t ch = (4 * (int64_t)sms + qblocks - 1) / qblocks;  // about four CTAs per SM
  const int64_t most = (ns + 15) / 16;                        // at least 16 support points each
  if (ch > most) ch = most;
  if (ch > kMaxDfChunks) ch = kMaxDfChunks;
  return (int)(ch < 1 ? 1 : ch);
}

cudaError_t launch_rescore_df(const ChainD &c, const DfRescoreArgs &a, cudaStream_t s) {
  if (a.nb <= 0) return cudaSuccess;
  // one warp per CTA: the FP64 kinematics spread over as many SMs as possible
  band_fk_kernel<<<(unsigned)((a.nb + 31) / 32), 32, 0, s>>>(c, a.q, a.band_idx, a.nb, a.gs, a.qdf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned qblocks = (unsigned)((a.nb + kDfThreads - 1) / kDfThreads);
  const bool gauss = c.summand == FK_SUMMAND_GAUSS;
  if (gauss) {
    switch (c.Mv) {  // the shapes with Gaussian score kernels
      case 3: e = launch_df_mv<3>(a, true, qblocks, s); break;
      case 7: e = launch_df_mv<7>(a, true, qblocks, s); break;
      case 11: e = launch_df_mv<11>(a, true, qblocks, s); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (c.Mv) {
      case 1: e = launch_df_mv<1>(a, false, qblocks, s); break;
      case 2: e = launch_df_mv<2>(a, false, qblocks, s); break;
      case 3: e = launch_df_mv<3>(a, false, qblocks, s); break;
      case 4: e = launch_df_mv<4>(a, false, qblocks, s); break;
      case 5: e = launch_df_mv<5>(a, false, qblocks, s); break;
      case 6: e = launch_df_mv<6>(a, false, qblocks, s); break;
      case 7: e = launch_df_mv<7>(a, false, qblocks, s); break;
      case 8: e = launch_df_mv<8>(a, false, qblocks, s); break;
      case 11: e = launch_df_mv<11>(a, false, qblocks, s); break;
      case 12: e = launch_df_mv<12>(a, false, qblocks, s); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  rescore_df_finish_kernel<<<(unsigned)((a.nb + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fk
