// Host-side launch wrappers shared between the fkfast translation units.
// Every wrapper enqueues work on `stream` and returns the cudaError_t of the
// launch; argument checking happens in the C-ABI layer (fkfast_api.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fk_device.cuh"

namespace fk {

// Forward kinematics: q [n][D] -> cp SoA [M][3][n] (all M control points).
cudaError_t launch_fk_forward_f32(const ChainF &c, const float *q, int64_t n, float *cp, cudaStream_t s);
cudaError_t launch_fk_forward_f64(const ChainD &c, const double *q, int64_t n, double *cp, cudaStream_t s);
// FP32 configurations widened to FP64 before FP64 kinematics.
cudaError_t launch_fk_forward_f32in_f64(const ChainD &c, const float *q, int64_t n, double *cp, cudaStream_t s);

// Kernel matrix from SoA control points (all M points).  sym != 0 requires
// cpa == cpb and na == nb and fills only the upper tiles, mirroring them.
// Summands of control points fixed to the base frame are exactly 1 and are
// added without evaluation.
cudaError_t launch_gram_f64(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb,
                            int64_t nb, int sym, double *K, cudaStream_t s);
// Double-float (FP32 pair) evaluation of the FP64 kernel matrix.  wa, wb:
// workspaces of Mv * 3 * na (nb) float2 for the split control points (wb
// unused when sym != 0).
cudaError_t launch_gram_df(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb, int64_t nb,
                           int sym, double *K, float2 *wa, float2 *wb, cudaStream_t s);
// The same, each entry rounded to FP32 once (the stored single-precision matrix).
cudaError_t launch_gram_df32(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb,
                             int64_t nb, int sym, float *K, float2 *wa, float2 *wb, cudaStream_t s);
cudaError_t launch_gram_f32(const ChainD &c, float gamma, const float *cpa, int64_t na, const float *cpb, int64_t nb,
                            int sym, float *K, cudaStream_t s);

// Fastron Algorithm 1 on a stored kernel matrix G [N][N], FP64 or FP32
// (g32 != 0), N <= 65,536.
struct TrainArgs {
  const void *G;
  int g32;
  const int8_t *y;
  int64_t N;
  double beta;
  int64_t iter_max, s_max;
  double *alpha;       // [N] in/out
  double *F;           // [N] in/out
  int64_t *stats;      // [6] out: iterations, adds, removes, converged, n_support, timeout (zeroed by the caller)
  int32_t *sup_idx;    // [N] out: ascending support indices
  double *sup_alpha;   // [N] out
  int8_t *trace_kind;  // [iter_max] or null
  int32_t *trace_idx;
  double *trace_delta;
  uint32_t wait_limit;  // polls per exchange wait of the cluster reduction
};
cudaError_t launch_fastron_train(const TrainArgs &a, cudaStream_t s);

// Two-stage active-learning samples and the margins of a carried-over model.
struct ActiveArgs {
  const double *S;  // [ns][D] support configurations
  int64_t ns;
  int D;
  int k_near;
  double sigma, qlim;
  int64_t n_uniform;
  uint64_t seed;
  double *X;        // [ns (1 + k_near) + n_uniform][D]
  float *X32;       // same, FP32, or null
};
cudaError_t launch_active_samples(const ActiveArgs &a, cudaStream_t s);
// F[j] = sum_{s < ns} alpha[s] G[s][j], G [N][N] FP64 or FP32 (g32 != 0).
cudaError_t launch_margins(const void *G, int g32, int64_t N, const double *alpha, int64_t ns, double *F,
                           cudaStream_t s);

// float4 entries of one support-pair record of the FP32 score: for each of
// the Mv configuration-dependent control points (x_a, x_b, y_a, y_b), then
// the z coordinates two points at a time (z_a, z_b, z_a', z_b'), then the
// circle form of point 0 (C_a, C_b, S_a, S_b) = 2 rho g (cos, sin) of half the
// joint-1 angle (ChainD::circ; zero otherwise), then the weights (w_a, w_b,
// |w_a|, |w_b|) with w = alpha / M; coordinates are scaled by
// g = sqrt(gamma / 2).
// Support pairs summed in plain FP32 by the score kernels before each
// partial sum is folded into a pair (two-sum) accumulator, and the smallest
// shared-memory tile (support pairs) of any score kernel; partial sums also
// restart at tile boundaries.  Both enter the error bound of the band.
constexpr int kFoldPairs = 16;
constexpr int kMinTilePairs = 32;

__host__ __device__ constexpr int rec_len(int mv) { return mv + (mv + 1) / 2 + 2; }
// Pair records of a support set of ns points: the points with alpha > 0 come
// first, then those with alpha < 0, each group padded to an even count with a
// zero-weight point, so every pair has one sign; one pair more than (ns + 1) / 2
// leaves room for both pads.
__host__ __device__ constexpr int64_t rec_pairs(int64_t ns) { return (ns + 1) / 2 + 1; }

// floats of one support point's double-float record (the band re-score): for
// each configuration-dependent control point (x_h, x_l, y_h, y_l, z_h, z_l) of
// sqrt(gamma/2) times its FP64 position, then (w_h, w_l, |w|, 0) with
// w = alpha / M as a pair, padded to a multiple of four.
__host__ __device__ constexpr int rec_df_len(int mv) { return (6 * mv + 4 + 3) / 4 * 4; }

// Packs a support set for scoring: gathers X[idx[s]] (FP64 configurations,
// idx may be null for identity), computes their FP64 control points and
// writes the FP32 score records and the FP64 SoA control points.
struct PackArgs {
  const double *X;
  const int32_t *idx;
  const double *alpha;
  int64_t ns;
  double gamma;
  float4 *rec;        // [rec_pairs(ns)][rec_len(Mv)], positive-weight pairs first
  double *cp64;       // SoA [M][3][ns]
  double *alpha_out;  // [ns] (copy of alpha, compacted)
  double *q_out;      // [ns][D] support configurations
  float *sdf;         // [ns][rec_df_len(Mv)] double-float records
  double scale;       // coordinate scale: sqrt(gamma/2) (RQ), sqrt(gamma/2 log2 e) (Gaussian)
  int32_t *slot;      // [ns] scratch: record half of each support point
  int32_t *npair_pos; // [2] out: [0] number of positive-weight pairs, [1] bits of the
                      // largest norm of a scaled support control point (float, rounded up)
};
cudaError_t launch_pack_support(const ChainF &cf, const ChainD &cd, const PackArgs &a, cudaStream_t s);

// FP32 score with per-query bound and band compaction.
struct ScoreArgs {
  const float *q;
  int64_t n;
  const float4 *rec;
  int64_t ns;          // record halves: 2 rec_pairs(support points)
  double gs;          // scale of the control points (PackArgs::scale)
  float eps0, eps1;   // band: |f| <= eps(q) B(q), eps(q) = eps0 + eps1 (|p(q)| + |s|max)
  float *f;           // [n] or null
  int8_t *label;      // [n]
  int32_t *band_idx;  // [n] or null (no rescore)
  int32_t *band_cnt;  // [1]
  int32_t *err;       // [1]
  uint32_t wait_limit;  // polls of a tile wait before it gives up
  int poly;           // Gaussian summand, 7 points: points per support point on the FMA polynomial
  const int32_t *npair_pos;  // device: [0] positive-weight pairs, which lead the records;
                             // [1] float bits of the largest scaled support-point norm
  float cnorm;        // > 0: point 0 in the circle form (FP32 RQ kernel), and the band
                      // takes max(|p(q)| + |s|max, cnorm) in place of |p(q)| + |s|max
};
cudaError_t launch_score_f32(const ChainF &c, const ScoreArgs &a, cudaStream_t s);

// FP64 re-evaluation of the compacted band queries.
struct RescoreArgs {
  const float *q;
  const int32_t *band_idx;
  const int32_t *band_cnt;
  int64_t n;
  const double *cp64;   // SoA [M][3][ns]
  const double *alpha;  // [ns]
  int64_t ns;
  double gamma;
  float *f;
  int8_t *label;
};
cudaError_t launch_rescore_f64(const ChainD &c, const RescoreArgs &a, cudaStream_t s);

// Double-float re-evaluation of the band (host-known size nb); queries whose
// |f| <= eps2 B(q) are appended to band2 for the FP64 re-score.
constexpr int kMaxDfChunks = 64;
struct DfRescoreArgs {
  const float *q;
  const int32_t *band_idx;  // [nb]
  int64_t nb;
  const float *sdf;         // [ns][rec_df_len(Mv)]
  int64_t ns;
  int n_const;              // control points fixed to the base (summand exactly 1)
  double gs;                // coordinate scale (PackArgs::scale)
  float2 *qdf;              // [Mv * 3][nb] scratch: band control points as pairs
  float4 *part;             // [chunks][nb] scratch: (f_h, f_l, B, 0) per chunk
  int chunks;
  int64_t chunk_len;
  double eps2;
  float *f;
  int8_t *label;
  int32_t *band2_idx;       // [nb]
  int32_t *band2_cnt;       // [1], zeroed by the caller
};
int rescore_df_chunks(int64_t nb, int64_t ns, int sms);
cudaError_t launch_rescore_df(const ChainD &c, const DfRescoreArgs &a, cudaStream_t s);

// Geometric labels: FP32 filter, FP64 for configurations too close to call.
constexpr int kMaxBoxes = 64;
struct Boxes {
  int nb;
  double r2;
  double b[kMaxBoxes][6];
};
cudaError_t launch_label(const ChainF &cf, const ChainD &c, const Boxes &bx, const float *q, int64_t n, int8_t *y,
                         cudaStream_t s);

// Throughput probe; fills per-block (smid, start, end) records.
cudaError_t launch_probe(int kind, int blocks, int threads, long long *rec, cudaStream_t s);

}  // namespace fk
