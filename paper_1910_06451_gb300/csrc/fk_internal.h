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
// Double-float (FP32 pair) evaluation of the FP64 kernel matrix.
cudaError_t launch_gram_df(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb, int64_t nb,
                           int sym, double *K, cudaStream_t s);
cudaError_t launch_gram_f32(const ChainD &c, float gamma, const float *cpa, int64_t na, const float *cpb, int64_t nb,
                            int sym, float *K, cudaStream_t s);

// Fastron Algorithm 1 on a stored FP64 kernel matrix G [N][N].
struct TrainArgs {
  const double *G;
  const int8_t *y;
  int64_t N;
  double beta;
  int64_t iter_max, s_max;
  double *alpha;       // [N] in/out
  double *F;           // [N] in/out
  int64_t *stats;      // [5] out: iterations, adds, removes, converged, n_support
  int32_t *sup_idx;    // [N] out: ascending support indices
  double *sup_alpha;   // [N] out
  int8_t *trace_kind;  // [iter_max] or null
  int32_t *trace_idx;
  double *trace_delta;
};
cudaError_t launch_fastron_train(const TrainArgs &a, cudaStream_t s);

// float4 entries of one support-pair record of the FP32 score: for each of
// the Mv configuration-dependent control points (x_a, x_b, y_a, y_b), then
// the z coordinates two points at a time (z_a, z_b, z_a', z_b'), then the
// weights (w_a, w_b, |w_a|, |w_b|) with w = alpha / M; coordinates are scaled
// by sqrt(gamma / 2).
__host__ __device__ constexpr int rec_len(int mv) { return mv + (mv + 1) / 2 + 1; }

// Packs a support set for scoring: gathers X[idx[s]] (FP64 configurations,
// idx may be null for identity), computes their FP64 control points and
// writes the FP32 score records and the FP64 SoA control points.
struct PackArgs {
  const double *X;
  const int32_t *idx;
  const double *alpha;
  int64_t ns;
  double gamma;
  float4 *rec;        // [(ns + 1) / 2][rec_len(Mv)]
  double *cp64;       // SoA [M][3][ns]
  double *alpha_out;  // [ns] (copy of alpha, compacted)
  double *q_out;      // [ns][D] support configurations
};
cudaError_t launch_pack_support(const ChainF &cf, const ChainD &cd, const PackArgs &a, cudaStream_t s);

// FP32 score with per-query bound and band compaction.
struct ScoreArgs {
  const float *q;
  int64_t n;
  const float4 *rec;
  int64_t ns;
  float gs;           // sqrt(gamma / 2): scale of the control points
  float eps;          // band: |f| <= eps * B(q)
  float *f;           // [n] or null
  int8_t *label;      // [n]
  int32_t *band_idx;  // [n] or null (no rescore)
  int32_t *band_cnt;  // [1]
  int32_t *err;       // [1]
  uint32_t wait_limit;  // polls of a tile wait before it gives up
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
