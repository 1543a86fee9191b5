// Arguments of the graph-replayed training step of the learned surrogate
// (surr_train.cu) and its launchers.
#pragma once

#include "tc_gemm.cuh"

namespace fk {

// Per-tile sums of the step, in this order: the bias gradients of layers 1-3
// (sums of the BF16 deltas over the tile's rows), the output weights'
// gradient (sum of bf16(h3) dout), the output bias's (sum of dout) and the
// tile's squared error.
constexpr int kTileStatB1 = 0, kTileStatB2 = kTileStatB1 + kSurrW, kTileStatB3 = kTileStatB2 + kSurrW,
              kTileStatW4 = kTileStatB3 + kSurrW, kTileStatB4 = kTileStatW4 + kSurrW,
              kTileStatLoss = kTileStatB4 + 1, kTileStats = kTileStatLoss + 1;

// The batch's activations and deltas, transposed for the weight-gradient
// products (K = batch row), are stored "chunk-blocked": 64 rows at a time, a
// tensor of U units occupies U x 128 bytes per chunk, element (u, row) at
//   (row / 64) U 128 + ((u / 8) 8 + (row mod 64) / 8) 128 + (u mod 8) 16 + (row mod 8) 2
// bytes: each chunk is the no-swizzle core-matrix layout of a [U][64]
// K-major operand tile, so one 1-D bulk copy loads it.
struct SurrStepArgs {
  const bf16 *X;                 // [rows][64] features of every training row
  const float *Y;                // [rows] targets
  int B;                         // batch rows (multiple of 128)
  int64_t steps_per_epoch;
  const int64_t *step;           // device: steps taken in this call
  const uint8_t *wc;             // the 17 weight blocks (surr_wc_off), 544 KB
  const float *b1, *b2, *b3, *w4, *b4;
  bf16 *xT;                      // chunk-blocked, U = 64
  bf16 *h1T, *h2T, *d3T, *d2T, *d1T;  // chunk-blocked, U = 256
  float *tstat;                  // [B / 128][kTileStats]
  int32_t *err;
  uint32_t wait_limit;
};

// The learning-rate schedule of a training call (cosine over the call's
// steps, or the step schedule: lr for the first two thirds of the epochs,
// lr / 3 after) and Adam's step count before it.
struct SurrSched {
  int64_t total;        // steps of the call
  int64_t steps_per_epoch;
  int64_t epochs;
  int64_t t0;           // Adam steps taken before the call
  float lr;
  int cosine;
};

// The three weight-gradient products dW3 = d3^T h2, dW2 = d2^T h1 and
// dW1 = d1^T x in one launch, each split along the batch into `splits`
// FP32 partials.  Partial z of a product with N columns holds entry (u, n)
// at part + z N 256 + u N + n (row-major).
// With sched not null, one otherwise idle thread of the launch also writes
// the step's learning rate and Adam's two bias corrections to sched[0..2].
struct SurrDwArgs {
  const bf16 *xT, *h1T, *h2T, *d1T, *d2T, *d3T;  // chunk-blocked
  int B;
  int splits;
  float *p1, *p2, *p3;           // partials of dW1, dW2, dW3
  const int64_t *step;
  SurrSched sch;
  float *sched;
  int32_t *err;
  uint32_t wait_limit;
};

// The step's reduction and update: the gradient G (flat parameter order W1,
// b1, W2, b2, W3, b3, w4, b4) as sums of the partials in split order and of
// the tile sums in tile order, the loss into loss_hist[step]; with `update`
// also Adam with the step's learning rate, the BF16 weight copies and the
// step counter.
struct SurrAdamArgs {
  float *p, *m, *v;
  float *G;
  const float *p1, *p2, *p3;    // SurrDwArgs partials
  int splits;
  const float *tstat;           // [ntiles][kTileStats]
  int ntiles;
  int B;
  float *loss_hist;             // [total steps] or null
  int64_t *step;
  uint32_t *done;               // block counter of the last-block step increment
  int update;
  const float *sched;   // the step's learning rate and bias corrections (SurrDwArgs)
  bf16 *w1, *w2, *w3;   // BF16 weights [out][in] (the inference kernel's)
  uint8_t *wc;          // and their blocks for the training step
};

cudaError_t launch_surr_tile(const SurrStepArgs &a, int sms, cudaStream_t s);
cudaError_t launch_surr_dw(const SurrDwArgs &a, cudaStream_t s);
cudaError_t launch_surr_adam(const SurrAdamArgs &a, cudaStream_t s);
// The weight blocks of the training step from BF16 weights [out][in].
cudaError_t launch_surr_wc(const bf16 *w1, const bf16 *w2, const bf16 *w3, uint8_t *wc, cudaStream_t s);
constexpr size_t kSurrWcBytes = (size_t)17 * kSurrW * kBK * 2;
// FP32 entries of one split's partials of all three products
constexpr int64_t kSurrDwPart = (int64_t)kSurrW * kSurrIn + 2 * (int64_t)kSurrW * kSurrW;

}  // namespace fk
