// Arguments of the graph-replayed training step of the learned surrogate
// (surr_train.cu) and its launchers.
#pragma once

#include "tc_gemm.cuh"

namespace fk {

struct SurrStepArgs {
  const bf16 *X;                 // [rows][64] features of every training row
  const float *Y;                // [rows] targets
  int B;                         // batch rows (multiple of 128)
  int64_t steps_per_epoch;
  const int64_t *step;           // device: steps taken in this call
  const uint8_t *wc;             // the 17 weight blocks (surr_wc_off), 544 KB
  const float *b1, *b2, *b3, *w4, *b4;
  bf16 *xT;                      // [64][B]
  bf16 *h1T, *h2T, *h3T, *d3T, *d2T, *d1T;  // [256][B]
  float *dout, *lrow;            // [B]: loss gradient of each output, squared error
  int32_t *err;
  uint32_t wait_limit;
};

// The step's reduction: weight gradients from split-K partials, bias and
// output-unit gradients as sums over the batch, the loss.
struct SurrReduceArgs {
  const float *p1, *p2, *p3;      // partials: [splits][256][64], [splits][256][256] x 2
  int splits;
  const bf16 *d1T, *d2T, *d3T, *h3T;
  const float *dout, *lrow;
  int B;
  float *G;
  float *loss_hist;               // [total steps] or null
  const int64_t *step;
};
// Adam with the step's learning rate (cosine or step schedule over the
// call's steps) and the BF16 weight copies.
struct SurrAdamArgs {
  float *p, *m, *v;
  const float *G;
  const int64_t *step;
  int64_t total;        // steps of the call (cosine schedule)
  int64_t steps_per_epoch;
  int64_t epochs;
  int64_t t0;           // Adam steps taken before the call
  float lr;
  int cosine;
  bf16 *w1, *w2, *w3;   // BF16 weights [out][in] (the inference kernel's)
  uint8_t *wc;          // and their blocks for the training step
};

cudaError_t launch_surr_tile(const SurrStepArgs &a, int sms, cudaStream_t s);
cudaError_t launch_surr_reduce(const SurrReduceArgs &a, cudaStream_t s);
cudaError_t launch_surr_adam(const SurrAdamArgs &a, cudaStream_t s);
cudaError_t launch_surr_advance(int64_t *step, cudaStream_t s);
// The weight blocks of the training step from BF16 weights [out][in].
cudaError_t launch_surr_wc(const bf16 *w1, const bf16 *w2, const bf16 *w3, uint8_t *wc, cudaStream_t s);
constexpr size_t kSurrWcBytes = (size_t)17 * kSurrW * kBK * 2;

}  // namespace fk
