// Learned surrogate of the FK-kernel score (not part of the paper): features
// from the control points and joint angles, a 64-256-256-256-1 ReLU MLP whose
// layers run on tcgen05 tensor cores (BF16 operands, FP32 accumulation),
// mean-squared-error training with Adam on FP32 master weights, and inference
// that answers confident queries and sends the rest to the exact score.
#include "surr_features.cuh"
#include "tc_gemm.cuh"

namespace fk {

template <int NT>
static cudaError_t launch_gemm_t(const GemmArgs &g, int splits, cudaStream_t s) {
  constexpr size_t smem = gemm_smem_bytes<NT>();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(g.M / kBM), (unsigned)(g.N / NT), (unsigned)splits);
  gemm_tc_kernel<NT><<<grid, kGemmThreads, smem, s>>>(g);
  return cudaGetLastError();
}

// D = A B^T with FP32 output, split along K into `splits` partial products
// written at Cf + z * M * N.
cudaError_t launch_gemm_f32(const GemmArgs &g0, int splits, cudaStream_t s) {
  GemmArgs g = g0;
  if (g.N % 256 == 0) return launch_gemm_t<256>(g, splits, s);
  if (g.N % 128 == 0) return launch_gemm_t<128>(g, splits, s);
  return launch_gemm_t<64>(g, splits, s);
}

}  // namespace fk

namespace fk {

// ------------------------------------------------------------ features ---
// One row of features per query (surr_features.cuh), written row-major.
// Rows n..n_pad-1 are zeros.
__global__ void surr_features_kernel(const ChainF c, const float *__restrict__ q, int64_t n, int64_t n_pad,
                                     bf16 *__restrict__ X) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  __align__(16) bf16 h[kSurrIn];
  surr_feature_row(c, k < n ? q + k * c.D : nullptr, h);
  uint4 *dst = reinterpret_cast<uint4 *>(X + k * kSurrIn);
#pragma unroll
  for (int i = 0; i < kSurrIn / 8; ++i) dst[i] = reinterpret_cast<const uint4 *>(h)[i];
}

// ---------------------------------------------------------------- Adam ---
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of a weight matrix W [rows][cols] (FP32): row-major and transposed.
__global__ void weights_bf16_kernel(const float *__restrict__ W, int rows, int cols, bf16 *__restrict__ Wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  Wb[i] = __float2bfloat16_rn(W[i]);
}

// ----------------------------------------------------------- inference ---
// Confident queries (|pred| > tau) take sign(pred); the rest are appended to
// the fallback list for the exact score.
__global__ void surr_decide_kernel(const float *__restrict__ out, float scale, int64_t n, float tau,
                                   float *__restrict__ pred, int8_t *__restrict__ label, int32_t *__restrict__ fb_idx,
                                   int32_t *__restrict__ fb_cnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31;
  const bool valid = k < n;
  const float p = valid ? out[k] * scale : 0.f;
  const bool fb = valid && !(fabsf(p) > tau);
  if (valid) {
    if (pred) pred[k] = p;
    label[k] = p >= 0.f ? 1 : -1;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, fb);
  if (bal) {
    int base = 0;
    if (lane == 0) base = atomicAdd(fb_cnt, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (fb) fb_idx[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)k;
  }
}

__global__ void gather_rows_kernel(const float *__restrict__ q, int D, const int32_t *__restrict__ idx, int64_t n,
                                   float *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * D) return;
  const int64_t r = i / D, c = i % D;
  out[i] = q[(int64_t)idx[r] * D + c];
}

__global__ void scatter_labels_kernel(const int8_t *__restrict__ src, const float *__restrict__ fsrc,
                                      const int32_t *__restrict__ idx, int64_t n, int8_t *__restrict__ label,
                                      float *__restrict__ pred) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  label[idx[i]] = src[i];
  if (pred) pred[idx[i]] = fsrc[i];
}

// sum of squares of x[0..n) into *acc (one atomic per block; used once per
// training call to scale the targets)
__global__ void sumsq_kernel(const float *__restrict__ x, int64_t n, double *__restrict__ acc) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i] * (double)x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
    atomicAdd(acc, t);
  }
}

__global__ void scale_kernel(float *__restrict__ x, int64_t n, float s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s;
}

// ------------------------------------------------------------ launchers ---
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_surr_features(const ChainF &c, const float *q, int64_t n, int64_t n_pad, bf16 *X, cudaStream_t s) {
  surr_features_kernel<<<blocks_for(n_pad, 128), 128, 0, s>>>(c, q, n, n_pad, X);
  return cudaGetLastError();
}

// D = A B^T with FP32 partial products, N tile 64, 128 or 256.
cudaError_t launch_gemm(int nt, const GemmArgs &g, int splits, cudaStream_t s) {
  switch (nt) {
    case 64: return launch_gemm_t<64>(g, splits, s);
    case 128: return launch_gemm_t<128>(g, splits, s);
    case 256: return launch_gemm_t<256>(g, splits, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adam(float *p, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                        float eps, int64_t t, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_weights_bf16(const float *W, int rows, int cols, bf16 *Wb, cudaStream_t s) {
  weights_bf16_kernel<<<blocks_for((int64_t)rows * cols, 256), 256, 0, s>>>(W, rows, cols, Wb);
  return cudaGetLastError();
}

cudaError_t launch_surr_decide(const float *out, float scale, int64_t n, float tau, float *pred, int8_t *label,
                               int32_t *fb_idx, int32_t *fb_cnt, cudaStream_t s) {
  surr_decide_kernel<<<blocks_for(n, 256), 256, 0, s>>>(out, scale, n, tau, pred, label, fb_idx, fb_cnt);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float *q, int D, const int32_t *idx, int64_t n, float *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_rows_kernel<<<blocks_for(n * D, 256), 256, 0, s>>>(q, D, idx, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scatter_labels(const int8_t *src, const float *fsrc, const int32_t *idx, int64_t n, int8_t *label,
                                  float *pred, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  scatter_labels_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, fsrc, idx, n, label, pred);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const float *x, int64_t n, double *acc, cudaStream_t s) {
  sumsq_kernel<<<152 * 4, 256, 0, s>>>(x, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_scale(float *x, int64_t n, float v, cudaStream_t s) {
  scale_kernel<<<blocks_for(n, 256), 256, 0, s>>>(x, n, v);
  return cudaGetLastError();
}

}  // namespace fk

namespace fk {

// tau for zero sign errors on a held-out set: the largest |pred| among the
// rows whose sign differs from the exact score's; also counts them.
__global__ void surr_calibrate_kernel(const float *__restrict__ pred, const float *__restrict__ f, int64_t n,
                                      unsigned *__restrict__ tau_bits, unsigned long long *__restrict__ wrong) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool w = (pred[i] >= 0.f) != (f[i] >= 0.f);
  if (w) {
    atomicMax(tau_bits, __float_as_uint(fabsf(pred[i])));
    atomicAdd(wrong, 1ull);
  }
}

__global__ void count_below_kernel(const float *__restrict__ pred, int64_t n, float tau,
                                   unsigned long long *__restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !(fabsf(pred[i]) > tau)) atomicAdd(cnt, 1ull);
}

cudaError_t launch_surr_calibrate(const float *pred, const float *f, int64_t n, unsigned *tau_bits,
                                  unsigned long long *wrong, unsigned long long *below_cnt, float tau_hint,
                                  cudaStream_t s) {
  surr_calibrate_kernel<<<blocks_for(n, 256), 256, 0, s>>>(pred, f, n, tau_bits, wrong);
  (void)tau_hint;
  (void)below_cnt;
  return cudaGetLastError();
}

cudaError_t launch_count_below(const float *pred, int64_t n, float tau, unsigned long long *cnt, cudaStream_t s) {
  count_below_kernel<<<blocks_for(n, 256), 256, 0, s>>>(pred, n, tau, cnt);
  return cudaGetLastError();
}

}  // namespace fk
