// The model update loop of Sec. III-B after Algorithm 1: two-stage active
// learning builds the next training set from the current support set, and
// the next update starts from the carried-over weights (loadPreviousModel).
//
//   active_samples  rows [0, ns): the support configurations; then k_near
//                   copies of the support set, each joint moved by a draw
//                   uniform in [-sigma, sigma] and clipped to the joint
//                   limits (stage 1, small changes of the C-space
//                   obstacles); then n_uniform configurations uniform in the
//                   limits (stage 2, new obstacles).  Draws come from
//                   SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
//                   counter-based generator: draw k of stream `seed` is the
//                   SplitMix64 finaliser of seed + (k + 1) * 0x9E3779B97F4A7C15,
//                   its top 53 bits scaled to [0, 1).  Draw (c ns + s) D + d
//                   moves joint d of support point s in copy c; draw
//                   k_near ns D + i D + d is joint d of uniform sample i.
//                   Values are formed in FP64 (lo + (hi - lo) u, the sum, the
//                   clip) and rounded to FP32 once; both an FP64 and an FP32
//                   copy are written.
//   margins         F_j = sum_{s < ns} alpha_s K_sj over the carried support
//                   points (the first ns rows), ascending s, one FP64 fused
//                   multiply-add per term as in Eq. 8; one thread per j reads
//                   row s of the symmetric stored matrix, so a warp's loads
//                   are contiguous.
#include "fk_internal.h"

namespace fk {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double draw_uniform(uint64_t seed, uint64_t k, double lo, double hi) {
  const double u = (double)(splitmix64(seed, k) >> 11) * 0x1p-53;
  return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u));
}

__global__ void __launch_bounds__(256) active_samples_kernel(const ActiveArgs a) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int D = a.D;
  const int64_t rows = a.ns * (1 + (int64_t)a.k_near) + a.n_uniform;
  if (e >= rows * D) return;
  const int64_t r = e / D;
  const int d = (int)(e % D);
  double v;
  if (r < a.ns) {
    v = a.S[r * D + d];
  } else if (r < a.ns * (1 + (int64_t)a.k_near)) {
    const int64_t cs = r - a.ns;  // c * ns + s
    const int64_t s = cs % a.ns;
    v = __dadd_rn(a.S[s * D + d], draw_uniform(a.seed, (uint64_t)(cs * D + d), -a.sigma, a.sigma));
    v = fmin(fmax(v, -a.qlim), a.qlim);
    v = (double)__double2float_rn(v);
  } else {
    const int64_t i = r - a.ns * (1 + (int64_t)a.k_near);
    v = draw_uniform(a.seed, (uint64_t)(a.k_near * a.ns * D + i * D + d), -a.qlim, a.qlim);
    v = (double)__double2float_rn(v);
  }
  a.X[e] = v;
  if (a.X32) a.X32[e] = (float)v;
}

cudaError_t launch_active_samples(const ActiveArgs &a, cudaStream_t s) {
  const int64_t total = (a.ns * (1 + (int64_t)a.k_near) + a.n_uniform) * a.D;
  if (total <= 0) return cudaSuccess;
  active_samples_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename GT>
__global__ void __launch_bounds__(256) margins_kernel(const GT *__restrict__ G, int64_t N,
                                                      const double *__restrict__ alpha, int64_t ns,
                                                      double *__restrict__ F) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double f = 0.0;
  for (int64_t s = 0; s < ns; ++s) f = __fma_rn(alpha[s], (double)G[s * N + j], f);
  F[j] = f;
}

cudaError_t launch_margins(const void *G, int g32, int64_t N, const double *alpha, int64_t ns, double *F,
                           cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((N + 255) / 256);
  if (g32)
    margins_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(G), N, alpha, ns, F);
  else
    margins_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(G), N, alpha, ns, F);
  return cudaGetLastError();
}

}  // namespace fk
