// Learned surrogate of the FK-kernel score (not part of the paper): features
// from the control points and joint angles, a 64-256-256-256-1 ReLU MLP whose
// layers run on tcgen05 tensor cores (BF16 operands, FP32 accumulation),
// mean-squared-error training with Adam on FP32 master weights, and inference
// that answers confident queries and sends the rest to the exact score.
#include "tc_gemm.cuh"

namespace fk {

template <int NT, int EPI>
static cudaError_t launch_gemm_t(const GemmArgs &g, int splits, cudaStream_t s) {
  constexpr size_t smem = gemm_smem_bytes<NT>();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<NT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(g.M / kBM), (unsigned)(g.N / NT), (unsigned)splits);
  gemm_tc_kernel<NT, EPI><<<grid, kGemmThreads, smem, s>>>(g);
  return cudaGetLastError();
}

// D = A B^T with FP32 output, split along K into `splits` partial products
// written at Cf + z * M * N.
cudaError_t launch_gemm_f32(const GemmArgs &g0, int splits, cudaStream_t s) {
  GemmArgs g = g0;
  if (g.N % 256 == 0) return launch_gemm_t<256, EPI_F32>(g, splits, s);
  if (g.N % 128 == 0) return launch_gemm_t<128, EPI_F32>(g, splits, s);
  return launch_gemm_t<64, EPI_F32>(g, splits, s);
}

}  // namespace fk
