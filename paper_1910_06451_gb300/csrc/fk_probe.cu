// Pipe throughput probes: register-only loops of one instruction class with
// eight independent dependency chains per thread, timed with the SM clock.
// They give the per-SM issue rates that bound the scoring kernels (FP32 FMA,
// packed FP32x2 FMA, MUFU reciprocal, packed FP16x2 FMA, FP64 FMA, FP16x2 ex2).
#include <cuda_fp16.h>

#include "fk_internal.h"

namespace fk {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void probe_kernel(int iters, long long *rec, float *sink) {
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  __syncthreads();
  const long long t0 = clock64();
  float acc = 0.f;
  if (KIND == 0 || KIND == 2) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (threadIdx.x + c);
    const float b = 0.999f, cc = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
          if (KIND == 0)
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(b), "f"(cc));
          else
            asm volatile("rcp.approx.ftz.f32 %0, %0;\n\tadd.f32 %0, %0, %1;" : "+f"(x[c]) : "f"(cc));
        }
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
  } else if (KIND == 1) {
    unsigned long long x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const float lo = 1.0f + 1e-3f * c, hi = 1.0f - 1e-3f * c;
      x[c] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    }
    const unsigned long long b = ((unsigned long long)__float_as_uint(0.999f) << 32) | __float_as_uint(0.999f);
    const unsigned long long cc = ((unsigned long long)__float_as_uint(1e-4f) << 32) | __float_as_uint(1e-4f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(b), "l"(cc));
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += __uint_as_float((unsigned)x[c]);
  } else if (KIND == 3 || KIND == 5) {
    uint32_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const __half2 h = __floats2half2_rn(0.5f + 1e-3f * c, 0.25f);
      x[c] = *reinterpret_cast<const uint32_t *>(&h);
    }
    const __half2 hb = __floats2half2_rn(0.999f, 0.999f), hc = __floats2half2_rn(1e-3f, 1e-3f);
    const uint32_t b = *reinterpret_cast<const uint32_t *>(&hb), cc = *reinterpret_cast<const uint32_t *>(&hc);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
          if (KIND == 3)
            asm volatile("fma.rn.f16x2 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(b), "r"(cc));
          else
            asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(x[c]));
        }
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += __half2float(reinterpret_cast<const __half2 *>(&x[c])->x);
  } else {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(0.999), "d"(1e-4));
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += (float)x[c];
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x + 0] = smid;
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
  if (acc == 12345.678f) sink[0] = acc;
}

// Mixed streams: kind 6 = FFMA2 + FFMA, 7 = FFMA2 + HFMA2, 8 = FFMA + HFMA2,
// 9 = FFMA2 + 2 FFMA; four independent chains of each instruction.
template <int KIND>
__global__ void probe_mixed_kernel(int iters, long long *rec, float *sink) {
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  __syncthreads();
  const long long t0 = clock64();
  unsigned long long x2[4];
  float xs[8];
  uint32_t xh[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    x2[c] = ((unsigned long long)__float_as_uint(1.0f - 1e-3f * c) << 32) | __float_as_uint(1.0f + 1e-3f * c);
    const __half2 h = __floats2half2_rn(0.5f + 1e-3f * c, 0.25f);
    xh[c] = *reinterpret_cast<const uint32_t *>(&h);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) xs[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  const unsigned long long b2 = ((unsigned long long)__float_as_uint(0.999f) << 32) | __float_as_uint(0.999f);
  const unsigned long long c2 = ((unsigned long long)__float_as_uint(1e-4f) << 32) | __float_as_uint(1e-4f);
  const __half2 hb = __floats2half2_rn(0.999f, 0.999f), hc = __floats2half2_rn(1e-3f, 1e-3f);
  const uint32_t bh = *reinterpret_cast<const uint32_t *>(&hb), ch = *reinterpret_cast<const uint32_t *>(&hc);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (KIND == 6 || KIND == 7 || KIND == 9)
          asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x2[c]) : "l"(b2), "l"(c2));
        if (KIND == 6 || KIND == 8 || KIND == 9)
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(xs[c]) : "f"(0.999f), "f"(1e-4f));
        if (KIND == 9)
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(xs[c + 4]) : "f"(0.999f), "f"(1e-4f));
        if (KIND == 7 || KIND == 8)
          asm volatile("fma.rn.f16x2 %0, %0, %1, %2;" : "+r"(xh[c]) : "r"(bh), "r"(ch));
      }
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c)
    acc += __uint_as_float((unsigned)x2[c]) + xs[c] + xs[c + 4] + __half2float(reinterpret_cast<const __half2 *>(&xh[c])->x);
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x + 0] = smid;
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
  if (acc == 12345.678f) sink[0] = acc;
}

int probe_iters(int kind) { return kind == 4 ? 64 : 2048; }
// lane-operations per iteration of the unrolled body
int probe_ops_per_iter(int kind) {
  switch (kind) {
    case 1: case 3: case 5: return kUnroll * kChains * 2;
    case 6: return kUnroll * 4 * 3;   // FFMA2 (2) + FFMA (1)
    case 7: return kUnroll * 4 * 4;   // FFMA2 (2) + HFMA2 (2)
    case 8: return kUnroll * 4 * 3;   // FFMA (1) + HFMA2 (2)
    case 9: return kUnroll * 4 * 4;   // FFMA2 (2) + 2 FFMA
    default: return kUnroll * kChains;
  }
}

cudaError_t launch_probe(int kind, int blocks, int threads, long long *rec, cudaStream_t s) {
  static float *sink = nullptr;
  if (!sink) {
    cudaError_t e = cudaMalloc(&sink, sizeof(float));
    if (e != cudaSuccess) return e;
  }
  const int iters = probe_iters(kind);
  switch (kind) {
    case 0: probe_kernel<0><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 1: probe_kernel<1><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 2: probe_kernel<2><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 3: probe_kernel<3><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 4: probe_kernel<4><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 5: probe_kernel<5><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 6: probe_mixed_kernel<6><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 7: probe_mixed_kernel<7><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 8: probe_mixed_kernel<8><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    case 9: probe_mixed_kernel<9><<<blocks, threads, 0, s>>>(iters, rec, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fk
