// Checks of the premises of the score kernel's error bound (the band of
// fk_score_band), run on the device that scores:
//   rcp      the MUFU reciprocal rcp.approx.ftz.f32 on every FP32 mantissa of
//            a range of binades: the bound assumes |rcp(x) x - 1| <= 2^-23;
//   sincos   the pair-arithmetic sine and cosine of fk_dfk.cuh on every FP32
//            angle of [-hi, hi] (plus a pair offset) against FP64;
//   forward  the pair-arithmetic kinematics of the score kernels, scaled and
//            rounded to FP32, for comparison with FP64 kinematics.
#include <cstdint>
#include <cstring>

#include "fk_dfk.cuh"
#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace fk {

// Largest of non-negative doubles through their bit patterns, which order
// like the values.
__device__ __forceinline__ void atomic_max_pos(unsigned long long *dst, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
    b = x > b ? x : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(dst, b);
}

__global__ void check_rcp_kernel(int e_lo, int64_t count, unsigned long long *out) {
  double worst = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint32_t m = (uint32_t)(i & ((1 << 23) - 1));
    const uint32_t e = (uint32_t)(e_lo + 127 + (int)(i >> 23));
    const float x = __uint_as_float((e << 23) | m);
    const float r = rcp_approx(x);
    worst = fmax(worst, fabs((double)r * (double)x - 1.0));  // the product is exact in FP64
  }
  atomic_max_pos(out, worst);
}

__global__ void check_sincos_kernel(uint32_t nbits, double th0, unsigned long long *out) {
  const float t0h = __double2float_rn(th0), t0l = __double2float_rn(th0 - (double)t0h);
  double worst = 0.0;
  const int64_t count = 2 * (int64_t)nbits;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) {
    const float a = __uint_as_float((uint32_t)(i >> 1));
    const float x = (i & 1) ? -a : a;
    dd s, c;
    dd_sincos(dd_add(dd_of(x), dd{t0h, t0l}), s, c);
    double rs, rc;
    sincos((double)x + th0, &rs, &rc);
    worst = fmax(worst, fmax(fabs((double)s.h + (double)s.l - rs), fabs((double)c.h + (double)c.l - rc)));
  }
  atomic_max_pos(out, worst);
}

__global__ void forward_dd_kernel(const ChainF c, const float *__restrict__ q, int64_t n, double scale,
                                  float *__restrict__ cp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float qv[FK_MAX_DOF];
  for (int k = 0; k < c.D; ++k) qv[k] = q[i * c.D + k];
  const float gh = __double2float_rn(scale);
  float p[FK_MAX_CP][3];
  fk_points_dd<FK_MAX_CP>(c, qv, dd{gh, __double2float_rn(scale - (double)gh)}, p);
  for (int v = 0; v < c.Mv; ++v)
    for (int r = 0; r < 3; ++r) cp[(v * 3 + r) * n + i] = p[v][r];
}

cudaError_t launch_check_rcp(int e_lo, int e_hi, unsigned long long *out, cudaStream_t s) {
  const int64_t count = (int64_t)(e_hi - e_lo + 1) << 23;
  check_rcp_kernel<<<1216, 256, 0, s>>>(e_lo, count, out);
  return cudaGetLastError();
}

cudaError_t launch_check_sincos(float hi, double th0, unsigned long long *out, cudaStream_t s) {
  uint32_t hb = 0;
  memcpy(&hb, &hi, sizeof hb);
  const uint32_t nbits = hb + 1u;  // every FP32 value of [0, hi]
  check_sincos_kernel<<<2432, 256, 0, s>>>(nbits, th0, out);
  return cudaGetLastError();
}

cudaError_t launch_forward_dd(const ChainF &c, const float *q, int64_t n, double scale, float *cp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  forward_dd_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c, q, n, scale, cp);
  return cudaGetLastError();
}

}  // namespace fk
