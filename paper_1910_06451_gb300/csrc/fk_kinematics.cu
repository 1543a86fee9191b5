// Forward kinematics (Sec. II-A, Eqs. 1-2) and the FK-kernel matrix
// (Sec. II-B with Eq. 4) on the GPU.
#include "df_arith.cuh"
#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace fk {

// ------------------------------------------------------------ forward ---
// One thread per configuration; the pose is carried link by link in
// registers and each control point is written when its frame is reached.

__global__ void fk_forward_f32_kernel(const ChainF c, const float *__restrict__ q, int64_t n, float *__restrict__ cp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  PoseF P;
  pose_base(c, P);
  auto emit = [&](int frame) {
    for (int m = 0; m < c.M; ++m)
      if (c.cj[m] == frame) {
        float o[3];
        pose_point(P, c.ct[m], o);
        for (int r = 0; r < 3; ++r) cp[(m * 3 + r) * n + k] = o[r];
      }
  };
  emit(0);
  for (int i = 0; i < c.D; ++i) {
    pose_step(c, i, q[k * c.D + i], P);
    emit(i + 1);
  }
}

template <typename QT>
__global__ void fk_forward_f64_kernel(const ChainD c, const QT *__restrict__ q, int64_t n, double *__restrict__ cp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  PoseD P;
  pose_base(c, P);
  auto emit = [&](int frame) {
    for (int m = 0; m < c.M; ++m)
      if (c.cj[m] == frame) {
        double o[3];
        pose_point(P, c.ct[m], o);
        for (int r = 0; r < 3; ++r) cp[(m * 3 + r) * n + k] = o[r];
      }
  };
  emit(0);
  for (int i = 0; i < c.D; ++i) {
    pose_step(c, i, (double)q[k * c.D + i], P);
    emit(i + 1);
  }
}

static inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_fk_forward_f32(const ChainF &c, const float *q, int64_t n, float *cp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fk_forward_f32_kernel<<<grid_for(n, 128), 128, 0, s>>>(c, q, n, cp);
  return cudaGetLastError();
}

// The FP64 chain runs at 1/64 of the FP32 rate: one warp per CTA spreads a
// few thousand configurations over every SM instead of a few dozen.
constexpr int kFk64Threads = 32;

cudaError_t launch_fk_forward_f64(const ChainD &c, const double *q, int64_t n, double *cp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fk_forward_f64_kernel<double><<<grid_for(n, kFk64Threads), kFk64Threads, 0, s>>>(c, q, n, cp);
  return cudaGetLastError();
}

cudaError_t launch_fk_forward_f32in_f64(const ChainD &c, const float *q, int64_t n, double *cp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fk_forward_f64_kernel<float><<<grid_for(n, kFk64Threads), kFk64Threads, 0, s>>>(c, q, n, cp);
  return cudaGetLastError();
}

// --------------------------------------------------------------- Gram ---
// K[i][j] = (1/M) sum_m K_RQ(FK_m(a_i), FK_m(b_j)) (or the chain's Gaussian
// summand, FK_SUMMAND_GAUSS, which is not the paper's).  One CTA computes a
// 32 x 32 tile with 256 threads (4 rows each).  Control points of the tile's
// 32 + 32 configurations are staged in shared memory as [M*3][32].  With
// sym != 0 only tiles with bi <= bj run; an off-diagonal tile is written
// twice, directly and transposed through shared memory, because the RQ
// summand is exactly symmetric in its arguments.

constexpr int kGT = 32;

struct GramCps {
  int M, Mv, n_const, summand;
  int vidx[FK_MAX_CP];
};

__device__ __forceinline__ double gram_entry(const GramCps &g, double hg, const double *A, const double *B, int ia,
                                             int jb) {
  double s = (double)g.n_const;
  for (int v = 0; v < g.Mv; ++v) {
    const int m = g.vidx[v];
    const double x[3] = {A[(m * 3 + 0) * kGT + ia], A[(m * 3 + 1) * kGT + ia], A[(m * 3 + 2) * kGT + ia]};
    const double y[3] = {B[(m * 3 + 0) * kGT + jb], B[(m * 3 + 1) * kGT + jb], B[(m * 3 + 2) * kGT + jb]};
    s += k_sum_f64(g.summand, hg, x, y);
  }
  return s / (double)g.M;
}

__device__ __forceinline__ float gram_entry(const GramCps &g, float hg, const float *A, const float *B, int ia,
                                            int jb) {
  float s = (float)g.n_const;
  for (int v = 0; v < g.Mv; ++v) {
    const int m = g.vidx[v];
    const float d0 = A[(m * 3 + 0) * kGT + ia] - B[(m * 3 + 0) * kGT + jb];
    const float d1 = A[(m * 3 + 1) * kGT + ia] - B[(m * 3 + 1) * kGT + jb];
    const float d2 = A[(m * 3 + 2) * kGT + ia] - B[(m * 3 + 2) * kGT + jb];
    const float d2s = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
    if (g.summand == FK_SUMMAND_GAUSS) {
      s += expf(-hg * d2s);
    } else {
      const float r = 1.f / fmaf(hg, d2s, 1.f);
      s = fmaf(r, r, s);
    }
  }
  return s / (float)g.M;
}

template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const GramCps g, T hg, const T *__restrict__ cpa, int64_t na,
                                                   const T *__restrict__ cpb, int64_t nb, int sym,
                                                   T *__restrict__ K) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (sym && bi > bj) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *A = reinterpret_cast<T *>(smem_raw);
  const int M = g.M;
  T *B = A + M * 3 * kGT;
  T *O = B + M * 3 * kGT;  // [kGT][kGT + 1] output tile for the transposed write
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)bi * kGT, j0 = (int64_t)bj * kGT;
  for (int e = threadIdx.x; e < M * 3 * kGT; e += blockDim.x) {
    const int row = e / kGT, col = e % kGT;
    A[e] = (i0 + col < na) ? cpa[row * na + i0 + col] : T(0);
    B[e] = (j0 + col < nb) ? cpb[row * nb + j0 + col] : T(0);
  }
  __syncthreads();
  const bool mirror = sym && bi != bj;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int il = ty + 8 * r;
    const T v = gram_entry(g, hg, A, B, il, tx);
    if (i0 + il < na && j0 + tx < nb) K[(i0 + il) * nb + j0 + tx] = v;
    if (mirror) O[il * (kGT + 1) + tx] = v;
  }
  if (!mirror) return;
  __syncthreads();
  // transposed tile: K[j0 + jl][i0 + il] = O[il][jl]
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jl = ty + 8 * r;
    if (j0 + jl < na && i0 + tx < nb) K[(j0 + jl) * nb + i0 + tx] = O[tx * (kGT + 1) + jl];
  }
}

template <typename T>
static cudaError_t launch_gram(const ChainD &c, T gamma, const T *cpa, int64_t na, const T *cpb, int64_t nb, int sym,
                               T *K, cudaStream_t s) {
  if (na <= 0 || nb <= 0) return cudaSuccess;
  GramCps g{c.M, c.Mv, c.n_const, c.summand, {}};
  for (int v = 0; v < c.Mv; ++v) g.vidx[v] = c.vidx[v];
  const int M = c.M;
  const size_t smem = sizeof(T) * (2 * (size_t)M * 3 * kGT + kGT * (kGT + 1));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(grid_for(nb, kGT), grid_for(na, kGT));
  gram_kernel<T><<<grid, 256, smem, s>>>(g, T(0.5) * gamma, cpa, na, cpb, nb, sym, K);
  return cudaGetLastError();
}

cudaError_t launch_gram_f64(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb,
                            int64_t nb, int sym, double *K, cudaStream_t s) {
  return launch_gram<double>(c, gamma, cpa, na, cpb, nb, sym, K, s);
}

cudaError_t launch_gram_f32(const ChainD &c, float gamma, const float *cpa, int64_t na, const float *cpb, int64_t nb,
                            int sym, float *K, cudaStream_t s) {
  return launch_gram<float>(c, gamma, cpa, na, cpb, nb, sym, K, s);
}

// ------------------------------------------------- double-float Gram ---
// The same matrix in double-float arithmetic (df_arith.cuh), on the FP32
// pipes (128 lanes/clk/SM) instead of the FP64 pipe (1.7 lanes/clk/SM on this
// part).  The FP64 control points are scaled by sqrt(gamma/2) and split into
// FP32 pairs once per point (df_split_kernel), so t = 1 + |p - s|^2 and each
// summand is df_rq_term; per entry only the final value touches FP64: the
// pair is widened exactly by integer operations and added (one DADD), then
// scaled by 1/M (one DMUL), the order of the FP64 definition, so a diagonal
// entry (every summand exactly 1) is exactly 1.  Entries come out within
// about 1e-13 of the FP64 ones.

// (h, l) of sqrt(gamma/2) cp for the configuration-dependent points:
// cp SoA [M][3][n] FP64 -> out SoA [Mv*3][n] float2.
__global__ void __launch_bounds__(256) df_split_kernel(const GramCps g, double gs, const double *__restrict__ cp,
                                                      int64_t n, float2 *__restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)g.Mv * 3 * n) return;
  const int row = (int)(e / n);
  const int64_t j = e % n;
  const int v = row / 3, r = row % 3;
  const dfl x = df_from_double(gs * cp[(g.vidx[v] * 3 + r) * n + j]);
  out[e] = make_float2(x.h, x.l);
}

// Exact FP32 -> FP64 widening of a normal value by integer operations (sign,
// rebiased exponent, shifted fraction); zero and subnormal values give 0,
// which for the low word of a pair whose high word is >= 1e-30 changes the
// sum by less than 1e-38.
__device__ __forceinline__ double widen_flush(float x) {
  const unsigned b = __float_as_uint(x), mag = b & 0x7fffffffu;
  if (mag < 0x00800000u) return 0.0;
  return __longlong_as_double((long long)((unsigned long long)(b >> 31) << 63) | (((long long)mag << 29) + (896LL << 52)));
}

template <typename OT>
__global__ void __launch_bounds__(256) gram_df_kernel(const GramCps g, const float2 *__restrict__ da, int64_t na,
                                                     const float2 *__restrict__ db, int64_t nb, int sym,
                                                     OT *__restrict__ K) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (sym && bi > bj) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Mv = g.Mv;
  // [Mv * 6][kGT]: for point v the words x_h, x_l, y_h, y_l, z_h, z_l, each a
  // row over the tile's configurations (consecutive lanes, consecutive words)
  float *A = reinterpret_cast<float *>(smem_raw);
  float *B = A + Mv * 6 * kGT;
  OT *O = reinterpret_cast<OT *>(B + Mv * 6 * kGT);  // [kGT][kGT + 1]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)bi * kGT, j0 = (int64_t)bj * kGT;
  for (int e = threadIdx.x; e < Mv * 3 * kGT; e += blockDim.x) {
    const int row = e / kGT, col = e % kGT;  // row = v * 3 + axis
    const float2 x = (i0 + col < na) ? da[row * na + i0 + col] : make_float2(0.f, 0.f);
    const float2 y = (j0 + col < nb) ? db[row * nb + j0 + col] : make_float2(0.f, 0.f);
    A[(2 * row) * kGT + col] = x.x;
    A[(2 * row + 1) * kGT + col] = x.y;
    B[(2 * row) * kGT + col] = y.x;
    B[(2 * row + 1) * kGT + col] = y.y;
  }
  __syncthreads();
  const double invM = 1.0 / (double)g.M;
  const bool mirror = sym && bi != bj;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int il = ty + 8 * r;
    float kh = (float)g.n_const, kl = 0.f;
    for (int v = 0; v < Mv; ++v) {
      const float *a6 = A + v * 6 * kGT + il, *b6 = B + v * 6 * kGT + tx;
      const float qh[3] = {a6[0], a6[2 * kGT], a6[4 * kGT]};
      const float ql[3] = {a6[kGT], a6[3 * kGT], a6[5 * kGT]};
      const float sv[6] = {b6[0], b6[kGT], b6[2 * kGT], b6[3 * kGT], b6[4 * kGT], b6[5 * kGT]};
      float rh, rl;
      df_rq_term(qh, ql, sv, rh, rl);
      const dfl ks = two_sum(kh, rh);
      kh = ks.h;
      kl += ks.l + rl;
    }
    const OT v = (OT)(__dadd_rn(widen_flush(kh), widen_flush(kl)) * invM);
    if (i0 + il < na && j0 + tx < nb) K[(i0 + il) * nb + j0 + tx] = v;
    if (mirror) O[il * (kGT + 1) + tx] = v;
  }
  if (!mirror) return;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jl = ty + 8 * r;
    if (j0 + jl < na && i0 + tx < nb) K[(j0 + jl) * nb + i0 + tx] = O[tx * (kGT + 1) + jl];
  }
}

template <typename OT>
static cudaError_t launch_gram_df_t(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb,
                                    int64_t nb, int sym, OT *K, float2 *wa, float2 *wb, cudaStream_t s) {
  if (c.summand != FK_SUMMAND_RQ) return cudaErrorInvalidValue;  // double-float form of the RQ summand only
  if (na <= 0 || nb <= 0) return cudaSuccess;
  GramCps g{c.M, c.Mv, c.n_const, c.summand, {}};
  for (int v = 0; v < c.Mv; ++v) g.vidx[v] = c.vidx[v];
  const double gs = sqrt(0.5 * gamma);
  const int64_t ea = (int64_t)c.Mv * 3 * na, eb = (int64_t)c.Mv * 3 * nb;
  if (ea > 0) df_split_kernel<<<(unsigned)((ea + 255) / 256), 256, 0, s>>>(g, gs, cpa, na, wa);
  if (!sym && eb > 0) df_split_kernel<<<(unsigned)((eb + 255) / 256), 256, 0, s>>>(g, gs, cpb, nb, wb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(float) * 2 * (size_t)c.Mv * 6 * kGT + sizeof(OT) * kGT * (kGT + 1);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(gram_df_kernel<OT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(grid_for(nb, kGT), grid_for(na, kGT));
  gram_df_kernel<OT><<<grid, 256, smem, s>>>(g, wa, na, sym ? wa : wb, nb, sym, K);
  return cudaGetLastError();
}

cudaError_t launch_gram_df(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb, int64_t nb,
                           int sym, double *K, float2 *wa, float2 *wb, cudaStream_t s) {
  return launch_gram_df_t<double>(c, gamma, cpa, na, cpb, nb, sym, K, wa, wb, s);
}

cudaError_t launch_gram_df32(const ChainD &c, double gamma, const double *cpa, int64_t na, const double *cpb,
                             int64_t nb, int sym, float *K, float2 *wa, float2 *wb, cudaStream_t s) {
  return launch_gram_df_t<float>(c, gamma, cpa, na, cpb, nb, sym, K, wa, wb, s);
}

}  // namespace fk
