// BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32 accumulators
// in tensor memory.  D[m][n] = sum_k A[m][k] B[n][k] over one K range:
// A is M x K and B is N x K, both K-contiguous ("K-major") BF16 in global
// memory.  One CTA of 128 threads computes a 128 x NT tile:
//
//   - operand tiles of 64 K-elements are copied with cp.async into shared
//     memory in the no-swizzle core-matrix layout: 8 rows x 16 bytes per core
//     matrix (128 B contiguous), core matrices along K 128 B apart (leading
//     byte offset), 8-row groups 1024 B apart (stride byte offset);
//   - two stages: the copy of chunk c+1 overlaps the MMAs of chunk c;
//   - one thread issues tcgen05.mma (M = 128, N = NT, K = 16 per
//     instruction) and tcgen05.commit to the stage's mbarrier;
//   - the 4 warps read the accumulator back with tcgen05.ld (warp w owns
//     TMEM lanes 32w..32w+31, i.e. tile rows) and run the epilogue.
//
// Every mbarrier wait is bounded; on a timeout the CTA agrees through
// __syncthreads_and, drains (bounded) the MMAs it issued, frees its tensor
// memory, raises an error bit and returns.
#pragma once

#include <cuda_bf16.h>

#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace fk {

typedef __nv_bfloat16 bf16;

struct GemmArgs {
  const bf16 *A;
  int64_t lda;
  const bf16 *B;
  int64_t ldb;
  int M, N, K;          // K of one split (grid.z splits along K)
  float *Cf;            // FP32 output; split z at Cf + z * zstride
  int64_t ldcf, zstride;
  int32_t *err;
  uint32_t wait_limit;
};

// Fused surrogate inference (mlp_fused.cu): features, three hidden layers and
// the output unit for n queries in one persistent launch.
struct MlpArgs {
  const float *q;            // [n][D]
  int64_t n, ntiles;         // ntiles is set by the launcher
  const bf16 *w1, *w2, *w3;  // [256][64], [256][256], [256][256], K-major
  const float *b1, *b2, *b3, *w4, *b4;
  float *out;                // network outputs [n] or null
  int decide;                // 1: labels and fallback list below
  float scale, tau;
  float *pred;               // [n] or null: out * scale
  int8_t *label;             // [n]
  int32_t *fb_idx, *fb_cnt;  // fallback list and its length
  int32_t *err;
  uint32_t wait_limit;
  const uint8_t *wc;         // set by the launcher: tiled weights
};
// wc: mlp_wc_bytes() bytes of scratch for the tiled weights.
cudaError_t launch_mlp_fused(const ChainF &c, const MlpArgs &a, uint8_t *wc, cudaStream_t s);
size_t mlp_wc_bytes();

constexpr int kSurrIn = 64;   // surrogate input width (56 features, zero-padded)
constexpr int kSurrW = 256;   // hidden width

constexpr int kGemmThreads = 128;
constexpr int kBM = 128, kBK = 64;
constexpr uint32_t kGemmDrain = 1u << 22;

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 columns of this warp's 32 TMEM lanes (one load, then its wait)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// A TMEM load of 32 columns without its wait, and the wait alone: the wait
// takes the destination registers as operands, so no use of them can be
// scheduled before it.  Lets a warp convert one chunk while the next is in
// flight.
__device__ __forceinline__ void tc_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NT>
constexpr size_t gemm_smem_bytes() {
  return 2 * (size_t)(kBM * kBK * 2 + NT * kBK * 2);
}

template <int NT>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_tc_kernel(const GemmArgs g) {
  static_assert(NT % 16 == 0 && NT >= 32 && NT <= 256, "N tile");
  constexpr uint32_t A_BYTES = kBM * kBK * 2;
  constexpr uint32_t B_BYTES = NT * kBK * 2;
  constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t NCOLS = NT;  // power of two >= 32 for the tiles used
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, NT);
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * NT, z = blockIdx.z;
  const int nk = g.K / kBK;
  const int64_t kbase = (int64_t)z * g.K;

  if (warp == 0) {
    tmem_alloc(&tmem_slot, NCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  auto load_chunk = [&](int c, int s) {
    uint8_t *As = gsm + s * STAGE;
    uint8_t *Bs = As + A_BYTES;
    const int64_t k0 = kbase + (int64_t)c * kBK;
    for (int p = tid; p < kBM * 8; p += kGemmThreads) {
      const int row = p % kBM, kg = p / kBM;
      cp_async16(As + ((row >> 3) * 8 + kg) * 128 + (row & 7) * 16, g.A + (int64_t)(m0 + row) * g.lda + k0 + kg * 8);
    }
    for (int p = tid; p < NT * 8; p += kGemmThreads) {
      const int row = p % NT, kg = p / NT;
      cp_async16(Bs + ((row >> 3) * 8 + kg) * 128 + (row & 7) * 16, g.B + (int64_t)(n0 + row) * g.ldb + k0 + kg * 8);
    }
    cp_async_commit();
  };

  int issued = 0;  // chunks whose MMAs were issued
  bool ok = true;
  load_chunk(0, 0);
  for (int c = 0; c < nk; ++c) {
    const int s = c & 1;
    if (c + 1 < nk) {
      const int s1 = (c + 1) & 1;
      if (c >= 1) {
        // the MMAs of chunk c-1 read stage s1: wait for their commit
        const bool got = mbar_wait_bounded(&bar[s1], ((c - 1) >> 1) & 1, g.wait_limit);
        if (!__syncthreads_and(got)) {
          ok = false;
          cp_async_wait<0>();
          break;
        }
      }
      load_chunk(c + 1, s1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_u32(gsm + s * STAGE), b_base = a_base + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ad = smem_desc(a_base + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b_base + kk * 256, 128, 1024);
        tc_mma(tmem, ad, bd, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&bar[s]);
    }
    issued = c + 1;
  }
  if (issued > 0) {
    const int c = issued - 1;
    const bool got = mbar_wait_bounded(&bar[c & 1], (c >> 1) & 1, ok ? g.wait_limit : kGemmDrain);
    ok = __syncthreads_and(got && ok);
    if (!ok) mbar_wait_bounded(&bar[c & 1], (c >> 1) & 1, kGemmDrain);  // drain what was issued
  } else {
    ok = false;
  }
  tc_fence_after();

  if (ok) {
    const int r = warp * 32 + lane;
    const int64_t gm = m0 + r;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int j0 = 0; j0 < NT; j0 += 16) {
      float v[16];
      tc_ld16(trow + j0, v);
      float *dst = g.Cf + (int64_t)z * g.zstride + gm * g.ldcf + n0 + j0;
#pragma unroll
      for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
  } else if (tid == 0) {
    atomicOr(g.err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

}  // namespace fk
