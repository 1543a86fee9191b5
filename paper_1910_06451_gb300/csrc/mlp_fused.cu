// Fused inference of the learned surrogate (not part of the paper): features,
// the three 256-wide layers and the output unit of the 64-256-256-256-1 MLP
// in one persistent kernel on the tcgen05 tensor cores, so that no hidden
// activation leaves the SM.
//
// One CTA of 128 threads per SM takes tiles of 128 queries in turn.  Per tile:
//   features   each thread computes its query's 64 BF16 features (the same
//              function as the training path) into shared memory, in the
//              no-swizzle core-matrix layout of an A operand;
//   layer 1    4 MMAs (M = 128, N = 256, K = 16) against W1, which stays in
//              shared memory for the whole launch; accumulator in tensor
//              memory columns 0..255;
//   epilogue   the 4 warps read their 32 rows back (tcgen05.ld), add the
//              bias, apply ReLU, round to BF16 and write the 128 x 256 hidden
//              tile into shared memory as the next layer's A operand;
//   layers 2/3 the same with W2 and W3 streamed from L2 in four 64-wide K
//              chunks through two 32 KB shared-memory stages (cp.async;
//              chunk c + 2 is copied once the MMAs of chunk c are committed),
//              accumulators alternating between columns 256..511 and 0..255;
//   output     bias + ReLU of layer 3, dot with w4 in FP32, plus b4: the
//              network output; optionally the confidence decision (label of
//              sign(out * scale) where |out * scale| > tau, else the query
//              joins the fallback list).
// The BF16 rounding points are those of the layer-by-layer path (features,
// hidden layers 1 and 2; layer 3 is used in FP32), and the MMAs accumulate in
// the same order, so both paths give the same outputs.
//
// Every mbarrier wait is bounded; on a timeout the CTA agrees through
// __syncthreads_and, drains (bounded) the MMAs it issued, frees its tensor
// memory, raises an error bit and returns.
#include "surr_features.cuh"
#include "tc_gemm.cuh"

namespace fk {

constexpr int kMlpThreads = 128;
constexpr uint32_t kW1Bytes = kSurrW * kSurrIn * 2;   // 32 KB
constexpr uint32_t kA0Bytes = kBM * kSurrIn * 2;      // 16 KB
constexpr uint32_t kHChunk = kBM * kBK * 2;           // 16 KB: 128 rows x 64 K
constexpr uint32_t kHBytes = 4 * kHChunk;             // 64 KB
constexpr uint32_t kWStage = kSurrW * kBK * 2;        // 32 KB: 256 rows x 64 K
constexpr uint32_t kOffA0 = kW1Bytes, kOffH = kOffA0 + kA0Bytes, kOffWS = kOffH + kHBytes;
constexpr uint32_t kMlpSmem = kOffWS + 2 * kWStage;   // 176 KB
constexpr uint32_t kMlpIdesc = idesc_bf16_f32(kBM, kSurrW);

// core-matrix offset of element (row, k) in a [rows][64] K-major tile
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// 256 x 64 K-chunk of a K-major weight matrix with leading dimension ld.
__device__ __forceinline__ void load_wchunk(uint8_t *dst, const bf16 *W, int ld, int k0, int tid) {
  for (int p = tid; p < kSurrW * 8; p += kMlpThreads) {
    const int row = p % kSurrW, kg = p / kSurrW;
    cp_async16(dst + ((row >> 3) * 8 + kg) * 128 + (row & 7) * 16, W + (int64_t)row * ld + k0 + kg * 8);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(kMlpThreads, 1) mlp_fused_kernel(const ChainF c, const MlpArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar_mma, bar_st[2];
  __shared__ uint32_t tmem_slot;
  uint8_t *W1s = sm, *A0 = sm + kOffA0, *H = sm + kOffH, *WS = sm + kOffWS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&tmem_slot, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_mma, 1);
    mbar_init(&bar_st[0], 1);
    mbar_init(&bar_st[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // W1 once for the whole launch
  for (int p = tid; p < kSurrW * 8; p += kMlpThreads) {
    const int row = p % kSurrW, kg = p / kSurrW;
    cp_async16(W1s + ((row >> 3) * 8 + kg) * 128 + (row & 7) * 16, a.w1 + (int64_t)row * kSurrIn + kg * 8);
  }
  cp_async_commit();
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
  const int r = warp * 32 + lane;                      // this thread's row of the tile

  uint32_t mma_phase = 0;       // completed waits on bar_mma
  uint32_t st_uses[2] = {0, 0};  // commits issued to each stage barrier
  bool ok = true;
  int last_stage = -1;           // stage of the last commit (for the drain)

  // one hidden layer: acc = Hin (128 x 256, four chunks) x W^T, W streamed
  auto layer = [&](const bf16 *W, uint32_t acc) -> bool {
    load_wchunk(WS, W, kSurrW, 0, tid);
    load_wchunk(WS + kWStage, W, kSurrW, kBK, tid);
    for (int kc = 0; kc < 4; ++kc) {
      const int s = kc & 1;
      if (kc < 3) cp_async_wait<1>(); else cp_async_wait<0>();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_base = smem_u32(H + kc * kHChunk), b_base = smem_u32(WS + s * kWStage);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)
          tc_mma(tmem + acc, smem_desc(a_base + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024),
                 kMlpIdesc, (kc > 0 || kk > 0) ? 1u : 0u);
        tc_commit(&bar_st[s]);
      }
      ++st_uses[s];
      last_stage = s;
      if (kc + 2 < 4) {
        // the MMAs of chunk kc read stage s: wait for them before refilling it
        const bool got = mbar_wait_bounded(&bar_st[s], (st_uses[s] - 1) & 1, a.wait_limit);
        if (!__syncthreads_and(got)) return false;
        load_wchunk(WS + s * kWStage, W, kSurrW, (kc + 2) * kBK, tid);
      }
    }
    // the last chunk's commit completes every MMA of the layer
    const bool got = mbar_wait_bounded(&bar_st[1], (st_uses[1] - 1) & 1, a.wait_limit);
    if (!__syncthreads_and(got)) return false;
    // the other stage's last commit precedes it; keep the phase bookkeeping exact
    const bool got0 = mbar_wait_bounded(&bar_st[0], (st_uses[0] - 1) & 1, a.wait_limit);
    if (!__syncthreads_and(got0)) return false;
    tc_fence_after();
    return true;
  };
  // bias + ReLU of accumulator columns, BF16 into H as the next A operand
  auto epilogue_hidden = [&](uint32_t acc, const float *bias) {
#pragma unroll 1
    for (int j0 = 0; j0 < kSurrW; j0 += 16) {
      float v[16];
      tc_ld16(tmem + trow + acc + j0, v);
      __align__(16) bf16 hb[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) hb[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[j0 + i], 0.f));
      uint8_t *chunk = H + (j0 >> 6) * kHChunk;
      *reinterpret_cast<uint4 *>(chunk + cm_off(r, j0 & 63)) = reinterpret_cast<const uint4 *>(hb)[0];
      *reinterpret_cast<uint4 *>(chunk + cm_off(r, (j0 & 63) + 8)) = reinterpret_cast<const uint4 *>(hb)[1];
    }
    tc_fence_before();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  };

  for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
    const int64_t row = t * kBM + r;
    // features of this thread's query into A0
    {
      __align__(16) bf16 h[kSurrIn];
      surr_feature_row(c, row < a.n ? a.q + row * c.D : nullptr, h);
#pragma unroll
      for (int kg = 0; kg < kSurrIn / 8; ++kg)
        *reinterpret_cast<uint4 *>(A0 + cm_off(r, kg * 8)) = reinterpret_cast<const uint4 *>(h)[kg];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // layer 1: A0 x W1^T -> columns 0..255
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_u32(A0), b_base = smem_u32(W1s);
#pragma unroll
      for (int kk = 0; kk < kSurrIn / 16; ++kk)
        tc_mma(tmem, smem_desc(a_base + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024), kMlpIdesc,
               kk > 0 ? 1u : 0u);
      tc_commit(&bar_mma);
    }
    {
      const bool got = mbar_wait_bounded(&bar_mma, mma_phase & 1, a.wait_limit);
      ++mma_phase;
      if (!__syncthreads_and(got)) {
        ok = false;
        if (tid == 0) mbar_wait_bounded(&bar_mma, (mma_phase - 1) & 1, kGemmDrain);
        break;
      }
    }
    tc_fence_after();
    epilogue_hidden(0, a.b1);
    // layer 2: H x W2^T -> columns 256..511, then back into H
    if (!layer(a.w2, 256)) {
      ok = false;
      break;
    }
    epilogue_hidden(256, a.b2);
    // layer 3: H x W3^T -> columns 0..255, then the output unit
    if (!layer(a.w3, 0)) {
      ok = false;
      break;
    }
    float dot = 0.f;
#pragma unroll 1
    for (int j0 = 0; j0 < kSurrW; j0 += 16) {
      float v[16];
      tc_ld16(tmem + trow + j0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) dot = fmaf(fmaxf(v[i] + a.b3[j0 + i], 0.f), a.w4[j0 + i], dot);
    }
    const float o = dot + *a.b4;
    const bool valid = row < a.n;
    if (valid && a.out) a.out[row] = o;
    if (a.decide) {
      const float p = o * a.scale;
      const bool fb = valid && !(fabsf(p) > a.tau);
      if (valid) {
        if (a.pred) a.pred[row] = p;
        a.label[row] = p >= 0.f ? 1 : -1;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, fb);
      if (bal) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.fb_cnt, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fb) a.fb_idx[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)row;
      }
    }
    // every warp is done with the accumulators and A0 before the next tile
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (!ok) {
    // drain (bounded) whatever was committed last, then report
    if (tid == 0) {
      if (last_stage >= 0) mbar_wait_bounded(&bar_st[last_stage], (st_uses[last_stage] - 1) & 1, kGemmDrain);
      atomicOr(a.err, kErrTimeout);
    }
    cp_async_wait<0>();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

cudaError_t launch_mlp_fused(const ChainF &c, const MlpArgs &a0, cudaStream_t s) {
  if (a0.n <= 0) return cudaSuccess;
  MlpArgs a = a0;
  a.ntiles = (a.n + kBM - 1) / kBM;
  cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = a.ntiles < sms ? a.ntiles : sms;
  mlp_fused_kernel<<<(unsigned)grid, kMlpThreads, kMlpSmem, s>>>(c, a);
  return cudaGetLastError();
}

}  // namespace fk
