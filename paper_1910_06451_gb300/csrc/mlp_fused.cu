// Fused inference of the learned surrogate (not part of the paper): the three
// 256-wide layers and the output unit of the 64-256-256-256-1 MLP in one
// persistent, warp-specialised kernel on the tcgen05 tensor cores, so that no
// hidden activation leaves the SM.
//
// Inputs are laid out for the tensor core once per call:
//   features   surr_features_tiled_kernel writes each tile of 128 queries'
//              BF16 features as one contiguous 16 KB block in the no-swizzle
//              core-matrix layout of an A operand;
//   weights    mlp_prep_weights_kernel writes W1 and the four 64-wide K
//              chunks of W2 and of W3 as nine contiguous 32 KB blocks in the
//              layout of a B operand (256 rows x 64 K),
// so that every operand transfer is one 1-D TMA bulk copy (cp.async.bulk with
// an mbarrier completing on the byte count).
//
// One CTA of 9 warps per SM takes tiles of 128 queries in turn:
//   warp 8     producer: one thread issues the bulk copies of W1 (once), of
//              each tile's features (two buffers) and of the eight weight
//              chunks of each tile (a ring of three 32 KB stages), each after
//              the MMAs that read the previous occupant have committed;
//   warps 0-7  thread 0 issues the MMAs (M = 128, N = 256, K = 16) and
//              commits them; all eight read the accumulators back
//              (tcgen05.ld, 32 columns per wait; warps w and w + 4 share TMEM
//              lanes 32 (w mod 4) .. + 31 and split the 256 columns), add the
//              bias, apply ReLU and write the BF16 hidden tile into shared
//              memory as the next layer's A operand; warps 0-3 compute the
//              output unit (bias + ReLU of layer 3, dot with w4 in FP32 in
//              ascending order, plus b4) and the optional confidence decision.
// Accumulators: layer 1 and 3 in TMEM columns 0..255, layer 2 in 256..511.
// The BF16 rounding points and the MMA order are those of the layer-by-layer
// path, so both give the same outputs.
//
// Every mbarrier wait is bounded (try_wait polls, which suspend the thread in
// hardware until the phase flips).  A thread whose wait gives up sets an abort
// flag in shared memory; every loop checks it; before the CTA exits, the MMAs
// and copies it issued are drained (bounded), tensor memory is freed and an
// error bit is raised.
#include "surr_features.cuh"
#include "tc_gemm.cuh"

namespace fk {

constexpr int kMlpCompute = 256;                        // warps 0-7
constexpr int kMlpThreads = kMlpCompute + 32;           // + producer warp 8
constexpr uint32_t kTileA = kBM * kSurrIn * 2;          // 16 KB of features per tile
constexpr uint32_t kWBlock = kSurrW * kBK * 2;          // 32 KB: 256 rows x 64 K
constexpr uint32_t kHChunk = kBM * kBK * 2;             // 16 KB: 128 rows x 64 K
constexpr uint32_t kOffA = kWBlock, kOffH = kOffA + 2 * kTileA, kOffWS = kOffH + 4 * kHChunk;
constexpr int kStages = 3;
constexpr uint32_t kMlpSmem = kOffWS + kStages * kWBlock;  // 224 KB
constexpr uint32_t kMlpIdesc = idesc_bf16_f32(kBM, kSurrW);

// core-matrix offset of element (row, k) in a [rows][64] K-major tile
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// ------------------------------------------------------------ layouts ---
__global__ void __launch_bounds__(128) surr_features_tiled_kernel(const ChainF c, const float *__restrict__ q, int64_t n,
                                                                 int64_t rows, uint8_t *__restrict__ Xc) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= rows) return;
  __align__(16) bf16 h[kSurrIn];
  surr_feature_row(c, k < n ? q + k * c.D : nullptr, h);
  uint8_t *tile = Xc + (k / kBM) * kTileA;
  const int r = (int)(k % kBM);
#pragma unroll
  for (int kg = 0; kg < kSurrIn / 8; ++kg)
    *reinterpret_cast<uint4 *>(tile + cm_off(r, kg * 8)) = reinterpret_cast<const uint4 *>(h)[kg];
}

// Wc = [W1][W2 chunk 0..3][W3 chunk 0..3], each 256 rows x 64 K in the
// core-matrix layout of a B operand.
__global__ void __launch_bounds__(256) mlp_prep_weights_kernel(const bf16 *__restrict__ w1, const bf16 *__restrict__ w2,
                                                              const bf16 *__restrict__ w3, uint8_t *__restrict__ Wc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte unit
  if (e >= 9 * kSurrW * 8) return;
  const int b = e / (kSurrW * 8), u = e % (kSurrW * 8);
  const int row = u % kSurrW, kg = u / kSurrW;
  const bf16 *src = b == 0 ? w1 + (int64_t)row * kSurrIn + kg * 8
                           : (b <= 4 ? w2 : w3) + (int64_t)row * kSurrW + ((b - 1) % 4) * kBK + kg * 8;
  *reinterpret_cast<uint4 *>(Wc + (size_t)b * kWBlock + ((row >> 3) * 8 + kg) * 128 + (row & 7) * 16) =
      *reinterpret_cast<const uint4 *>(src);
}

// -------------------------------------------------------------- kernel ---
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

// barrier over the compute warps only (the producer warp never joins)
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kMlpCompute) : "memory"); }
// the same barrier, returning the AND of v over the compute threads: every
// compute thread takes the same decision from it
__device__ __forceinline__ bool compute_sync_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kMlpCompute)
      : "memory");
  return r != 0;
}

struct MlpShared {
  uint64_t bar_w1, full_a[2], empty_a[2], full_w[kStages], empty_w[kStages], bar_acc;
  uint32_t tmem_slot;
  int abort;
};

__global__ void __launch_bounds__(kMlpThreads, 1) mlp_fused_kernel(const MlpArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ MlpShared sh;
  uint8_t *W1s = sm, *Abuf = sm + kOffA, *H = sm + kOffH, *WS = sm + kOffWS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&sh.tmem_slot, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&sh.bar_w1, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.full_a[i], 1);
      mbar_init(&sh.empty_a[i], 1);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh.full_w[i], 1);
      mbar_init(&sh.empty_w[i], 1);
    }
    mbar_init(&sh.bar_acc, 1);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem_slot;
  const uint32_t lim = a.wait_limit;
  auto give_up = [&]() { atomicExch(&sh.abort, 1); };
  auto aborted = [&]() { return *(volatile int *)&sh.abort != 0; };

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t issued_a[2] = {0, 0}, issued_w[kStages] = {0, 0, 0};
      mbar_arrive_expect_tx(&sh.bar_w1, kWBlock);
      tma_bulk_load(W1s, a.wc, kWBlock, &sh.bar_w1);
      int64_t g = 0;
      for (int64_t it = 0, t = blockIdx.x; t < a.ntiles && !aborted(); ++it, t += gridDim.x) {
        const int ab = (int)(it & 1);
        if (issued_a[ab] > 0 && !mbar_wait_suspend(&sh.empty_a[ab], (issued_a[ab] - 1) & 1, lim)) {
          give_up();
          break;
        }
        mbar_arrive_expect_tx(&sh.full_a[ab], kTileA);
        tma_bulk_load(Abuf + ab * kTileA, a.xc + t * kTileA, kTileA, &sh.full_a[ab]);
        ++issued_a[ab];
        bool stop = false;
        for (int j = 0; j < 8; ++j, ++g) {
          const int s = (int)(g % kStages);
          if (issued_w[s] > 0 && !mbar_wait_suspend(&sh.empty_w[s], (issued_w[s] - 1) & 1, lim)) {
            give_up();
            stop = true;
            break;
          }
          mbar_arrive_expect_tx(&sh.full_w[s], kWBlock);
          tma_bulk_load(WS + s * kWBlock, a.wc + (size_t)(1 + j) * kWBlock, kWBlock, &sh.full_w[s]);
          ++issued_w[s];
        }
        if (stop) break;
      }
      if (aborted()) {
        // let every copy this thread issued land before the CTA can exit
        for (int i = 0; i < 2; ++i)
          if (issued_a[i] > 0) mbar_wait_suspend(&sh.full_a[i], (issued_a[i] - 1) & 1, kGemmDrain);
        for (int i = 0; i < kStages; ++i)
          if (issued_w[i] > 0) mbar_wait_suspend(&sh.full_w[i], (issued_w[i] - 1) & 1, kGemmDrain);
        mbar_wait_suspend(&sh.bar_w1, 0, kGemmDrain);
      }
    }
  } else {
    // ------------------------------------------------------------ compute
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t trow = (uint32_t)(quad * 32) << 16;  // this warp's TMEM lanes
    const int r = quad * 32 + lane;                     // this thread's row of the tile
    uint32_t n_acc = 0;                                 // commits to bar_acc so far
    bool acc_pending = false;                           // a commit not yet waited for
    int64_t g = 0;
    bool ok = mbar_wait_suspend(&sh.bar_w1, 0, lim);
    if (!ok) give_up();
    ok = compute_sync_and(ok);

    // wait for the layer's MMAs (every compute thread), then read TMEM; all
    // compute threads agree on going on (a failed wait anywhere, the
    // producer's included, stops them all at the same point)
    auto wait_acc = [&]() -> bool {
      const bool got = mbar_wait_suspend(&sh.bar_acc, (n_acc - 1) & 1, lim);
      if (!got) give_up();
      acc_pending = !got;
      if (!compute_sync_and(got && !aborted())) return false;
      tc_fence_after();
      return true;
    };
    // bias + ReLU of this warp's half of the columns, BF16 into H
    auto epilogue_hidden = [&](uint32_t col0, const float *bias) {
#pragma unroll 1
      for (int j0 = half * 128; j0 < half * 128 + 128; j0 += 32) {
        float v[32];
        tc_ld32(tmem + trow + col0 + j0, v);
        __align__(16) bf16 hb[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) hb[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[j0 + i], 0.f));
        uint8_t *chunk = H + (j0 >> 6) * kHChunk;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          *reinterpret_cast<uint4 *>(chunk + cm_off(r, (j0 & 63) + 8 * u)) = reinterpret_cast<const uint4 *>(hb)[u];
      }
      tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      compute_sync();
    };
    // layer 2 or 3: H (four chunks) x W^T, the chunks from the ring
    auto issue_layer = [&](uint32_t col0) {
      if (tid == 0) {
        tc_fence_after();
        for (int kc = 0; kc < 4; ++kc) {
          const int64_t gg = g + kc;
          const int s = (int)(gg % kStages);
          if (!mbar_wait_suspend(&sh.full_w[s], (uint32_t)((gg / kStages) & 1), lim)) {
            give_up();
            break;
          }
          const uint32_t a_base = smem_u32(H + kc * kHChunk), b_base = smem_u32(WS + s * kWBlock);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            tc_mma(tmem + col0, smem_desc(a_base + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024),
                   kMlpIdesc, (kc > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&sh.empty_w[s]);
        }
        // committed even after a failed wait, so that nobody waits for it in vain
        tc_commit(&sh.bar_acc);
      }
      g += 4;
      ++n_acc;
      acc_pending = true;
    };

    for (int64_t it = 0, t = blockIdx.x; ok && t < a.ntiles; ++it, t += gridDim.x) {
      const int ab = (int)(it & 1);
      // layer 1: features x W1^T -> columns 0..255
      if (tid == 0) {
        if (!mbar_wait_suspend(&sh.full_a[ab], (uint32_t)((it >> 1) & 1), lim)) {
          give_up();
        } else {
          tc_fence_after();
          const uint32_t a_base = smem_u32(Abuf + ab * kTileA), b_base = smem_u32(W1s);
#pragma unroll
          for (int kk = 0; kk < kSurrIn / 16; ++kk)
            tc_mma(tmem, smem_desc(a_base + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024),
                   kMlpIdesc, kk > 0 ? 1u : 0u);
          tc_commit(&sh.empty_a[ab]);
        }
        tc_commit(&sh.bar_acc);  // also after a failed wait (see issue_layer)
      }
      ++n_acc;
      acc_pending = true;
      if (!wait_acc()) break;
      epilogue_hidden(0, a.b1);
      // layer 2 -> columns 256..511
      issue_layer(256);
      if (!wait_acc()) break;
      epilogue_hidden(256, a.b2);
      // layer 3 -> columns 0..255, then the output unit
      issue_layer(0);
      if (!wait_acc()) break;
      if (warp < 4) {
        float dot = 0.f;
#pragma unroll 1
        for (int j0 = 0; j0 < kSurrW; j0 += 32) {
          float v[32];
          tc_ld32(tmem + trow + j0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) dot = fmaf(fmaxf(v[i] + a.b3[j0 + i], 0.f), a.w4[j0 + i], dot);
        }
        const int64_t row = t * kBM + r;
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
      }
      // the next tile's layer 1 overwrites columns 0..255
      tc_fence_before();
      compute_sync();
    }
    if (aborted() && tid == 0 && acc_pending) mbar_wait_suspend(&sh.bar_acc, (n_acc - 1) & 1, kGemmDrain);
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && sh.abort) atomicOr(a.err, kErrTimeout);
  if (warp == 0) tmem_dealloc(tmem, 512);
}

cudaError_t launch_mlp_fused(const ChainF &c, const MlpArgs &a0, uint8_t *xc, uint8_t *wc, cudaStream_t s) {
  if (a0.n <= 0) return cudaSuccess;
  MlpArgs a = a0;
  a.ntiles = (a.n + kBM - 1) / kBM;
  a.xc = xc;
  a.wc = wc;
  const int64_t rows = a.ntiles * kBM;
  surr_features_tiled_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(c, a.q, a.n, rows, xc);
  mlp_prep_weights_kernel<<<(9 * kSurrW * 8 + 255) / 256, 256, 0, s>>>(a.w1, a.w2, a.w3, wc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = a.ntiles < sms ? a.ntiles : sms;
  mlp_fused_kernel<<<(unsigned)grid, kMlpThreads, kMlpSmem, s>>>(a);
  return cudaGetLastError();
}

size_t mlp_xc_bytes(int64_t n) { return (size_t)((n + kBM - 1) / kBM) * kTileA; }
size_t mlp_wc_bytes() { return 9 * (size_t)kWBlock; }

}  // namespace fk
