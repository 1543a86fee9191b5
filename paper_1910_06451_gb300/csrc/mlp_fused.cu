// Fused inference of the learned surrogate (not part of the paper): the three
// 256-wide layers and the output unit of the 64-256-256-256-1 MLP in one
// persistent, warp-specialised kernel on the tcgen05 tensor cores, so that no
// hidden activation leaves the SM.
//
// The weights are laid out for the tensor core once per call:
// mlp_prep_weights_kernel writes W1 and the four 64-wide K chunks of W2 and of
// W3 as nine contiguous 32 KB blocks in the no-swizzle core-matrix layout of
// a B operand (256 rows x 64 K), so that every weight transfer is one 1-D TMA
// bulk copy (cp.async.bulk with an mbarrier completing on the byte count).
//
// One CTA of 14 warps per SM takes tiles of 128 queries in turn:
//   warps 10-13 features: one query per thread (forward kinematics, sin/cos
//              of the joints, surr_feature_row), written as BF16 straight
//              into the A-operand layout of one of two 16 KB feature buffers,
//              two tiles ahead of their use; a buffer is refilled once the
//              layer-1 MMAs that read it have committed;
//   warp 8     producer: one thread issues the bulk copies of W1 (once) and
//              of the eight weight chunks of each tile (a ring of two 32 KB
//              stages), each after the MMAs that read the previous occupant
//              have committed;
//   warp 9     MMA issuer: one thread issues the MMAs (M = 128, N = 256,
//              K = 16) and commits them; layers 2 and 3 go K chunk by K chunk
//              (64 wide), each chunk as soon as the eight epilogue warps have
//              written that chunk of the hidden tile (one mbarrier per chunk,
//              one arrival per warp), so the tensor pipe works on chunk c
//              while the warps convert chunk c + 1;
//   warps 0-7  epilogues: read the accumulators back (tcgen05.ld, 32 columns
//              per wait; warps w and w + 4 share TMEM lanes 32 (w mod 4) ..
//              + 31 and take the two 32-column halves of each 64-column
//              chunk), add the bias (b1, b2, b3, w4 staged in shared memory), apply
//              ReLU and write the BF16 hidden tile
//              into shared memory as the next layer's A operand; then the
//              output unit (bias + ReLU of layer 3, dot with w4 in FP32: each
//              thread sums its 128 columns in four interleaved partial sums,
//              warps w + 4 hand their half to warps w, which add it and b4)
//              and the optional confidence decision.  TMEM loads of the next
//              32 columns are in flight while the current ones are converted.
// Accumulators: two regions of 256 TMEM columns.  Tile i of a CTA puts layers
// 1 and 3 in region i mod 2 and layer 2 in the other, so the next tile's
// layer 1 (in the other region, free once layer 2 has been read) runs on the
// tensor pipe while this tile's output unit is computed.
// The BF16 rounding points and the MMA order are those of the layer-by-layer
// path.
//
// Every mbarrier wait is bounded (try_wait polls, which suspend the thread in
// hardware until the phase flips; the MMA warp polls without suspending).  A
// thread whose wait gives up sets an abort flag in shared memory; every loop
// checks it; before the CTA exits, the MMAs and copies it issued are drained
// (bounded), tensor memory is freed and an error bit is raised.
#include <cstddef>

#include "surr_features.cuh"
#include "tc_gemm.cuh"

namespace fk {

constexpr int kMlpCompute = 256;                        // warps 0-7
constexpr int kMlpFeat = 128;                           // warps 10-13: features
constexpr int kMlpThreads = kMlpCompute + 64 + kMlpFeat;  // + producer warp 8, MMA warp 9
constexpr uint32_t kTileA = kBM * kSurrIn * 2;          // 16 KB of features per tile
constexpr uint32_t kWBlock = kSurrW * kBK * 2;          // 32 KB: 256 rows x 64 K
constexpr uint32_t kHChunk = kBM * kBK * 2;             // 16 KB: 128 rows x 64 K
constexpr uint32_t kOffA = kWBlock, kOffH = kOffA + 2 * kTileA, kOffWS = kOffH + 4 * kHChunk;
constexpr int kStages = 2;  // measured against 3: 1.531 against 1.559 ms for 4M queries
constexpr uint32_t kMlpSmem = kOffWS + kStages * kWBlock;  // 192 KB
constexpr uint32_t kMlpIdesc = idesc_bf16_f32(kBM, kSurrW);

// core-matrix offset of element (row, k) in a [rows][64] K-major tile
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// ------------------------------------------------------------ layouts ---
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
// Packed FP32x2 helpers: x + b for two columns in one add.rn.f32x2, and
// ReLU plus rounding to BF16 of both in one cvt (the lower half of the result
// holds the first column; ReLU after rounding equals rounding after ReLU).
__device__ __forceinline__ unsigned long long add2(uint32_t x0, uint32_t x1, float b0, float b1) {
  unsigned long long x, b, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "r"(x0), "r"(x1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(b));
  return r;
}
__device__ __forceinline__ uint32_t relu_bf16x2(unsigned long long v) {
  uint32_t out;
  asm("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tcvt.rn.relu.bf16x2.f32 %0, hi, lo;\n\t}"
      : "=r"(out)
      : "l"(v));
  return out;
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
  uint64_t bar_w1, full_a[2], empty_a[2], full_w[kStages], empty_w[kStages], bar_acc[2], h_full[4], drain;
  uint32_t tmem_slot;
  int abort;
  float half_dot[kBM];  // output unit: the second half of each row's dot
  __align__(16) float bias12[2][kSurrW];  // b1 and b2, read by the epilogues as float4
  __align__(16) float b3w4[2][kSurrW];    // b3 and w4, read by the output unit as float4
};
static_assert(offsetof(MlpShared, bias12) % 16 == 0 && offsetof(MlpShared, b3w4) % 16 == 0,
              "float4 reads of the staged biases");
static_assert(kMlpSmem + sizeof(MlpShared) <= 232448, "above 227 KB of shared memory per CTA");

__global__ void __launch_bounds__(kMlpThreads) mlp_fused_kernel(const MlpArgs a, const ChainF c) {
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
      mbar_init(&sh.full_a[i], kMlpFeat / 32);  // one arrival per feature warp
      mbar_init(&sh.empty_a[i], 1);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh.full_w[i], 1);
      mbar_init(&sh.empty_w[i], 1);
    }
    mbar_init(&sh.bar_acc[0], 1);
    mbar_init(&sh.bar_acc[1], 1);
    for (int c = 0; c < 4; ++c) mbar_init(&sh.h_full[c], 8);  // one arrival per epilogue warp
    mbar_init(&sh.drain, 1);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // b1, b2, b3 and w4 staged once per CTA: the epilogues read them from
  // shared memory instead of through L1 (measured for 4M queries: b1, b2
  // 1.667 -> 1.558 ms; b3, w4 with the two-stage ring 1.531 -> 1.518 ms)
  for (int i = tid; i < 2 * kSurrW; i += kMlpThreads) {
    sh.bias12[i / kSurrW][i % kSurrW] = (i < kSurrW ? a.b1 : a.b2)[i % kSurrW];
    sh.b3w4[i / kSurrW][i % kSurrW] = (i < kSurrW ? a.b3 : a.w4)[i % kSurrW];
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
      uint32_t issued_w[kStages] = {};
      mbar_arrive_expect_tx(&sh.bar_w1, kWBlock);
      tma_bulk_load(W1s, a.wc, kWBlock, &sh.bar_w1);
      const int64_t nt = a.ntiles > (int64_t)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      bool ok = true;
      int64_t g = 0;
      for (int64_t it = 0; it < nt && ok && !aborted(); ++it) {
        for (int j = 0; j < 8 && ok; ++j, ++g) {
          const int s = (int)(g % kStages);
          if (issued_w[s] > 0 && !mbar_wait_suspend(&sh.empty_w[s], (issued_w[s] - 1) & 1, lim)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&sh.full_w[s], kWBlock);
          tma_bulk_load(WS + s * kWBlock, a.wc + (size_t)(1 + j) * kWBlock, kWBlock, &sh.full_w[s]);
          ++issued_w[s];
        }
      }
      if (!ok) give_up();
      if (aborted()) {
        // let every copy this thread issued land before the CTA can exit
        for (int i = 0; i < kStages; ++i)
          if (issued_w[i] > 0) mbar_wait_suspend(&sh.full_w[i], (issued_w[i] - 1) & 1, kGemmDrain);
        mbar_wait_suspend(&sh.bar_w1, 0, kGemmDrain);
      }
    }
  } else if (warp >= 10) {
    // ------------------------------------------------------------ features
    // one query row per thread, written straight into the A-operand layout
    // of the tile's feature buffer (k & 1 for the k-th tile of this CTA),
    // two tiles ahead of its layer 1
    const int fr = tid - (kMlpCompute + 64);
    const int64_t nt = a.ntiles > (int64_t)blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    for (int64_t k = 0; k < nt; ++k) {
      const int ab = (int)(k & 1);
      if (k >= 2) {
        // the buffer's previous tile (k - 2) has been read by its layer 1
        bool got = false;
        for (uint32_t i = 0; i < lim && !got; ++i) {
          got = mbar_try_wait(&sh.empty_a[ab], (uint32_t)(((k >> 1) - 1) & 1));
          if (!got && aborted()) break;
        }
        if (!got) {
          give_up();
          break;
        }
      }
      const int64_t row = (blockIdx.x + k * gridDim.x) * kBM + fr;
      __align__(16) bf16 h[kSurrIn];
      surr_feature_row(c, row < a.n ? a.q + row * c.D : nullptr, h);
      uint8_t *tile = Abuf + ab * kTileA;
#pragma unroll
      for (int kg = 0; kg < kSurrIn / 8; ++kg)
        *reinterpret_cast<uint4 *>(tile + cm_off(fr, kg * 8)) = reinterpret_cast<const uint4 *>(h)[kg];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.full_a[ab]);
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // Bounded wait without suspension: rounds of 64 back-to-back polls.
      // This thread's waits are on the critical path of every 64-wide chunk,
      // and a suspending try_wait wakes up late (measured: 1.79 -> 1.67 ms
      // for 4M queries).  lim / 8 rounds last about as long as the library's
      // other bounded waits; a failed wait elsewhere makes these run out too,
      // so they need no abort check.
      const uint32_t rounds = lim / 8u + (lim % 8u != 0u);
      auto wait = [&](uint64_t *b, uint32_t parity) -> bool {
        for (uint32_t i = 0; i < rounds; ++i) {
#pragma unroll
          for (int k = 0; k < 64; ++k)
            if (mbar_test_wait(b, parity)) return true;
        }
        return false;
      };
      int64_t g = 0;
      // layer 1 of the it-th tile of this CTA: features x W1^T into region reg
      auto layer1 = [&](int64_t it, int reg) -> bool {
        const int ab = (int)(it & 1);
        const bool got = wait(&sh.full_a[ab], (uint32_t)((it >> 1) & 1));
        if (!got) give_up();  // before the commit below wakes the epilogue warps
        if (got) {
          tc_fence_after();
          const uint32_t a_base = smem_u32(Abuf + ab * kTileA), b_base = smem_u32(W1s);
#pragma unroll
          for (int kk = 0; kk < kSurrIn / 16; ++kk)
            tc_mma(tmem + 256 * reg, smem_desc(a_base + kk * 256, 128, 1024),
                   smem_desc(b_base + kk * 256, 128, 1024), kMlpIdesc, kk > 0 ? 1u : 0u);
          tc_commit(&sh.empty_a[ab]);
        }
        // committed even after a failed wait, so that nobody waits for it in vain
        tc_commit(&sh.bar_acc[reg]);
        return got;
      };
      // layer 2 or 3: each 64-wide K chunk of the hidden tile once the
      // epilogue warps have written it (h_full phase hpar), times the
      // matching weight chunk from the ring, into region dst
      auto hidden = [&](uint32_t hpar, int dst) -> bool {
        bool got = true;
        for (int c = 0; c < 4 && got; ++c) {
          const int64_t gg = g + c;
          const int s = (int)(gg % kStages);
          got = wait(&sh.h_full[c], hpar) && wait(&sh.full_w[s], (uint32_t)((gg / kStages) & 1));
          if (!got) give_up();  // before the commit below wakes the epilogue warps
          if (got) {
            tc_fence_after();
            const uint32_t a_base = smem_u32(H + c * kHChunk), b_base = smem_u32(WS + s * kWBlock);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              tc_mma(tmem + 256 * dst, smem_desc(a_base + kk * 256, 128, 1024),
                     smem_desc(b_base + kk * 256, 128, 1024), kMlpIdesc, (c > 0 || kk > 0) ? 1u : 0u);
            tc_commit(&sh.empty_w[s]);
          }
        }
        g += 4;
        tc_commit(&sh.bar_acc[dst]);  // also after a failed wait
        return got;
      };
      bool ok = wait(&sh.bar_w1, 0);
      if (ok && (int64_t)blockIdx.x < a.ntiles) ok = layer1(0, 0);
      for (int64_t it = 0, t = blockIdx.x; ok && t < a.ntiles; ++it, t += gridDim.x) {
        const int R = (int)(it & 1);
        ok = hidden(0, 1 - R) && hidden(1, R);  // layers 2 and 3
        if (ok && t + gridDim.x < a.ntiles) ok = layer1(it + 1, 1 - R);
      }
      if (!ok) give_up();
      // every MMA issued here completes before the CTA can exit
      tc_commit(&sh.drain);
      mbar_wait_suspend(&sh.drain, 0, kGemmDrain);
    }
  } else {
    // ----------------------------------------------------------- epilogues
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t trow = (uint32_t)(quad * 32) << 16;  // this warp's TMEM lanes
    const int r = quad * 32 + lane;                     // this thread's row of the tile
    uint32_t waits0 = 0, waits1 = 0;                    // completions of bar_acc[i] waited for

    // wait for the MMAs committed to region reg (every epilogue thread), then
    // read TMEM; all epilogue threads agree on going on (a failed wait
    // anywhere stops them all at the same point)
    auto wait_acc = [&](int reg) -> bool {
      uint32_t &w = reg ? waits1 : waits0;
      const bool got = mbar_wait_suspend(&sh.bar_acc[reg], w & 1, lim);
      ++w;
      if (!got) give_up();
      if (!compute_sync_and(got && !aborted())) return false;
      tc_fence_after();
      return true;
    };
    // bias + ReLU of the hidden layer in region src, BF16 into H, one
    // 64-column chunk at a time (this warp's 32 of them), each chunk handed to
    // the MMA warp as soon as this warp has written it
    auto convert_chunk = [&](const uint32_t (&v)[32], const float *bias, int c) {
      const int j0 = 64 * c + 32 * half;
      uint32_t hb[16];
#pragma unroll
      for (int g8 = 0; g8 < 4; ++g8) {  // 16-byte aligned: bias12 and offsets of 4-float multiples
        const float4 b0 = *reinterpret_cast<const float4 *>(bias + j0 + 8 * g8);
        const float4 b1 = *reinterpret_cast<const float4 *>(bias + j0 + 8 * g8 + 4);
        const int e = 8 * g8;
        hb[4 * g8 + 0] = relu_bf16x2(add2(v[e + 0], v[e + 1], b0.x, b0.y));
        hb[4 * g8 + 1] = relu_bf16x2(add2(v[e + 2], v[e + 3], b0.z, b0.w));
        hb[4 * g8 + 2] = relu_bf16x2(add2(v[e + 4], v[e + 5], b1.x, b1.y));
        hb[4 * g8 + 3] = relu_bf16x2(add2(v[e + 6], v[e + 7], b1.z, b1.w));
      }
      uint8_t *chunk = H + c * kHChunk;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<uint4 *>(chunk + cm_off(r, 32 * half + 8 * u)) =
            make_uint4(hb[4 * u], hb[4 * u + 1], hb[4 * u + 2], hb[4 * u + 3]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.h_full[c]);
    };
    auto hidden_out = [&](int src, const float *bias) {
      const uint32_t base = tmem + trow + 256 * src + 32 * half;
      uint32_t va[32], vb[32];  // chunk c in va (c even) or vb (c odd); the next one in flight meanwhile
      tc_ld32_issue(base, va);
      tc_wait_ld32(va);
      tc_ld32_issue(base + 64, vb);
      convert_chunk(va, bias, 0);
      tc_wait_ld32(vb);
      tc_ld32_issue(base + 128, va);
      convert_chunk(vb, bias, 1);
      tc_wait_ld32(va);
      tc_ld32_issue(base + 192, vb);
      convert_chunk(va, bias, 2);
      tc_wait_ld32(vb);
      convert_chunk(vb, bias, 3);
    };

    for (int64_t it = 0, t = blockIdx.x; t < a.ntiles; ++it, t += gridDim.x) {
      const int R = (int)(it & 1);
      if (!wait_acc(R)) break;
      hidden_out(R, sh.bias12[0]);  // layer 1 out, layer 2 in
      if (!wait_acc(1 - R)) break;
      hidden_out(1 - R, sh.bias12[1]);  // layer 2 out, layer 3 in
      if (!wait_acc(R)) break;
      // output unit: this thread's 128 columns of layer 3, in four
      // interleaved partial sums (column j into sum j mod 4)
      unsigned long long acc2[2] = {0ull, 0ull};  // (sum 0, sum 1), (sum 2, sum 3)
      auto dot_part = [&](const uint32_t (&v)[32], int j0) {
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {  // 8 columns at a time: b3 and w4 are 16-byte aligned like the biases
          const float4 b0 = *reinterpret_cast<const float4 *>(sh.b3w4[0] + j0 + 8 * g8);
          const float4 b1 = *reinterpret_cast<const float4 *>(sh.b3w4[0] + j0 + 8 * g8 + 4);
          const float4 w0 = *reinterpret_cast<const float4 *>(sh.b3w4[1] + j0 + 8 * g8);
          const float4 w1 = *reinterpret_cast<const float4 *>(sh.b3w4[1] + j0 + 8 * g8 + 4);
          const float bf[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
          const float wf[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int e = 8 * g8 + 2 * i;
            float lo, hi;
            const unsigned long long sv = add2(v[e], v[e + 1], bf[2 * i], bf[2 * i + 1]);
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(sv));
            unsigned long long rv, wp;
            asm("mov.b64 %0, {%1, %2};" : "=l"(rv) : "f"(fmaxf(lo, 0.f)), "f"(fmaxf(hi, 0.f)));
            asm("mov.b64 %0, {%1, %2};" : "=l"(wp) : "f"(wf[2 * i]), "f"(wf[2 * i + 1]));
            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[i & 1]) : "l"(rv), "l"(wp));
          }
        }
      };
      {
        const uint32_t base = tmem + trow + 256 * R + half * 128;
        uint32_t va[32], vb[32];
        tc_ld32_issue(base, va);
        tc_wait_ld32(va);
        tc_ld32_issue(base + 32, vb);
        dot_part(va, half * 128);
        tc_wait_ld32(vb);
        tc_ld32_issue(base + 64, va);
        dot_part(vb, half * 128 + 32);
        tc_wait_ld32(va);
        tc_ld32_issue(base + 96, vb);
        dot_part(va, half * 128 + 64);
        tc_wait_ld32(vb);
        dot_part(vb, half * 128 + 96);
      }
      float s0, s1, s2, s3;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(s0), "=f"(s1) : "l"(acc2[0]));
      asm("mov.b64 {%0, %1}, %2;" : "=f"(s2), "=f"(s3) : "l"(acc2[1]));
      const float dot = (s0 + s1) + (s2 + s3);
      if (half) sh.half_dot[r] = dot;
      compute_sync();
      if (!half) {
        const int64_t row = t * kBM + r;
        const float o = (dot + sh.half_dot[r]) + *a.b4;
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
      // half_dot is rewritten only after the next tile's wait_acc barriers,
      // which warps 0-3 reach after reading it
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && sh.abort) atomicOr(a.err, kErrTimeout);
  if (warp == 0) tmem_dealloc(tmem, 512);
}

cudaError_t launch_mlp_fused(const ChainF &c, const MlpArgs &a0, uint8_t *wc, cudaStream_t s) {
  if (a0.n <= 0) return cudaSuccess;
  MlpArgs a = a0;
  a.ntiles = (a.n + kBM - 1) / kBM;
  a.wc = wc;
  mlp_prep_weights_kernel<<<(9 * kSurrW * 8 + 255) / 256, 256, 0, s>>>(a.w1, a.w2, a.w3, wc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = a.ntiles < sms ? a.ntiles : sms;
  mlp_fused_kernel<<<(unsigned)grid, kMlpThreads, kMlpSmem, s>>>(a, c);
  return cudaGetLastError();
}

size_t mlp_wc_bytes() { return 9 * (size_t)kWBlock; }

}  // namespace fk
