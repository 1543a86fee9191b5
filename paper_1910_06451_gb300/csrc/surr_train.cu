// One training step of the learned surrogate (not part of the paper) in a few
// launches, replayed from a CUDA graph:
//
//   surr_tile_kernel  persistent, one CTA of 256 threads per SM, over tiles of
//                     128 batch rows: the three forward layers and the two
//                     backward-delta products of every row run back to back
//                     on the tensor cores, the hidden tiles held in shared
//                     memory (BF16, the A-operand layout), the weights streamed
//                     through a three-slot ring; each epilogue also writes its
//                     tile transposed ([unit][batch row]) for the weight
//                     gradients, whose sums run over the batch;
//   gemm_tc_kernel    dW3 = d3^T h2, dW2 = d2^T h1, dW1 = d1^T x as split-K
//                     products with FP32 partials (three independent launches);
//   surr_reduce       the partials summed in split order, the bias gradients
//                     and the output unit's gradient as row sums over the
//                     batch, the batch loss;
//   surr_adam         Adam on the FP32 master weights, then their BF16 copies
//                     (row-major, and the weight blocks the tile kernel
//                     streams) for the next step;
//   surr_advance      the step counter.
//
// The batch, the learning rate and Adam's step count come from a step counter
// in device memory, so every step launches the same graph.  The rounding
// points are those of the layer-by-layer definition: features, h1, h2 and
// every delta stored in BF16; h3 in FP32 for the output and in BF16 for the
// w4 gradient; all sums in FP32, every reduction in a fixed order.
#include <cmath>

#include "surr_step.h"

namespace fk {

constexpr int kTrThreads = 256;  // two warps per TMEM lane quadrant, each half the columns
constexpr uint32_t kTrH = kBM * kSurrW * 2;      // 64 KB: a hidden tile (4 K chunks)
constexpr uint32_t kTrChunk = kBM * kBK * 2;     // 16 KB: one K chunk of a hidden tile
constexpr uint32_t kTrW = kSurrW * kBK * 2;      // 32 KB: 256 weight rows x 64 K
constexpr int kTrSlots = 3;                      // weight ring
constexpr uint32_t kTrSmem = 2 * kTrH + kTrSlots * kTrW;  // 224 KB
constexpr uint32_t kTrIdesc = idesc_bf16_f32(kBM, kSurrW);
// Weight blocks of one tile, in the order the tile's MMAs read them: W1, the
// four K chunks of W2, of W3, of W3^T (B operand of d3 W3) and of W2^T.
constexpr int kTrBlocks = 17;

// core-matrix offset of element (row, k) of a [rows][64] K-major tile
__device__ __forceinline__ uint32_t tr_cm(int row, int k) {
  return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Weight ring, fed by 1-D TMA bulk copies of the pre-laid-out 32 KB blocks
// (surr_wc_off): chunk g of the CTA's sequence (block g mod 17) goes to slot
// g mod 3, announced on full[slot]; its MMAs commit to done[slot].  Both
// barriers complete their (g / 3)-th phase for chunk g.  Thread 0 keeps the
// copies two chunks ahead of the MMAs, refilling a slot once the MMAs of its
// previous chunk have committed.
struct TrRing {
  uint8_t *base;
  uint64_t *full, *done;
  const uint8_t *wc;
  uint32_t next_load;  // thread 0: next chunk to copy
  uint32_t next_mma;   // next chunk to multiply (every thread)
  uint32_t end;        // chunks of this CTA (tiles x 17)
  uint32_t issued;     // thread 0: chunks whose MMAs have been committed
};

// thread 0: copies up to chunk `upto` (bounded by the CTA's chunk count);
// false if a wait for a slot gave up
__device__ __forceinline__ bool tr_fill(TrRing &r, uint32_t upto, uint32_t limit) {
  for (; r.next_load <= upto && r.next_load < r.end; ++r.next_load) {
    const uint32_t gl = r.next_load, s = gl % kTrSlots;
    if (gl >= kTrSlots && !mbar_wait_bounded(&r.done[s], ((gl - kTrSlots) / kTrSlots) & 1, limit)) return false;
    mbar_arrive_expect_tx(&r.full[s], kTrW);
    tma_bulk_load(r.base + s * kTrW, r.wc + (size_t)(gl % kTrBlocks) * kTrW, kTrW, &r.full[s]);
  }
  return true;
}

// The MMAs of one layer: A = nk K chunks of [128][64] at a_base + c 16 KB
// (shared memory) times the next nk weight chunks of the ring, into tmem
// (cols 0..255).  Returns once the last commit has landed, or false in every
// thread if a wait gave up (*abort is then set).
__device__ __forceinline__ bool tr_layer(TrRing &r, uint32_t a_base, int nk, uint32_t tmem, uint32_t limit,
                                         int *abort) {
  const int tid = threadIdx.x;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A written by the generic proxy
  __syncthreads();
  if (tid == 0 && !*abort) {
    tc_fence_after();
    for (int c = 0; c < nk; ++c) {
      const uint32_t gc = r.next_mma + c, s = gc % kTrSlots;
      if (!mbar_wait_bounded(&r.full[s], (gc / kTrSlots) & 1, limit)) {
        *abort = 1;
        break;
      }
      const uint32_t b_base = smem_u32(r.base + s * kTrW), a_c = a_base + c * kTrChunk;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        tc_mma(tmem, smem_desc(a_c + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024), kTrIdesc,
               (c > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&r.done[s]);
      r.issued = gc + 1;
      if (!tr_fill(r, gc + 2, limit)) {
        *abort = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (*abort) return false;
  r.next_mma += nk;
  const uint32_t gl = r.next_mma - 1;
  const bool got = mbar_wait_bounded(&r.done[gl % kTrSlots], (gl / kTrSlots) & 1, limit);
  if (!__syncthreads_and(got)) {
    if (tid == 0) *abort = 1;
    return false;
  }
  tc_fence_after();
  return true;
}

// 16-byte store of 8 BF16 values into a hidden tile at (row, k), k % 8 == 0
__device__ __forceinline__ void tr_put8(uint8_t *H, int row, int k, const bf16 *v) {
  *reinterpret_cast<uint4 *>(H + (k >> 6) * kTrChunk + tr_cm(row, k & 63)) = *reinterpret_cast<const uint4 *>(v);
}

// Byte offset in the weight blocks of entry (o, i) of W1 (layer 0), W2 (1)
// or W3 (2) (o the output unit, i the input): the B operand of layer L + 1
// has row n = o and K index k = i; W2 and W3 appear a second time
// transposed (B operands of the deltas: d3 W3 and d2 W2), row n = i, k = o.
// Within a 32 KB block (256 rows x 64 K) the no-swizzle core-matrix layout
// of the ring.
// 32 consecutive FP32 biases (16-byte aligned) as eight vector loads
__device__ __forceinline__ void tr_bias32(const float *__restrict__ b, float (&o)[32]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(b) + k);
    o[4 * k] = t.x;
    o[4 * k + 1] = t.y;
    o[4 * k + 2] = t.z;
    o[4 * k + 3] = t.w;
  }
}
__device__ __forceinline__ uint32_t surr_wc_off(int block, int n, int k) {
  return (uint32_t)block * kTrW + (uint32_t)(((n >> 3) * 8 + ((k & 63) >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ void surr_wc_put(uint8_t *wc, int layer, int o, int i, bf16 v) {
  if (layer == 0) {
    *reinterpret_cast<bf16 *>(wc + surr_wc_off(0, o, i)) = v;
    return;
  }
  const int first = layer == 1 ? 1 : 5, firstT = layer == 1 ? 13 : 9;
  *reinterpret_cast<bf16 *>(wc + surr_wc_off(first + i / kBK, o, i)) = v;
  *reinterpret_cast<bf16 *>(wc + surr_wc_off(firstT + o / kBK, i, o)) = v;
}

// The weight blocks from the BF16 weights ([out][in] row-major).
__global__ void surr_wc_kernel(const bf16 *__restrict__ w1, const bf16 *__restrict__ w2, const bf16 *__restrict__ w3,
                               uint8_t *__restrict__ wc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n1 = kSurrW * kSurrIn, n2 = kSurrW * kSurrW;
  if (e < n1)
    surr_wc_put(wc, 0, e / kSurrIn, e % kSurrIn, w1[e]);
  else if (e < n1 + n2)
    surr_wc_put(wc, 1, (e - n1) / kSurrW, (e - n1) % kSurrW, w2[e - n1]);
  else if (e < n1 + 2 * n2)
    surr_wc_put(wc, 2, (e - n1 - n2) / kSurrW, (e - n1 - n2) % kSurrW, w3[e - n1 - n2]);
}

__global__ void __launch_bounds__(kTrThreads, 1) surr_tile_kernel(const SurrStepArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t full[kTrSlots], done[kTrSlots];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float sw4[kSurrW];  // b1, b2, b3 are read as vectors through L1 (shared memory is full)
  __shared__ float sout[2][kBM];               // the two halves of each row's output dot product
  uint8_t *HA = sm, *HB = sm + kTrH;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntiles = a.B / kBM;
  const int mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // tiles of this CTA
  TrRing r{sm + 2 * kTrH, full, done, a.wc, 0, 0, (uint32_t)mine * kTrBlocks, 0};
  if (warp == 0) {
    tmem_alloc(&tmem_slot, kSurrW);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kTrSlots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&done[i], 1);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < kSurrW; i += kTrThreads) sw4[i] = a.w4[i];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && !tr_fill(r, 2, a.wait_limit)) abort_flag = 1;  // the first three chunks
  const uint32_t tmem = tmem_slot;
  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (tile rows) and the columns
  // of half w / 4 (128 each)
  const int lane = tid & 31, quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane, c0 = half * (kSurrW / 2);
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
  const int64_t B = a.B;
  const int64_t row0 = (*a.step % a.steps_per_epoch) * B;   // the batch's first training row
  const float b4 = *a.b4;
  const float invB2 = 2.f / (float)a.B;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t rb = (int64_t)tile * kBM + row;  // this thread's row within the batch
    // features of the tile into HB (A layout, one K chunk), each thread half
    // of its row; and transposed to global
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.X + (row0 + rb) * kSurrIn);
#pragma unroll
      for (int i = half * 4; i < half * 4 + 4; ++i) {
        uint4 u = src[i];
        *reinterpret_cast<uint4 *>(HB + tr_cm(row, 8 * i)) = u;
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) a.xT[(int64_t)(8 * i + j) * B + rb] = e[j];
      }
    }

    uint32_t m1[4], m2[4], m3[4];  // ReLU masks of h1, h2, h3 on this thread's 128 units, one bit each
    // ---- layer 1: h1 = relu(x W1^T + b1) -> HA, h1T
    if (!tr_layer(r, smem_u32(HB), 1, tmem, a.wait_limit, &abort_flag)) break;
    // a hidden layer's epilogue: each 32-column chunk's biases are loaded as
    // vectors before its TMEM wait, and the next chunk's TMEM load is in flight
    // while this one is converted and stored
    auto hidden = [&](const float *__restrict__ bias, uint8_t *H, bf16 *__restrict__ hT, uint32_t (&m)[4]) {
      uint32_t v[32];
      tc_ld32_issue(trow + c0, v);
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        const int j0 = c0 + 32 * j;
        float x[32];
        tr_bias32(bias + j0, x);
        tc_wait_ld32(v);
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] += __uint_as_float(v[i]);
        if (j < 3) tc_ld32_issue(trow + j0 + 32, v);
        __align__(16) bf16 hb[32];
        uint32_t bits = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          hb[i] = __float2bfloat16_rn(fmaxf(x[i], 0.f));
          bits |= (uint32_t)(__bfloat162float(hb[i]) > 0.f) << i;
          hT[(int64_t)(j0 + i) * B + rb] = hb[i];
        }
        m[j] = bits;
#pragma unroll
        for (int i = 0; i < 32; i += 8) tr_put8(H, row, j0 + i, hb + i);
      }
      tc_fence_before();
    };
    hidden(a.b1, HA, a.h1T, m1);
    // ---- layer 2: h2 = relu(h1 W2^T + b2) -> HB, h2T
    if (!tr_layer(r, smem_u32(HA), 4, tmem, a.wait_limit, &abort_flag)) break;
    hidden(a.b2, HB, a.h2T, m2);
    // ---- layer 3 and the output unit: out = relu(z3) . w4 + b4 (FP32),
    // dout = 2 (out - y) / B, d3 = bf16(dout w4 [z3 > 0]) -> HA, d3T; h3T
    if (!tr_layer(r, smem_u32(HB), 4, tmem, a.wait_limit, &abort_flag)) break;
    float out = 0.f;
    const float y = a.Y[row0 + rb];
    {
      uint32_t v[32];
      tc_ld32_issue(trow + c0, v);
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        const int j0 = c0 + 32 * j;
        float x[32];
        tr_bias32(a.b3 + j0, x);
        tc_wait_ld32(v);
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] += __uint_as_float(v[i]);
        if (j < 3) tc_ld32_issue(trow + j0 + 32, v);
        uint32_t bits = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float h = fmaxf(x[i], 0.f);
          out = fmaf(h, sw4[j0 + i], out);
          const bf16 hb = __float2bfloat16_rn(h);
          bits |= (uint32_t)(__bfloat162float(hb) > 0.f) << i;
          a.h3T[(int64_t)(j0 + i) * B + rb] = hb;
        }
        m3[j] = bits;
      }
    }
    tc_fence_before();
    // the row's two halves of the dot product, added in a fixed order
    sout[half][row] = out;
    __syncthreads();
    out = (sout[0][row] + sout[1][row]) + b4;
    const float e = out - y;
    const float dout = e * invB2;
    if (half == 0) {
      a.dout[rb] = dout;
      a.lrow[rb] = e * e;
    }
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      const int j0 = c0 + 32 * j;
      __align__(16) bf16 db[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        db[i] = __float2bfloat16_rn(((m3[j] >> i) & 1u) ? dout * sw4[j0 + i] : 0.f);
        a.d3T[(int64_t)(j0 + i) * B + rb] = db[i];
      }
#pragma unroll
      for (int i = 0; i < 32; i += 8) tr_put8(HA, row, j0 + i, db + i);
    }
    // ---- back through layer 3 and 2: d = bf16((d W) [h > 0])
    auto delta = [&](uint8_t *H, bf16 *__restrict__ dT, const uint32_t (&m)[4]) {
      uint32_t v[32];
      tc_ld32_issue(trow + c0, v);
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        const int j0 = c0 + 32 * j;
        tc_wait_ld32(v);
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(v[i]);
        if (j < 3) tc_ld32_issue(trow + j0 + 32, v);
        __align__(16) bf16 db[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          db[i] = __float2bfloat16_rn(((m[j] >> i) & 1u) ? x[i] : 0.f);
          dT[(int64_t)(j0 + i) * B + rb] = db[i];
        }
        if (H) {
#pragma unroll
          for (int i = 0; i < 32; i += 8) tr_put8(H, row, j0 + i, db + i);
        }
      }
      tc_fence_before();
    };
    if (!tr_layer(r, smem_u32(HA), 4, tmem, a.wait_limit, &abort_flag)) break;
    delta(HB, a.d2T, m2);
    if (!tr_layer(r, smem_u32(HB), 4, tmem, a.wait_limit, &abort_flag)) break;
    delta(nullptr, a.d1T, m1);
  }
  __syncthreads();
  if (abort_flag && tid == 0) {
    // let the copies and MMAs already issued land (bounded) before the
    // shared and tensor memory are released, and report
    for (uint32_t gl = r.issued; gl < r.next_load; ++gl)  // copies not yet consumed
      mbar_wait_bounded(&r.full[gl % kTrSlots], (gl / kTrSlots) & 1, kGemmDrain);
    if (r.issued > 0)  // the last commit lands after every earlier MMA
      mbar_wait_bounded(&r.done[(r.issued - 1) % kTrSlots], ((r.issued - 1) / kTrSlots) & 1, kGemmDrain);
    atomicOr(a.err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kSurrW);
}

// ------------------------------------------------------------ reduction --
// The step's gradient G (flat parameter order W1, b1, W2, b2, W3, b3, w4, b4)
// and loss: weight entries as the sum of their split-K partials in split
// order (one thread each); biases, w4 and b4 as sums over the batch rows of
// dT[u][.], h3T[u][.] dout[.] and dout[.] (one block each, threads over the
// rows, a fixed-order reduction); the loss (mean of lrow) into loss_hist[step].
constexpr int64_t kTrOffW1 = 0, kTrOffB1 = kTrOffW1 + (int64_t)kSurrW * kSurrIn, kTrOffW2 = kTrOffB1 + kSurrW,
                  kTrOffB2 = kTrOffW2 + (int64_t)kSurrW * kSurrW, kTrOffW3 = kTrOffB2 + kSurrW,
                  kTrOffB3 = kTrOffW3 + (int64_t)kSurrW * kSurrW, kTrOffW4 = kTrOffB3 + kSurrW,
                  kTrOffB4 = kTrOffW4 + kSurrW, kTrParams = kTrOffB4 + 1;
constexpr int kRedThreads = 256;
constexpr int64_t kRedW = (int64_t)kSurrW * kSurrIn + 2 * (int64_t)kSurrW * kSurrW;  // weight entries
constexpr int kRedWBlocks = (int)((kRedW + kRedThreads - 1) / kRedThreads);
constexpr int kRedRows = 4 * kSurrW + 2;  // b1, b2, b3, w4 rows; b4; loss
constexpr int kRedRowBlocks = kRedRows;

__global__ void __launch_bounds__(kRedThreads) surr_reduce_kernel(const SurrReduceArgs a) {
  if (blockIdx.x < kRedWBlocks) {
    const int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
    if (i >= kRedW) return;
    const float *src;
    int64_t j, n, dst;
    if (i < (int64_t)kSurrW * kSurrIn) {
      src = a.p1, j = i, n = (int64_t)kSurrW * kSurrIn, dst = kTrOffW1 + i;
    } else if (i < (int64_t)kSurrW * kSurrIn + (int64_t)kSurrW * kSurrW) {
      j = i - (int64_t)kSurrW * kSurrIn, src = a.p2, n = (int64_t)kSurrW * kSurrW, dst = kTrOffW2 + j;
    } else {
      j = i - (int64_t)kSurrW * kSurrIn - (int64_t)kSurrW * kSurrW, src = a.p3, n = (int64_t)kSurrW * kSurrW,
      dst = kTrOffW3 + j;
    }
    float s = 0.f;
    for (int z = 0; z < a.splits; ++z) s += src[(int64_t)z * n + j];
    a.G[dst] = s;
    return;
  }
  // one block per row sum: lanes over the batch rows, a fixed-order reduction
  const int row = blockIdx.x - kRedWBlocks;
  if (row >= kRedRows) return;
  const int t = threadIdx.x;
  float s = 0.f;
  if (row < 3 * kSurrW) {  // b1, b2, b3: sum over the batch of the layer's delta
    const int layer = row / kSurrW, u = row % kSurrW;
    const bf16 *dT = layer == 0 ? a.d1T : (layer == 1 ? a.d2T : a.d3T);
    const uint4 *src = reinterpret_cast<const uint4 *>(dT + (int64_t)u * a.B);
    for (int c = t; c < a.B / 8; c += kRedThreads) {
      uint4 v = src[c];
      const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int k = 0; k < 8; ++k) s += __bfloat162float(e[k]);
    }
  } else if (row < 4 * kSurrW) {  // w4: sum over the batch of h3 dout
    const int u = row - 3 * kSurrW;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.h3T + (int64_t)u * a.B);
    for (int c = t; c < a.B / 8; c += kRedThreads) {
      uint4 v = src[c];
      const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int k = 0; k < 8; ++k) s = fmaf(__bfloat162float(e[k]), a.dout[8 * c + k], s);
    }
  } else {  // b4, loss
    const float *src = row == 4 * kSurrW ? a.dout : a.lrow;
    for (int c = t; c < a.B; c += kRedThreads) s += src[c];
  }
  __shared__ float part[kRedThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((t & 31) == 0) part[t >> 5] = s;
  __syncthreads();
  if (t != 0) return;
  s = 0.f;
  for (int w = 0; w < kRedThreads / 32; ++w) s += part[w];
  if (row < 3 * kSurrW) {
    const int layer = row / kSurrW, u = row % kSurrW;
    a.G[(layer == 0 ? kTrOffB1 : (layer == 1 ? kTrOffB2 : kTrOffB3)) + u] = s;
  } else if (row < 4 * kSurrW) {
    a.G[kTrOffW4 + row - 3 * kSurrW] = s;
  } else if (row == 4 * kSurrW) {
    a.G[kTrOffB4] = s;
  } else if (a.loss_hist) {
    a.loss_hist[*a.step] = s / (float)a.B;
  }
}

// -------------------------------------------------------------- update ---
// Adam (beta1 0.9, beta2 0.999, eps 1e-8) with the step's learning rate and
// bias correction from the device counter, then the BF16 copies of W1, W2,
// W3 ([out][in]) and of the transposes of W2 and W3 ([in][out]).
__global__ void __launch_bounds__(256) surr_adam_kernel(const SurrAdamArgs a) {
  // the step's learning rate and bias corrections, once per block (the
  // cosine in FP64 would occupy the narrow FP64 pipe in every thread)
  __shared__ float s_lr, s_c1, s_c2;
  if (threadIdx.x == 0) {
    const int64_t st = *a.step;
    if (a.cosine) {
      s_lr = (float)(0.5 * (double)a.lr * (1.0 + cos(M_PI * (double)st / (double)a.total)));
    } else {
      const int64_t ep = st / a.steps_per_epoch;
      s_lr = ep < (2 * a.epochs + 2) / 3 ? a.lr : a.lr / 3.f;
    }
    const int64_t t = a.t0 + st + 1;
    s_c1 = 1.f - powf(0.9f, (float)t);
    s_c2 = 1.f - powf(0.999f, (float)t);
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTrParams) return;
  const float lr = s_lr, c1 = s_c1, c2 = s_c2;
  const float gi = a.G[i];
  const float mi = 0.9f * a.m[i] + 0.1f * gi;
  const float vi = 0.999f * a.v[i] + 0.001f * gi * gi;
  a.m[i] = mi;
  a.v[i] = vi;
  const float pi = a.p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  a.p[i] = pi;
  const bf16 h = __float2bfloat16_rn(pi);
  if (i < kTrOffB1) {
    a.w1[i] = h;
    surr_wc_put(a.wc, 0, (int)(i / kSurrIn), (int)(i % kSurrIn), h);
  } else if (i >= kTrOffW2 && i < kTrOffB2) {
    const int64_t j = i - kTrOffW2;
    a.w2[j] = h;
    surr_wc_put(a.wc, 1, (int)(j / kSurrW), (int)(j % kSurrW), h);
  } else if (i >= kTrOffW3 && i < kTrOffB3) {
    const int64_t j = i - kTrOffW3;
    a.w3[j] = h;
    surr_wc_put(a.wc, 2, (int)(j / kSurrW), (int)(j % kSurrW), h);
  }
}

__global__ void surr_advance_kernel(int64_t *step) { *step += 1; }

// ------------------------------------------------------------ launchers --
static_assert(kTrSmem + kSurrW * sizeof(float) + 2 * kBM * sizeof(float) + 128 <= 232448, "tile kernel above 227 KB of shared memory");

cudaError_t launch_surr_tile(const SurrStepArgs &a, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(surr_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrSmem);
  if (e != cudaSuccess) return e;
  const int ntiles = a.B / kBM;
  surr_tile_kernel<<<(unsigned)(ntiles < sms ? ntiles : sms), kTrThreads, kTrSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_surr_reduce(const SurrReduceArgs &a, cudaStream_t s) {
  surr_reduce_kernel<<<kRedWBlocks + kRedRowBlocks, kRedThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_surr_adam(const SurrAdamArgs &a, cudaStream_t s) {
  surr_adam_kernel<<<(unsigned)((kTrParams + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_surr_wc(const bf16 *w1, const bf16 *w2, const bf16 *w3, uint8_t *wc, cudaStream_t s) {
  constexpr int n = kSurrW * kSurrIn + 2 * kSurrW * kSurrW;
  surr_wc_kernel<<<(n + 255) / 256, 256, 0, s>>>(w1, w2, w3, wc);
  return cudaGetLastError();
}

cudaError_t launch_surr_advance(int64_t *step, cudaStream_t s) {
  surr_advance_kernel<<<1, 1, 0, s>>>(step);
  return cudaGetLastError();
}

}  // namespace fk
