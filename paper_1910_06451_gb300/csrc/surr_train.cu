// One training step of the learned surrogate (not part of the paper) in three
// launches, replayed from a CUDA graph:
//
//   surr_tile_kernel  persistent, clusters of two CTAs (256 threads each), one
//                     cluster per tile of 128 batch rows: the three forward
//                     layers and the two backward-delta products run back to
//                     back on the tensor cores, each CTA computing half of every
//                     layer's 256 output units (its half of the weights streamed
//                     through a six-slot ring) and sending its half of each
//                     hidden or delta tile into its peer's shared memory (the
//                     A operand of the next layer needs all 256 units).  While
//                     a layer's MMAs run, the CTA writes its half of the
//                     layer's input tile transposed for the weight gradients
//                     and sums it over the tile's rows for the bias gradients;
//   surr_dw_kernel    dW3 = d3^T h2, dW2 = d2^T h1, dW1 = d1^T x as split-K
//                     products with FP32 partials, all three in one launch;
//   surr_adam_kernel  the partials summed in split order and the tile sums in
//                     tile order, Adam on the FP32 master weights, their BF16
//                     copies (row-major, and the weight blocks the tile kernel
//                     streams) for the next step, the step counter.
//
// The batch, the learning rate and Adam's step count come from a step counter
// in device memory, so every step launches the same graph.  The rounding
// points are those of the layer-by-layer definition: features, h1, h2 and
// every delta stored in BF16; h3 in FP32 for the output and in BF16 for the
// w4 gradient; all sums in FP32, every reduction in a fixed order.
#include <cmath>

#include "surr_step.h"

namespace fk {

constexpr int kTrThreads = 256;  // two warps per TMEM lane quadrant, each half the CTA's columns
constexpr int kTrN = kSurrW / 2;   // output units of one CTA (one half of each layer)
constexpr uint32_t kTrH = kBM * kSurrW * 2;      // 64 KB: a hidden tile (4 K chunks)
constexpr uint32_t kTrChunk = kBM * kBK * 2;     // 16 KB: one K chunk of a hidden tile
constexpr uint32_t kTrW = kSurrW * kBK * 2;      // 32 KB: a weight block, 256 rows x 64 K
constexpr uint32_t kTrHalfW = kTrN * kBK * 2;    // 16 KB: the CTA's 128 rows of a block
constexpr int kTrSlots = 6;                      // weight ring: more than one layer's chunks
constexpr uint32_t kTrSmem = 2 * kTrH + kTrSlots * kTrHalfW;  // 224 KB
constexpr uint32_t kTrIdesc = idesc_bf16_f32(kBM, kTrN);
// Weight blocks of one tile, in the order the tile's MMAs read them: W1, the
// four K chunks of W2, of W3, of W3^T (B operand of d3 W3) and of W2^T.
constexpr int kTrBlocks = 17;

// core-matrix offset of element (row, k) of a [rows][64] K-major tile
__device__ __forceinline__ uint32_t tr_cm(int row, int k) {
  return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Weight ring, fed by 1-D TMA bulk copies of the CTA's half (rows 128 rank ..
// + 127, 16 KB contiguous) of the pre-laid-out 32 KB blocks (surr_wc_off):
// chunk g of the CTA's sequence (block g mod 17) goes to slot g mod 6,
// announced on full[slot]; its MMAs commit to done[slot].  Both barriers
// complete their (g / 6)-th phase for chunk g.  Thread 0 refills a slot once
// the MMAs of its previous chunk have committed.
struct TrRing {
  uint8_t *base;
  uint64_t *full, *done;
  const uint8_t *wc;   // the blocks, offset to this CTA's half
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
    mbar_arrive_expect_tx(&r.full[s], kTrHalfW);
    tma_bulk_load(r.base + s * kTrHalfW, r.wc + (size_t)(gl % kTrBlocks) * kTrW, kTrHalfW, &r.full[s]);
  }
  return true;
}

// Bounded wait with acquire semantics at cluster scope (a phase completed by
// the peer CTA's arrivals).
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_test_wait_cluster(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

// The exchange between the two CTAs of a tile.  Exchange k of a CTA's
// sequence (five per tile: h1, h2, the output unit's partial sums, d3, d2)
// completes phase k / 2 of the peer's barrier xin[k mod 2]: every warp of the
// sender, once its lanes' stores into the peer's shared memory are done,
// makes them visible to the peer's tensor-core reads (proxy fence) and
// arrives with release semantics; the receiver waits with acquire semantics.
// A CTA sends exchange k + 1 only after it has received exchange k, so a
// barrier is never more than one phase ahead of its waiter.
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void tr_xsend(uint32_t peer_bar) {
  asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
  __syncwarp();
  if ((threadIdx.x & 31) == 0)
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(peer_bar) : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The MMAs of one layer, in two halves so that the CTA can work between
// them: tr_issue (every thread; after the barrier thread 0 issues) multiplies
// A = nk K chunks of [128][64] at a_base + c 16 KB (shared memory) by the next
// nk weight chunks of the ring into tmem (cols 0..127), waiting first (if xbar
// is given) for the exchange that completes A, then refills the ring up to a
// full slot count past the layer; tr_wait returns once the last commit has
// landed, or false in every thread if a wait gave up (*abort is then set).
// Between the two the A tiles may be read, not written.
__device__ __forceinline__ void tr_issue(TrRing &r, uint32_t a_base, int nk, uint32_t tmem, uint32_t limit,
                                         int *abort, uint64_t *xbar, uint32_t xpar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A written by the generic proxy
  __syncthreads();
  if (threadIdx.x == 0 && !*abort) {
    if (xbar && !mbar_wait_cluster_bounded(xbar, xpar, limit)) {
      *abort = 1;
      return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_after();
    for (int c = 0; c < nk; ++c) {
      const uint32_t gc = r.next_mma + c, s = gc % kTrSlots;
      if (!mbar_wait_bounded(&r.full[s], (gc / kTrSlots) & 1, limit)) {
        *abort = 1;
        return;
      }
      const uint32_t b_base = smem_u32(r.base + s * kTrHalfW), a_c = a_base + c * kTrChunk;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        tc_mma(tmem, smem_desc(a_c + kk * 256, 128, 1024), smem_desc(b_base + kk * 256, 128, 1024), kTrIdesc,
               (c > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&r.done[s]);
      r.issued = gc + 1;
    }
    if (!tr_fill(r, r.next_mma + nk - 1 + kTrSlots, limit)) *abort = 1;
  }
}
__device__ __forceinline__ bool tr_wait(TrRing &r, int nk, uint32_t limit, int *abort) {
  __syncthreads();  // thread 0's issue, and *abort, before anyone reads them
  if (*abort) return false;
  r.next_mma += nk;
  const uint32_t gl = r.next_mma - 1;
  const bool got = mbar_wait_bounded(&r.done[gl % kTrSlots], (gl / kTrSlots) & 1, limit);
  if (!__syncthreads_and(got)) {
    if (threadIdx.x == 0) *abort = 1;
    return false;
  }
  tc_fence_after();
  return true;
}

// Programmatic dependent launch: the three kernels of a step (and the next
// step's first) are launched so that a kernel's CTAs may start while its
// predecessor drains.  Each kernel sets up its shared and tensor memory, then
// waits for the predecessor's completion (and memory) before it touches
// global memory, then lets its own dependents launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Four 8x8 BF16 core matrices, transposed: lanes 8i..8i+7 address the eight
// 16-byte lines of matrix i; lane t receives, of each matrix, lines
// 2 (t mod 4) and 2 (t mod 4) + 1 at element t / 4 (low and high half).
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// Unit groups ug0 .. ug0 + nug - 1 (8 units each) of a tile of 128 rows x U
// units held in shared memory (the A-operand layout of tr_put8) written
// transposed into the chunk-blocked tensor T (rows tile 128 ..), and/or their
// column sums (weighted by w[row] if w is given) into sums[u].  A core matrix
// of the tile (8 rows x 8 units) transposed is a core matrix of T (8 units x
// 8 rows): one ldmatrix reads four row groups of one unit group, each lane
// then holds two rows of one unit per matrix and the warp's store of one
// matrix is 128 contiguous bytes.  Warps 1-7 share the unit groups (warp 0
// holds the thread that issues the MMAs and keeps the weight ring full); the
// sums add, per unit, the tile's rows in a fixed order.
template <int U, bool STORE, bool SUM>
__device__ __forceinline__ void tr_copy_t(const uint8_t *H, bf16 *T, int tile, float *sums, const float *w,
                                          int ug0, int nug) {
  constexpr int kCopyWarps = kTrThreads / 32 - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) return;
  const uint32_t hs = smem_u32(H);
#pragma unroll 1
  for (int ug = ug0 + warp - 1; ug < ug0 + nug; ug += kCopyWarps) {
    float acc = 0.f;
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) {  // a quarter of the row groups
      uint32_t v[4];
      ldsm_x4_trans(hs + (uint32_t)(ug >> 3) * kTrChunk + (uint32_t)(((rq * 4 + (lane >> 3)) * 8 + (ug & 7)) * 128) +
                        (uint32_t)(lane & 7) * 16,
                    v);
      if (STORE) {
        // row groups rq 4 + i of the tile: chunk 2 tile + rq / 2, core row (rq mod 2) 4 + i
        uint8_t *dst = reinterpret_cast<uint8_t *>(T) + ((size_t)tile * 2 + (rq >> 1)) * U * 128 +
                       (size_t)(ug * 8 + (rq & 1) * 4) * 128 + lane * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) *reinterpret_cast<uint32_t *>(dst + i * 128) = v[i];
      }
      if (SUM) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float lo = __uint_as_float(v[i] << 16), hi = __uint_as_float(v[i] & 0xffff0000u);
          if (w) {
            const int r0 = (rq * 4 + i) * 8 + 2 * (lane & 3);
            acc = fmaf(lo, w[r0], acc);
            acc = fmaf(hi, w[r0 + 1], acc);
          } else {
            acc += lo;
            acc += hi;
          }
        }
      }
    }
    if (SUM) {  // the unit group's 128 rows: add the four lanes of each unit
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if ((lane & 3) == 0) sums[ug * 8 + (lane >> 2)] = acc;
    }
  }
}

// 16-byte store of 8 BF16 values into a hidden tile at (row, k), k % 8 == 0,
// and (with peer, the tile's address in the peer CTA) the same store there
__device__ __forceinline__ uint32_t tr_off(int row, int k) { return (k >> 6) * kTrChunk + tr_cm(row, k & 63); }
__device__ __forceinline__ void tr_put8(uint8_t *H, int row, int k, const bf16 *v) {
  *reinterpret_cast<uint4 *>(H + tr_off(row, k)) = *reinterpret_cast<const uint4 *>(v);
}
__device__ __forceinline__ void tr_put8x(uint8_t *H, uint32_t peer, int row, int k, const bf16 *v) {
  const uint32_t o = tr_off(row, k);
  const uint4 q = *reinterpret_cast<const uint4 *>(v);
  *reinterpret_cast<uint4 *>(H + o) = q;
  st_cluster_v4(peer + o, q);
}

// 32 FP32 values to BF16 (two per conversion) and their mask: bit i set iff
// the rounded value i is non-zero (the values are >= 0 or exactly +0, so this
// is bf16(v) > 0, the ReLU mask of the stored activation)
__device__ __forceinline__ uint32_t tr_bf16x32(const float (&v)[32], bf16 (&o)[32]) {
  uint32_t bits = 0;
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[i], v[i + 1]);
    const uint32_t u = *reinterpret_cast<const uint32_t *>(&h);
    *reinterpret_cast<uint32_t *>(&o[i]) = u;
    bits |= (uint32_t)((u & 0xffffu) != 0u) << i;
    bits |= (uint32_t)((u >> 16) != 0u) << (i + 1);
  }
  return bits;
}

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

// Byte offset in the weight blocks of entry (o, i) of W1 (layer 0), W2 (1)
// or W3 (2) (o the output unit, i the input): the B operand of layer L + 1
// has row n = o and K index k = i; W2 and W3 appear a second time
// transposed (B operands of the deltas: d3 W3 and d2 W2), row n = i, k = o.
// Within a 32 KB block (256 rows x 64 K) the no-swizzle core-matrix layout
// of the ring.
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

// Entries (o, i .. i + 3) of one layer, i % 4 == 0: the four inputs are
// adjacent in the forward block (one 8-byte store), four rows apart in the
// transposed one.
__device__ __forceinline__ void surr_wc_put4(uint8_t *wc, int layer, int o, int i, const bf16 (&v)[4]) {
  const int first = layer == 0 ? 0 : (layer == 1 ? 1 : 5);
  *reinterpret_cast<uint2 *>(wc + surr_wc_off(first + i / kBK, o, i)) = *reinterpret_cast<const uint2 *>(v);
  if (layer == 0) return;
  const int firstT = layer == 1 ? 13 : 9;
#pragma unroll
  for (int q = 0; q < 4; ++q) *reinterpret_cast<bf16 *>(wc + surr_wc_off(firstT + o / kBK, i + q, o)) = v[q];
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
  __shared__ __align__(8) uint64_t full[kTrSlots], done[kTrSlots], xin[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float sw4[kTrN];     // w4 of this CTA's units; b1, b2, b3 are read as vectors through L1
  __shared__ float sout[2][kBM];  // the two column halves of this CTA's part of each row's output; then dout, e^2
  __shared__ float sx[2][kBM];    // the two CTAs' parts of each row's output dot product
  uint8_t *HA = sm, *HB = sm + kTrH;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank(), peer = rank ^ 1u;
  const int ntiles = a.B / kBM, cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int mine = cl < ntiles ? (ntiles - 1 - cl) / ncl + 1 : 0;  // tiles of this cluster
  TrRing r{sm + 2 * kTrH, full, done, a.wc + rank * kTrHalfW, 0, 0, (uint32_t)mine * kTrBlocks, 0};
  if (warp == 0) {
    tmem_alloc(&tmem_slot, kTrN);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kTrSlots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&done[i], 1);
    }
    mbar_init(&xin[0], kTrThreads / 32);
    mbar_init(&xin[1], kTrThreads / 32);
    abort_flag = 0;
    mbar_fence_init_cluster();
  }
  tc_fence_before();
  cluster_sync_all();  // both CTAs' barriers initialised before any exchange
  tc_fence_after();
  pdl_wait();
  pdl_trigger();
  for (int i = tid; i < kTrN; i += kTrThreads) sw4[i] = a.w4[rank * kTrN + i];
  if (tid == 0 && !tr_fill(r, kTrSlots - 1, a.wait_limit)) abort_flag = 1;  // the ring's first chunks
  const uint32_t tmem = tmem_slot;
  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (tile rows) and the 64
  // columns of half w / 4; column c of this CTA is unit 128 rank + c
  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane, cc = half * (kTrN / 2), u0 = (int)rank * kTrN + cc;
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
  const uint32_t pHA = cluster_addr(HA, peer), pHB = cluster_addr(HB, peer);
  const uint32_t pxin[2] = {cluster_addr(&xin[0], peer), cluster_addr(&xin[1], peer)};
  const uint32_t psx = cluster_addr(&sx[rank][0], peer);
  const int ug0 = (int)rank * (kTrN / 8);  // this CTA's unit groups: ug0 .. + 15
  uint32_t xk = 0;                         // exchanges of this CTA so far
  const int64_t row0 = (*a.step % a.steps_per_epoch) * a.B;  // the batch's first training row
  const float b4 = *a.b4;
  const float invB2 = 2.f / (float)a.B;

  // a hidden layer's epilogue on this thread's 64 units, into H here and in
  // the peer: the biases of the first 32-column chunk (xb) are loaded before
  // the MMA wait, the second chunk's while the first is converted, and the
  // second chunk's TMEM load is in flight meanwhile
  auto hidden = [&](const float *__restrict__ bias, uint8_t *H, uint32_t pH, uint32_t (&m)[2], float (&xb)[32]) {
    uint32_t v[32];
    tc_ld32_issue(trow + cc, v);
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const int u = u0 + 32 * j;
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = xb[i];
      if (j < 1) tr_bias32(bias + u + 32, xb);
      tc_wait_ld32(v);
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] += __uint_as_float(v[i]);
      if (j < 1) tc_ld32_issue(trow + cc + 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = fmaxf(x[i], 0.f);
      __align__(16) bf16 hb[32];
      m[j] = tr_bf16x32(x, hb);
#pragma unroll
      for (int i = 0; i < 32; i += 8) tr_put8x(H, pH, row, u + i, hb + i);
    }
    tc_fence_before();
  };
  // back through a layer: d = bf16((d W) [h > 0]) on this thread's units,
  // into H (and with pH != 0 into the peer's H)
  auto delta = [&](uint8_t *H, uint32_t pH, const uint32_t (&m)[2]) {
    uint32_t v[32];
    tc_ld32_issue(trow + cc, v);
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const int u = u0 + 32 * j;
      tc_wait_ld32(v);
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(v[i]);
      if (j < 1) tc_ld32_issue(trow + cc + 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = ((m[j] >> i) & 1u) ? x[i] : 0.f;
      __align__(16) bf16 db[32];
      tr_bf16x32(x, db);
      if (pH) {
#pragma unroll
        for (int i = 0; i < 32; i += 8) tr_put8x(H, pH, row, u + i, db + i);
      } else {
#pragma unroll
        for (int i = 0; i < 32; i += 8) tr_put8(H, row, u + i, db + i);
      }
    }
    tc_fence_before();
  };
  auto xsend = [&]() { tr_xsend(pxin[xk & 1]); };
  auto xbar = [&]() { return &xin[xk & 1]; };
  auto xpar = [&]() { return (xk >> 1) & 1u; };

  for (int tile = cl; tile < ntiles; tile += ncl) {
    const int64_t rb = (int64_t)tile * kBM + row;  // this thread's row within the batch
    float *ts = a.tstat + (size_t)tile * kTileStats;
    // features of the tile into HB (A layout, one K chunk), each thread half of its row
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.X + (row0 + rb) * kSurrIn);
#pragma unroll
      for (int i = half * 4; i < half * 4 + 4; ++i) *reinterpret_cast<uint4 *>(HB + tr_cm(row, 8 * i)) = src[i];
    }
    uint32_t m1[2], m2[2], m3[2];  // ReLU masks of h1, h2, h3 on this thread's 64 units, one bit each
    float xb[32];
    // ---- layer 1: h1 = relu(x W1^T + b1) -> HA (both CTAs); this CTA's half of x^T out
    tr_issue(r, smem_u32(HB), 1, tmem, a.wait_limit, &abort_flag, nullptr, 0);
    tr_copy_t<kSurrIn, true, false>(HB, a.xT, tile, nullptr, nullptr, (int)rank * (kSurrIn / 16), kSurrIn / 16);
    tr_bias32(a.b1 + u0, xb);
    if (!tr_wait(r, 1, a.wait_limit, &abort_flag)) break;
    hidden(a.b1, HA, pHA, m1, xb);
    xsend();
    // ---- layer 2: h2 = relu(h1 W2^T + b2) -> HB; h1^T out
    tr_issue(r, smem_u32(HA), 4, tmem, a.wait_limit, &abort_flag, xbar(), xpar());
    ++xk;
    tr_copy_t<kSurrW, true, false>(HA, a.h1T, tile, nullptr, nullptr, ug0, kTrN / 8);
    tr_bias32(a.b2 + u0, xb);
    if (!tr_wait(r, 4, a.wait_limit, &abort_flag)) break;
    hidden(a.b2, HB, pHB, m2, xb);
    xsend();
    // ---- layer 3 and the output unit: out = relu(z3) . w4 + b4 (FP32),
    // dout = 2 (out - y) / B, d3 = bf16(dout w4 [z3 > 0]) -> HA (both CTAs),
    // bf16(h3) -> HB (this CTA's units); h2^T out
    tr_issue(r, smem_u32(HB), 4, tmem, a.wait_limit, &abort_flag, xbar(), xpar());
    ++xk;
    tr_copy_t<kSurrW, true, false>(HB, a.h2T, tile, nullptr, nullptr, ug0, kTrN / 8);
    tr_bias32(a.b3 + u0, xb);
    const float y = a.Y[row0 + rb];
    if (!tr_wait(r, 4, a.wait_limit, &abort_flag)) break;
    float out = 0.f;
    {
      uint32_t v[32];
      tc_ld32_issue(trow + cc, v);
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const int u = u0 + 32 * j;
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = xb[i];
        if (j < 1) tr_bias32(a.b3 + u + 32, xb);
        tc_wait_ld32(v);
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] += __uint_as_float(v[i]);
        if (j < 1) tc_ld32_issue(trow + cc + 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          x[i] = fmaxf(x[i], 0.f);
          out = fmaf(x[i], sw4[cc + 32 * j + i], out);
        }
        __align__(16) bf16 hb[32];
        m3[j] = tr_bf16x32(x, hb);
#pragma unroll
        for (int i = 0; i < 32; i += 8) tr_put8(HB, row, u + i, hb + i);
      }
    }
    tc_fence_before();
    // the row's dot product: this CTA's two column halves, then the two CTAs'
    // parts, added in a fixed order (unit 0 upwards) in both CTAs
    sout[half][row] = out;
    __syncthreads();
    if (half == 0) {
      const float part = sout[0][row] + sout[1][row];
      sx[rank][row] = part;
      st_cluster_f32(psx + row * 4, part);
    }
    xsend();
    {
      const bool got = mbar_wait_cluster_bounded(xbar(), xpar(), a.wait_limit);
      ++xk;
      if (!__syncthreads_and(got)) {
        if (tid == 0) abort_flag = 1;
        break;
      }
    }
    out = (sx[0][row] + sx[1][row]) + b4;
    const float e = out - y;
    const float dout = e * invB2;
    if (half == 0) {  // sout's reads are behind the barrier above
      sout[0][row] = dout;
      sout[1][row] = e * e;
    }
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const int u = u0 + 32 * j;
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = ((m3[j] >> i) & 1u) ? dout * sw4[cc + 32 * j + i] : 0.f;
      __align__(16) bf16 db[32];
      tr_bf16x32(x, db);
#pragma unroll
      for (int i = 0; i < 32; i += 8) tr_put8x(HA, pHA, row, u + i, db + i);
    }
    xsend();
    // ---- d2 = d3 W3 -> HB (both CTAs): d3^T out with the b3 sums, the w4 sums
    // from h3 and dout, the tile's dout and squared-error sums
    tr_issue(r, smem_u32(HA), 4, tmem, a.wait_limit, &abort_flag, xbar(), xpar());
    ++xk;
    tr_copy_t<kSurrW, true, true>(HA, a.d3T, tile, ts + kTileStatB3, nullptr, ug0, kTrN / 8);
    tr_copy_t<kSurrW, false, true>(HB, nullptr, tile, ts + kTileStatW4, sout[0], ug0, kTrN / 8);
    if (rank == 0 && warp == kTrThreads / 32 - 1) {
      float sd = 0.f, se = 0.f;
#pragma unroll
      for (int k = 0; k < kBM / 32; ++k) {
        sd += sout[0][lane + 32 * k];
        se += sout[1][lane + 32 * k];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
      }
      if (lane == 0) {
        ts[kTileStatB4] = sd;
        ts[kTileStatLoss] = se;
      }
    }
    if (!tr_wait(r, 4, a.wait_limit, &abort_flag)) break;
    delta(HB, pHB, m2);
    xsend();
    // ---- d1 = d2 W2 -> HA (this CTA's units): d2^T out with the b2 sums
    tr_issue(r, smem_u32(HB), 4, tmem, a.wait_limit, &abort_flag, xbar(), xpar());
    ++xk;
    tr_copy_t<kSurrW, true, true>(HB, a.d2T, tile, ts + kTileStatB2, nullptr, ug0, kTrN / 8);
    if (!tr_wait(r, 4, a.wait_limit, &abort_flag)) break;
    delta(HA, 0u, m1);
    __syncthreads();
    tr_copy_t<kSurrW, true, true>(HA, a.d1T, tile, ts + kTileStatB1, nullptr, ug0, kTrN / 8);
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
  cluster_sync_all();  // the peer's stores into this CTA are done before either exits
  if (warp == 0) tmem_dealloc(tmem, kTrN);
}

// --------------------------------------------------- weight gradients --
// dW3 = d3^T h2, dW2 = d2^T h1, dW1 = d1^T x: CTA (product, 128-row M tile,
// split z) multiplies the split's 64-row chunks of the chunk-blocked
// operands (A: 128 units of the delta, 16 KB; B: all N units of the
// activation, N x 128 bytes; one bulk copy each) through a four-stage ring:
// lane 0 of warp 0 copies, lane 0 of warp 1 issues the MMAs (M 128, N 256 or
// 64) and commits each stage back; the four warps then write the FP32
// accumulator as the split's row-major partial (SurrDwArgs).
constexpr int kDwThreads = 128;
constexpr int kDwStages = 4;
constexpr uint32_t kDwA = kBM * kBK * 2;         // 16 KB
constexpr uint32_t kDwB = kSurrW * kBK * 2;      // 32 KB (N = 256)
constexpr uint32_t kDwStage = kDwA + kDwB;
constexpr uint32_t kDwSmem = kDwStages * kDwStage;  // 192 KB

__global__ void __launch_bounds__(kDwThreads, 1) surr_dw_kernel(const SurrDwArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t full[kDwStages], empty[kDwStages], accum;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, loaded, issued;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = a.splits;
  const int prod = blockIdx.x / (2 * S), mt = (blockIdx.x % (2 * S)) / S, z = blockIdx.x % S;
  const uint8_t *A, *Bm;
  float *P;
  int N;
  if (prod == 0) {
    A = reinterpret_cast<const uint8_t *>(a.d3T), Bm = reinterpret_cast<const uint8_t *>(a.h2T), P = a.p3, N = kSurrW;
  } else if (prod == 1) {
    A = reinterpret_cast<const uint8_t *>(a.d2T), Bm = reinterpret_cast<const uint8_t *>(a.h1T), P = a.p2, N = kSurrW;
  } else {
    A = reinterpret_cast<const uint8_t *>(a.d1T), Bm = reinterpret_cast<const uint8_t *>(a.xT), P = a.p1, N = kSurrIn;
  }
  const int kc = a.B / kBK;
  const int cbeg = (int)((int64_t)z * kc / S), nk = (int)((int64_t)(z + 1) * kc / S) - cbeg;
  const uint32_t bbytes = (uint32_t)N * kBK * 2;
  if (warp == 0) {
    tmem_alloc(&tmem_slot, kSurrW);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < kDwStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&accum, 1);
    abort_flag = 0;
    loaded = 0;
    issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_wait();
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {  // producer
    for (int c = 0; c < nk && !*(volatile int *)&abort_flag; ++c) {
      const int st = c % kDwStages;
      if (c >= kDwStages && !mbar_wait_bounded(&empty[st], ((c - kDwStages) / kDwStages) & 1, a.wait_limit)) {
        abort_flag = 1;
        break;
      }
      uint8_t *sa = sm + st * kDwStage;
      mbar_arrive_expect_tx(&full[st], kDwA + bbytes);
      tma_bulk_load(sa, A + (size_t)(cbeg + c) * (kSurrW * 128) + (size_t)mt * kDwA, kDwA, &full[st]);
      tma_bulk_load(sa + kDwA, Bm + (size_t)(cbeg + c) * bbytes, bbytes, &full[st]);
      loaded = c + 1;
    }
  } else if (tid == 64 && blockIdx.x == 0 && a.sched) {
    // the step's learning rate and Adam's bias corrections (FP64 cosine: its
    // latency is spent here, beside the MMAs, not in every update block)
    const int64_t st = *a.step;
    float lr;
    if (a.sch.cosine) {
      lr = (float)(0.5 * (double)a.sch.lr * (1.0 + cos(M_PI * (double)st / (double)a.sch.total)));
    } else {
      const int64_t ep = st / a.sch.steps_per_epoch;
      lr = ep < (2 * a.sch.epochs + 2) / 3 ? a.sch.lr : a.sch.lr / 3.f;
    }
    const int64_t t = a.sch.t0 + st + 1;
    a.sched[0] = lr;
    a.sched[1] = 1.f - powf(0.9f, (float)t);
    a.sched[2] = 1.f - powf(0.999f, (float)t);
  } else if (tid == 32) {  // MMA issuer
    const uint32_t idesc = idesc_bf16_f32(kBM, N);
    for (int c = 0; c < nk; ++c) {
      const int st = c % kDwStages;
      if (!mbar_wait_bounded(&full[st], (c / kDwStages) & 1, a.wait_limit)) {
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(sm + st * kDwStage), sb = sa + kDwA;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        tc_mma(tmem, smem_desc(sa + kk * 256, 128, 1024), smem_desc(sb + kk * 256, 128, 1024), idesc,
               (c > 0 || kk > 0) ? 1u : 0u);
      tc_commit(&empty[st]);
      issued = c + 1;
    }
    if (issued == nk) tc_commit(&accum);
  }
  __syncthreads();
  bool ok = !abort_flag && issued == nk;
  if (ok) ok = __syncthreads_and(mbar_wait_bounded(&accum, 0, a.wait_limit));
  else __syncthreads();
  if (ok) {
    // the accumulator through the (now idle) ring memory, rows padded by
    // 16 bytes so that the lanes' rows fall in different banks, then one bulk
    // store per row into the split's row-major partial
    tc_fence_after();
    const int rl = warp * 32 + lane;  // this thread's accumulator row (TMEM lane)
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t pitch = (uint32_t)N * 4 + 16;
    float *srow = reinterpret_cast<float *>(sm + (size_t)rl * pitch);
    uint32_t v[32];
    tc_ld32_issue(trow, v);
#pragma unroll 1
    for (int j0 = 0; j0 < N; j0 += 32) {
      tc_wait_ld32(v);
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(v[i]);
      if (j0 + 32 < N) tc_ld32_issue(trow + j0 + 32, v);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4 *>(srow + j0 + 4 * q) = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    tma_bulk_store(P + (size_t)z * N * kSurrW + (size_t)(mt * kBM + rl) * N, srow, (uint32_t)N * 4);
    tma_bulk_store_wait();
  } else if (tid == 0) {
    // let the copies and MMAs already issued land (bounded) before the
    // shared and tensor memory are released, and report
    for (int c = issued; c < loaded; ++c) mbar_wait_bounded(&full[c % kDwStages], (c / kDwStages) & 1, kGemmDrain);
    if (issued > 0)
      mbar_wait_bounded(&empty[(issued - 1) % kDwStages], ((issued - 1) / kDwStages) & 1, kGemmDrain);
    atomicOr(a.err, kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kSurrW);
}

// -------------------------------------------------------------- update ---
// Flat parameter order: W1, b1, W2, b2, W3, b3, w4, b4.
constexpr int64_t kTrOffW1 = 0, kTrOffB1 = kTrOffW1 + (int64_t)kSurrW * kSurrIn, kTrOffW2 = kTrOffB1 + kSurrW,
                  kTrOffB2 = kTrOffW2 + (int64_t)kSurrW * kSurrW, kTrOffW3 = kTrOffB2 + kSurrW,
                  kTrOffB3 = kTrOffW3 + (int64_t)kSurrW * kSurrW, kTrOffW4 = kTrOffB3 + kSurrW,
                  kTrOffB4 = kTrOffW4 + kSurrW;
constexpr int kAdThreads = 256;
constexpr int kAdW1 = kSurrW * kSurrIn / 4, kAdW2 = kSurrW * kSurrW / 4;  // threads: four entries each
constexpr int kAdZ = 4;  // threads per four-entry group, each over every fourth split
constexpr int kAdWBlocks = (kAdW1 + 2 * kAdW2) / (kAdThreads / kAdZ);
constexpr int kAdSBlocks = (kTileStats + 31) / 32;
static_assert((kAdW1 + 2 * kAdW2) % (kAdThreads / kAdZ) == 0 && kAdW1 % (kAdThreads / kAdZ) == 0 &&
                  kAdW2 % (kAdThreads / kAdZ) == 0,
              "whole blocks of weight threads, each within one matrix");

__device__ __forceinline__ void adam1(float &p, float &m, float &v, float g, float lr, float c1, float c2) {
  m = 0.9f * m + 0.1f * g;
  v = 0.999f * v + 0.001f * g * g;
  p = p - lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

// Four threads per four consecutive entries (u, 4 c4 .. + 3) of one weight
// matrix (the partials' float4); eight per bias, output weight, the output
// bias and the loss.  Gradients: weight entries sum their partials in
// split order, the others their tile sums in tile order.  With `update`,
// Adam (beta1 0.9, beta2 0.999, eps 1e-8) at the step's learning rate and
// bias correction from the device counter, the BF16 copies of W1, W2, W3
// ([out][in] and the training step's weight blocks), and the last block to
// finish advances the step counter.
__global__ void __launch_bounds__(kAdThreads) surr_adam_kernel(const SurrAdamArgs a) {
  __shared__ float s_lr, s_c1, s_c2;
  __shared__ int64_t s_step;
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) {
    s_step = *a.step;
    if (a.update) {
      s_lr = a.sched[0];
      s_c1 = a.sched[1];
      s_c2 = a.sched[2];
    }
  }
  __syncthreads();
  const float lr = s_lr, c1 = s_c1, c2 = s_c2;
  if (blockIdx.x < kAdWBlocks) {
    // 64 four-entry groups per block; thread group zg (of 4) sums splits
    // zg, zg + 4, ...; group 0 adds the four sums in group order
    __shared__ float4 zpart[kAdZ][kAdThreads / kAdZ];
    const int el = threadIdx.x % (kAdThreads / kAdZ), zg = threadIdx.x / (kAdThreads / kAdZ);
    int t = blockIdx.x * (kAdThreads / kAdZ) + el, layer, N;
    const float *part;
    int64_t off;
    bf16 *wb;
    if (t < kAdW1) {
      layer = 0, N = kSurrIn, part = a.p1, off = kTrOffW1, wb = a.w1;
    } else if (t < kAdW1 + kAdW2) {
      t -= kAdW1, layer = 1, N = kSurrW, part = a.p2, off = kTrOffW2, wb = a.w2;
    } else {
      t -= kAdW1 + kAdW2, layer = 2, N = kSurrW, part = a.p3, off = kTrOffW3, wb = a.w3;
    }
    const int u = t / (N / 4), c4 = t % (N / 4);  // entries (u, 4 c4 .. + 3), flat index 4 t
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *src = reinterpret_cast<const float4 *>(part) + t;
#pragma unroll 2
    for (int z = zg; z < a.splits; z += kAdZ) {
      const float4 q = src[(size_t)z * N * kSurrW / 4];
      g.x += q.x, g.y += q.y, g.z += q.z, g.w += q.w;
    }
    zpart[zg][el] = g;
    __syncthreads();
    if (zg == 0) {
#pragma unroll
      for (int k = 1; k < kAdZ; ++k) {
        const float4 q = zpart[k][el];
        g.x += q.x, g.y += q.y, g.z += q.z, g.w += q.w;
      }
      const int64_t i = off + (int64_t)u * N + 4 * c4;
      *reinterpret_cast<float4 *>(a.G + i) = g;
      if (a.update) {
        float4 p = *reinterpret_cast<const float4 *>(a.p + i), m = *reinterpret_cast<const float4 *>(a.m + i),
               v = *reinterpret_cast<const float4 *>(a.v + i);
        adam1(p.x, m.x, v.x, g.x, lr, c1, c2);
        adam1(p.y, m.y, v.y, g.y, lr, c1, c2);
        adam1(p.z, m.z, v.z, g.z, lr, c1, c2);
        adam1(p.w, m.w, v.w, g.w, lr, c1, c2);
        *reinterpret_cast<float4 *>(a.p + i) = p;
        *reinterpret_cast<float4 *>(a.m + i) = m;
        *reinterpret_cast<float4 *>(a.v + i) = v;
        __align__(8) bf16 h[4] = {__float2bfloat16_rn(p.x), __float2bfloat16_rn(p.y), __float2bfloat16_rn(p.z),
                                  __float2bfloat16_rn(p.w)};
        *reinterpret_cast<uint2 *>(wb + (int64_t)u * N + 4 * c4) = *reinterpret_cast<const uint2 *>(h);
        surr_wc_put4(a.wc, layer, u, 4 * c4, h);
      }
    }
  } else {
    // 32 entries per block: thread group k (of 8) sums tiles k, k + 8, ...;
    // then the eight group sums are added in group order
    __shared__ float part[kAdThreads / 32][32];
    const int el = threadIdx.x & 31, k = threadIdx.x >> 5;
    const int e = (blockIdx.x - kAdWBlocks) * 32 + el;
    float g = 0.f;
    if (e < kTileStats)
      for (int t = k; t < a.ntiles; t += kAdThreads / 32) g += a.tstat[(size_t)t * kTileStats + e];
    part[k][el] = g;
    __syncthreads();
    if (k == 0 && e < kTileStats) {
      g = 0.f;
#pragma unroll
      for (int j = 0; j < kAdThreads / 32; ++j) g += part[j][el];
      if (e == kTileStatLoss) {
        if (a.loss_hist) a.loss_hist[s_step] = g / (float)a.B;
      } else {
        const int64_t i = e < kTileStatW4 ? (e < kTileStatB2 ? kTrOffB1 + e
                                                             : (e < kTileStatB3 ? kTrOffB2 + (e - kTileStatB2)
                                                                                : kTrOffB3 + (e - kTileStatB3)))
                                          : (e < kTileStatB4 ? kTrOffW4 + (e - kTileStatW4) : kTrOffB4);
        a.G[i] = g;
        if (a.update) adam1(a.p[i], a.m[i], a.v[i], g, lr, c1, c2);
      }
    }
  }
  if (!a.update) return;
  // every thread of the block is past its reads of the step counter
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1u) == gridDim.x - 1) {
      __threadfence();
      *a.done = 0;
      *a.step += 1;
    }
  }
}

// ------------------------------------------------------------ launchers --
static_assert(kTrSmem + kTrN * sizeof(float) + 4 * kBM * sizeof(float) + 256 <= 232448,
              "tile kernel above 227 KB of shared memory");

// a launch that may begin while the stream's previous kernel drains (each
// kernel waits for it with pdl_wait before touching global memory)
template <typename Arg>
static cudaError_t launch_pdl(void (*kernel)(Arg), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              const Arg &arg) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, arg);
}

cudaError_t launch_surr_tile(const SurrStepArgs &a, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(surr_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrSmem);
  if (e != cudaSuccess) return e;
  const int ntiles = a.B / kBM, clusters = ntiles < sms / 2 ? ntiles : sms / 2;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(2 * clusters));
  cfg.blockDim = dim3(kTrThreads);
  cfg.dynamicSmemBytes = kTrSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, surr_tile_kernel, a);
}

cudaError_t launch_surr_dw(const SurrDwArgs &a, cudaStream_t s) {
  if (a.B % kBK || a.splits < 1 || a.splits > a.B / kBK) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(surr_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwSmem);
  if (e != cudaSuccess) return e;
  return launch_pdl(surr_dw_kernel, (unsigned)(6 * a.splits), kDwThreads, kDwSmem, s, a);
}

cudaError_t launch_surr_adam(const SurrAdamArgs &a, cudaStream_t s) {
  return launch_pdl(surr_adam_kernel, kAdWBlocks + kAdSBlocks, kAdThreads, 0, s, a);
}

cudaError_t launch_surr_wc(const bf16 *w1, const bf16 *w2, const bf16 *w3, uint8_t *wc, cudaStream_t s) {
  constexpr int n = kSurrW * kSurrIn + 2 * kSurrW * kSurrW;
  surr_wc_kernel<<<(n + 255) / 256, 256, 0, s>>>(w1, w2, w3, wc);
  return cudaGetLastError();
}

}  // namespace fk
