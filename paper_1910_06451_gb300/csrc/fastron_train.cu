// Fastron model update, Algorithm 1 (Sec. III-B), as one persistent
// thread-block cluster.
//
// Ownership: the cluster has C CTAs of 256 threads; global thread
// g = rank * 256 + tid owns the training points j = g + 256 C k.  Its
// margins F_j (FP64) live in registers, its weights alpha_j (FP64) in its
// CTA's shared memory (read and written only by the owner).  Each pass:
//   1. every thread holds the same candidate, the argmin of y_j F_j with its
//      label and alpha, and takes the same decision: add/adjust (Eqs. 6-8)
//      or, when no add applies, form the removal candidate (the argmax over
//      alpha_j != 0 of y_j (F_j - alpha_j)) and remove it or stop;
//   2. every thread updates its F_j with row i of the stored kernel matrix
//      (symmetric, so row i is column i; FP64, or FP32 entries widened to
//      FP64 exactly); the owner of i updates alpha_i;
//   3. the argmin candidate is reduced: per thread, warp, one __syncthreads
//      for the CTA, then lane r of warp 0 sends the CTA's candidate into
//      slot `rank` of CTA r with asynchronous distributed-shared-memory
//      stores that complete bytes on CTA r's exchange mbarrier (20 bytes
//      from each of the C CTAs complete a phase).  Warp 0 polls its own
//      barrier, a CTA barrier hands the outcome to the other warps, and
//      every warp reduces the C slots itself.  Slots and barriers are
//      double-buffered by round parity.  (Measured on a 16-CTA cluster: about
//      700 cycles per exchange against about 1230 for a hardware cluster
//      barrier after plain remote stores.)  Each warp-level step is three
//      redux.sync reductions and one shuffle rather than a shuffle butterfly.
//      The removal candidate (argmax) is formed and reduced the same way, but
//      only in a pass where no add applies.
// The row of the argmin candidate is requested before the decision is taken
// (an add step is the common case), so its latency overlaps the decision;
// the decision's FP64 arithmetic runs in one lane per warp and is broadcast.
// Comparisons run on int64 keys that order like the doubles (sign-magnitude
// folded to two's complement, zeros made +0), so the argmin/argmax work stays
// off the FP64 pipe, which on this part runs at 1/64 of the FP32 rate; ties
// go to the lowest index, as in a left-to-right scan.  F and alpha are
// updated in FP64 in the order of Eqs. 6-8, F by one fused multiply-add per
// entry.  Each exchange wait polls at most wait_limit times; a CTA whose
// wait runs out reports a timeout in stats[5] and leaves the loop (every
// other CTA then runs out at its next wait), waits a bounded time for stores
// still in flight toward it, and a final cluster barrier keeps every CTA
// resident until all CTAs are past their last store.  The loop is bounded by
// iter_max.
#include <cooperative_groups.h>

#include <climits>

#include "fk_internal.h"
#include "fk_ptx.cuh"

namespace cg = cooperative_groups;

namespace fk {

constexpr int kTrainThreads = 256;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kMaxCluster = 16;
constexpr long long kMag = 0x7fffffffffffffffLL;
constexpr long long kSign = (long long)0x8000000000000000ULL;

struct Cand {
  long long key;  // ordered key of the margin (argmin) or removal margin (argmax)
  double alpha;   // alpha of the candidate
  int iy;         // index | (label < 0) << 31; INT_MAX if none
};

// Order-preserving int64 image of the double with bit pattern b: for
// non-negative values the pattern, for negative values the pattern with all
// but the sign bit flipped.  -0.0 maps to the key of +0.0, so the two compare
// equal, as doubles do.
__device__ __forceinline__ long long bits_key(long long b) {
  if ((b & kMag) == 0) return 0;
  return b ^ ((b >> 63) & kMag);
}
__device__ __forceinline__ double key_value(long long k) { return __longlong_as_double(k >= 0 ? k : (k ^ kMag)); }
__device__ __forceinline__ bool nonzero(double v) { return (__double_as_longlong(v) & kMag) != 0; }

// Exact FP32 -> FP64 widening of kernel-matrix entries by integer operations,
// keeping the conversion off the FP64 pipe: a positive normal value gets its
// exponent rebiased (127 -> 1023) and its fraction shifted; zero stays zero.
// Other values (subnormal entries, possible only for enormous gamma without a
// base control point) are flagged by needs_cast and take the ordinary
// conversion instead.
__device__ __forceinline__ double widen_fast(float x) {
  const unsigned b = __float_as_uint(x);
  return b ? __longlong_as_double(((long long)b << 29) + (896LL << 52)) : 0.0;
}
__device__ __forceinline__ bool needs_cast(float x) {
  const unsigned b = __float_as_uint(x);
  return b != 0u && b - 0x00800000u >= 0x7f000000u;
}
__device__ __forceinline__ double widen_fast(double x) { return x; }
__device__ __forceinline__ bool needs_cast(double) { return false; }

__device__ __forceinline__ int cidx(const Cand &c) { return c.iy & 0x7fffffff; }
// Warp-wide argmin / argmax with the single-instruction warp reductions
// (redux.sync): first the high 32 bits of the key (signed), then the low 32
// bits among the lanes that tie on the high part (unsigned), then the lowest
// index among full ties; the winner's alpha and label come from its lane by
// one shuffle.  Every lane of the warp gets the same candidate.
__device__ __forceinline__ Cand warp_argmin(const Cand &c) {
  const unsigned full = 0xffffffffu;
  const int hi = (int)(c.key >> 32);
  const unsigned lo = (unsigned)c.key, ix = (unsigned)cidx(c);
  const int mh = __reduce_min_sync(full, hi);
  const unsigned ml = __reduce_min_sync(full, hi == mh ? lo : 0xffffffffu);
  const bool tie = hi == mh && lo == ml;
  const unsigned mi = __reduce_min_sync(full, tie ? ix : 0xffffffffu);
  const int src = __ffs(__ballot_sync(full, tie && ix == mi)) - 1;
  Cand r;
  r.key = ((long long)mh << 32) | (long long)ml;
  r.alpha = __shfl_sync(full, c.alpha, src);
  r.iy = __shfl_sync(full, c.iy, src);
  return r;
}

__device__ __forceinline__ Cand warp_argmax(const Cand &c) {
  const unsigned full = 0xffffffffu;
  const int hi = (int)(c.key >> 32);
  const unsigned lo = (unsigned)c.key, ix = (unsigned)cidx(c);
  const int mh = __reduce_max_sync(full, hi);
  const unsigned ml = __reduce_max_sync(full, hi == mh ? lo : 0u);
  const bool tie = hi == mh && lo == ml;
  const unsigned mi = __reduce_min_sync(full, tie ? ix : 0xffffffffu);
  const int src = __ffs(__ballot_sync(full, tie && ix == mi)) - 1;
  Cand r;
  r.key = ((long long)mh << 32) | (long long)ml;
  r.alpha = __shfl_sync(full, c.alpha, src);
  r.iy = __shfl_sync(full, c.iy, src);
  return r;
}

// Every decision below must be identical in every thread of the cluster,
// because every thread then meets the same barriers; the warp reductions give
// every lane the same answer.

__device__ __forceinline__ Cand no_min() { return {LLONG_MAX, 0.0, INT_MAX}; }
__device__ __forceinline__ Cand no_max() { return {LLONG_MIN, 0.0, INT_MAX}; }

// One exchanged candidate: key and alpha in one 16-byte store, index|label in
// a second 4-byte store.
struct __align__(16) Msg {
  long long key;
  double alpha;
};
constexpr uint32_t kMsgBytes = sizeof(Msg) + sizeof(int);
// polls of an exchange barrier after a timeout, before the final cluster
// barrier (independent of the caller's wait limit, so that stores in flight
// toward this CTA land while it is still resident)
constexpr uint32_t kDrainPolls = 1u << 16;

struct TrainShared {
  uint64_t xbar[2];  // exchange barriers, one per round parity
  Msg msg_min[2][kMaxCluster], msg_max[2][kMaxCluster];
  int iy_min[2][kMaxCluster], iy_max[2][kMaxCluster];
  Cand wmin[kTrainWarps], wmax[kTrainWarps];
  int slot_cnt[kMaxCluster], wcnt[kTrainWarps];
  double dec_delta;  // the add step's delta, computed by one thread of the CTA
  int dec_nz;        // whether alpha_i + delta is nonzero
};

__device__ __forceinline__ double neg(double x) { return __longlong_as_double(__double_as_longlong(x) ^ kSign); }

template <int KMAX, typename GT>
__global__ void __launch_bounds__(kTrainThreads, 1) fastron_train_kernel(const TrainArgs a) {
  static_assert(KMAX <= 32, "labels are kept as a bit mask");
  const GT *__restrict__ G = static_cast<const GT *>(a.G);
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TrainShared sh;
  double *alpha = reinterpret_cast<double *>(smem_raw);  // [KMAX][kTrainThreads], owner-private

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int stride = kTrainThreads * C;
  const int g = rank * kTrainThreads + tid;
  const int N = (int)a.N;
  // slice k of this warp holds points j0 + stride k .. + 31: a slice wholly
  // past N is skipped by the whole warp (no FP64 work on padding)
  const int j0w = rank * kTrainThreads + warp * 32;
  auto live = [&](int k) { return j0w + stride * k < N; };

  double F[KMAX];
  unsigned yneg = 0;  // bit k: label of point g + stride k is -1
  int nnz_local = 0;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int j = g + stride * k;
    F[k] = 0.0;
    double aj = 0.0;
    if (j < N) {
      F[k] = a.F[j];
      yneg |= (a.y[j] > 0 ? 0u : 1u) << k;
      aj = a.alpha[j];
      nnz_local += nonzero(aj);
    }
    alpha[k * kTrainThreads + tid] = aj;
  }
  if (tid == 0) {
    // one local arrival (the arming) and C x kMsgBytes per phase
    mbar_init(&sh.xbar[0], 1u);
    mbar_init(&sh.xbar[1], 1u);
    mbar_fence_init_cluster();
    mbar_arrive_expect_tx(&sh.xbar[0], kMsgBytes * (uint32_t)C);
    mbar_arrive_expect_tx(&sh.xbar[1], kMsgBytes * (uint32_t)C);
  }
  // every CTA of the cluster is running, with its barriers initialised and
  // armed, before any remote store
  cluster.sync();

  // |{alpha != 0}| over the cluster: identical in every thread afterwards and
  // updated uniformly by the decisions below.
  long long nnz;
  {
    int w = nnz_local;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) sh.wcnt[warp] = w;
    __syncthreads();
    if (warp == 0) {
      int t = lane < kTrainWarps ? sh.wcnt[lane] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane < C) *cluster.map_shared_rank(&sh.slot_cnt[rank], lane) = t;
    }
    cluster.sync();
    int t = lane < C ? sh.slot_cnt[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    nnz = t;
  }

  int parity = 0;
  uint32_t phase = 0;  // bit b: parity of the current phase of xbar[b]
  Cand mn, mx;
  // argmin of the margins y_j F_j (every pass)
  auto local_min = [&]() {
    mn = no_min();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int j = g + stride * k;
      if (live(k) && j < N) {
        const unsigned yn = (yneg >> k) & 1u;
        const long long km = bits_key(__double_as_longlong(F[k]) ^ ((long long)yn << 63));  // key of y_j F_j
        if (km < mn.key) mn = {km, alpha[k * kTrainThreads + tid], j | (int)(yn << 31)};  // j ascends
      }
    }
  };
  // argmax over alpha_j != 0 of y_j (F_j - alpha_j): only in passes where
  // no add applies, which are few (removals and the final check)
  auto local_max = [&]() {
    mx = no_max();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int j = g + stride * k;
      if (live(k) && j < N) {
        const double aj = alpha[k * kTrainThreads + tid];
        if (nonzero(aj)) {
          const unsigned yn = (yneg >> k) & 1u;
          const long long kr = bits_key(__double_as_longlong(__dsub_rn(F[k], aj)) ^ ((long long)yn << 63));
          if (kr > mx.key) mx = {kr, aj, j | (int)(yn << 31)};
        }
      }
    }
  };
  // warp, then CTA through shared memory, then cluster through one slot per
  // CTA in every CTA and the exchange barriers.  Slots and barriers
  // alternate by round parity: a CTA stores round r + 2 into a slot only
  // after its own round r + 1 wait, which needs every CTA's round r + 1
  // stores, which each CTA issues after all its warps have read their round r
  // slots; and the phase of round r + 2 is armed after the phase of round r
  // completed.  Returns false (in every thread of the CTA) if the wait ran
  // out.
  const uint32_t lim = a.wait_limit;
  const uint32_t xbytes = kMsgBytes * (uint32_t)C;
  auto exchange = [&](Msg (*msg)[kMaxCluster], int (*iy)[kMaxCluster], const Cand &c) -> bool {
    bool ok = true;
    if (warp == 0) {
      if (lane < C) {
        const uint32_t rb = cluster_addr(&sh.xbar[parity], (uint32_t)lane);
        st_async_b64x2(cluster_addr(&msg[parity][rank], (uint32_t)lane), c.key, __double_as_longlong(c.alpha), rb);
        st_async_b32(cluster_addr(&iy[parity][rank], (uint32_t)lane), c.iy, rb);
      }
      const uint32_t want = (phase >> parity) & 1u;
      ok = false;
      for (uint32_t it = 0; it < lim && !ok; ++it) ok = mbar_test_wait_cluster(&sh.xbar[parity], want);
      if (ok && lane == 0) mbar_arrive_expect_tx(&sh.xbar[parity], xbytes);  // the phase of round r + 2
    }
    const int bad = __syncthreads_or(!ok);
    phase ^= 1u << parity;
    return bad == 0;
  };
  auto slot = [&](Msg (*msg)[kMaxCluster], int (*iy)[kMaxCluster], int r) -> Cand {
    const Msg m = msg[parity][r];
    return {m.key, m.alpha, iy[parity][r]};
  };
  auto reduce_min = [&]() -> bool {
    mn = warp_argmin(mn);
    if (lane == 0) sh.wmin[warp] = mn;
    __syncthreads();
    const Cand c = warp == 0 ? warp_argmin(lane < kTrainWarps ? sh.wmin[lane] : no_min()) : no_min();
    if (!exchange(sh.msg_min, sh.iy_min, c)) return false;
    mn = warp_argmin(lane < C ? slot(sh.msg_min, sh.iy_min, lane) : no_min());
    parity ^= 1;
    return true;
  };
  auto reduce_max = [&]() -> bool {
    mx = warp_argmax(mx);
    if (lane == 0) sh.wmax[warp] = mx;
    __syncthreads();
    const Cand c = warp == 0 ? warp_argmax(lane < kTrainWarps ? sh.wmax[lane] : no_max()) : no_max();
    if (!exchange(sh.msg_max, sh.iy_max, c)) return false;
    mx = warp_argmax(lane < C ? slot(sh.msg_max, sh.iy_max, lane) : no_max());
    parity ^= 1;
    return true;
  };

  local_min();
  bool timed_out = !reduce_min();
  long long iters = 0, adds = 0, removes = 0;
  int converged = 0;
  for (long long iter = 1; iter <= a.iter_max && !timed_out; ++iter) {
    // request the argmin's row first: an add step is the common case
    GT gk[KMAX];
    const int imin = cidx(mn);
    const bool min_valid = imin != INT_MAX;
    if (min_valid) {
      const GT *row = G + (long long)imin * N;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int j = g + stride * k;
        gk[k] = live(k) && j < N ? row[j] : GT(0);
      }
    }
    int kind, i;
    double coef, delta;
    if (min_valid && mn.key <= 0 && (nnz < a.s_max || nonzero(mn.alpha))) {
      // add / adjust support point i: delta = b_i y_i - F_i (Eq. 6); the FP64
      // arithmetic runs in one thread of the CTA (an FP64 instruction costs
      // the whole warp's share of this part's narrow FP64 pipe even with one
      // lane active) and is shared through shared memory
      kind = 1;
      i = imin;
      if (tid == 0) {
        const bool yn = mn.iy < 0;
        // F_i = y_i * (y_i F_i): a sign flip of the margin's bit pattern
        const double Fi = __longlong_as_double(__double_as_longlong(key_value(mn.key)) ^ (yn ? kSign : 0LL));
        const double by = yn ? -1.0 : a.beta;  // b_i y_i with b_i = beta^(0.5 (y_i + 1))
        const double dl = __dsub_rn(by, Fi);
        // alpha_i + delta (Eq. 7) is zero exactly when delta == -alpha_i
        const long long bd = __double_as_longlong(dl), ba = __double_as_longlong(mn.alpha);
        sh.dec_delta = dl;
        sh.dec_nz = !(((bd ^ kSign) == ba) || (!nonzero(dl) && !nonzero(mn.alpha)));
      }
      __syncthreads();
      delta = sh.dec_delta;
      const int nz_new = sh.dec_nz;
      coef = delta;
      nnz += (long long)nz_new - (long long)nonzero(mn.alpha);
      const int gi = i % stride;
      if (gi / kTrainThreads == rank && gi % kTrainThreads == tid)
        alpha[(i / stride) * kTrainThreads + tid] = __dadd_rn(mn.alpha, delta);
      ++adds;
    } else {
      local_max();
      if (!reduce_max()) {
        timed_out = true;
        break;
      }
      if (cidx(mx) == INT_MAX || mx.key <= 0) {
        converged = 1;
        break;
      }
      // remove the redundant support point i
      kind = 2;
      i = cidx(mx);
      coef = mx.alpha;
      delta = neg(mx.alpha);
      const int gi = i % stride;
      if (gi / kTrainThreads == rank && gi % kTrainThreads == tid) alpha[(i / stride) * kTrainThreads + tid] = 0.0;
      --nnz;
      ++removes;
      const GT *row = G + (long long)i * N;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int j = g + stride * k;
        gk[k] = live(k) && j < N ? row[j] : GT(0);
      }
    }
    ++iters;
    if (rank == 0 && tid == 0 && a.trace_kind) {
      a.trace_kind[iter - 1] = (int8_t)kind;
      a.trace_idx[iter - 1] = i;
      a.trace_delta[iter - 1] = delta;
    }
    // Eq. 8: F += delta K e_i (add), or F -= alpha_i K e_i (removal), each
    // entry one fused multiply-add rounded once, with the signed coefficient
    const double c = kind == 1 ? coef : neg(coef);
    bool cast = false;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) cast |= needs_cast(gk[k]);
    if (!__any_sync(0xffffffffu, cast)) {
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (live(k)) F[k] = __fma_rn(c, widen_fast(gk[k]), F[k]);
    } else {
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (live(k)) F[k] = __fma_rn(c, (double)gk[k], F[k]);
    }
    local_min();
    timed_out = !reduce_min();
  }

#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int j = g + stride * k;
    if (j < N) {
      a.F[j] = F[k];
      a.alpha[j] = alpha[k * kTrainThreads + tid];
    }
  }
  if (rank == 0 && tid == 0) {
    a.stats[0] = iters;
    a.stats[1] = adds;
    a.stats[2] = removes;
    a.stats[3] = converged;
  }
  if (timed_out && tid == 0) {
    a.stats[5] = 1;  // zeroed by the host before the launch
    // stores of this round or the next may still be on their way here: wait
    // for both phases, each for at most kDrainPolls polls (a phase that a
    // missing CTA keeps open runs the bound out, long after any store issued
    // before it has landed)
    for (int b = 0; b < 2; ++b) {
      bool done = false;
      for (uint32_t it = 0; it < kDrainPolls && !done; ++it) done = mbar_test_wait_cluster(&sh.xbar[b], (phase >> b) & 1u);
    }
  }
  // every CTA is past its last store before any CTA leaves
  cluster.sync();
}

// removeNonsupportPoints: ascending indices with alpha != 0, one CTA.
constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads) compact_kernel(const double *__restrict__ alpha, int N,
                                                                 int32_t *__restrict__ sup_idx,
                                                                 double *__restrict__ sup_alpha,
                                                                 int64_t *__restrict__ stats) {
  __shared__ int tot[kCompactThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int base = 0;
  for (int c0 = 0; c0 < N; c0 += kCompactThreads) {
    const int j = c0 + tid;
    const double aj = j < N ? alpha[j] : 0.0;
    const bool keep = nonzero(aj);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) {
      const int t = tot[w];
      before += w < warp ? t : 0;
      total += t;
    }
    if (keep) {
      const int pos = base + before + __popc(bal & ((1u << lane) - 1u));
      sup_idx[pos] = j;
      sup_alpha[pos] = aj;
    }
    base += total;
    __syncthreads();
  }
  if (tid == 0) stats[4] = base;
}

template <int KMAX, typename GT>
static cudaError_t launch_k(const TrainArgs &a, int C, cudaStream_t s) {
  auto kern = fastron_train_kernel<KMAX, GT>;
  const size_t smem = sizeof(double) * KMAX * kTrainThreads;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kTrainThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorLaunchOutOfResources;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename GT>
static cudaError_t launch_c(const TrainArgs &a, int C, cudaStream_t s) {
  const int64_t per = (int64_t)kTrainThreads * C;
  const int64_t kneed = (a.N + per - 1) / per;
  if (kneed <= 1) return launch_k<1, GT>(a, C, s);
  if (kneed <= 2) return launch_k<2, GT>(a, C, s);
  if (kneed <= 4) return launch_k<4, GT>(a, C, s);
  if (kneed <= 8) return launch_k<8, GT>(a, C, s);
  if (kneed <= 16) return launch_k<16, GT>(a, C, s);
  return cudaErrorInvalidValue;
}

static cudaError_t launch_any(const TrainArgs &a, int C, cudaStream_t s) {
  return a.g32 ? launch_c<float>(a, C, s) : launch_c<double>(a, C, s);
}

cudaError_t launch_fastron_train(const TrainArgs &a, cudaStream_t s) {
  // as many CTAs as the points need (at least 2 per thread below 16 CTAs)
  int C = 1;
  while (C < kMaxCluster && (int64_t)kTrainThreads * C * 2 < a.N) C *= 2;
  cudaError_t e = launch_any(a, C, s);
  if (e != cudaSuccess && C > 8 && a.N <= (int64_t)kTrainThreads * 8 * 16) {
    cudaGetLastError();  // the non-portable size may be unavailable: fall back to 8
    e = launch_any(a, 8, s);
  }
  if (e != cudaSuccess) return e;
  compact_kernel<<<1, kCompactThreads, 0, s>>>(a.alpha, (int)a.N, a.sup_idx, a.sup_alpha, a.stats);
  return cudaGetLastError();
}

}  // namespace fk
