// Fastron model update, Algorithm 1 (Sec. III-B), as one persistent CTA.
//
// The training margins F (FP64) live in registers: thread t owns the points
// j = t + 1024 k.  The weights alpha (FP64) live in shared memory and are only
// ever read or written by their owner thread.  Each pass:
//   1. every thread holds the block-wide argmin of y_j F_j and the block-wide
//      argmax over alpha_j != 0 of y_j (F_j - alpha_j); each candidate carries
//      its label and its alpha through the reduction, so no thread reads
//      another thread's alpha (F_i = y_i * margin is exact for y_i = +-1);
//   2. the add/adjust step (Eqs. 6-8) or the removal step is applied: every
//      thread updates its F_j with row i of the stored kernel matrix (the
//      matrix is symmetric, so row i is column i);
//   3. the new candidates are reduced: warp shuffles, one __syncthreads, and
//      every warp reduces the 32 warp results itself (the per-warp slots are
//      double-buffered by pass parity, so one barrier per pass suffices).
// Ties go to the lowest index, as in a left-to-right scan.  F and alpha are
// updated with separately rounded products and sums, in the order of Eqs. 6-8.
// The loop has no inter-CTA waits.
#include <climits>

#include "fk_internal.h"

namespace fk {

constexpr int kTrainThreads = 1024;
constexpr int kTrainWarps = kTrainThreads / 32;

struct Cand {
  double v;      // margin y F (argmin) or removal margin y (F - alpha) (argmax)
  double alpha;  // alpha of the candidate
  int i;         // index; INT_MAX if none
  int y;         // label of the candidate
};

__device__ __forceinline__ bool better_min(const Cand &a, const Cand &b) {
  return a.v < b.v || (a.v == b.v && a.i < b.i);
}
__device__ __forceinline__ bool better_max(const Cand &a, const Cand &b) {
  return a.v > b.v || (a.v == b.v && a.i < b.i);
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int lane_mask) {
  Cand o;
  o.v = __shfl_xor_sync(0xffffffffu, c.v, lane_mask);
  o.alpha = __shfl_xor_sync(0xffffffffu, c.alpha, lane_mask);
  o.i = __shfl_xor_sync(0xffffffffu, c.i, lane_mask);
  o.y = __shfl_xor_sync(0xffffffffu, c.y, lane_mask);
  return o;
}

__device__ __forceinline__ void warp_reduce(Cand &mn, Cand &mx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const Cand a = shfl_cand(mn, o), b = shfl_cand(mx, o);
    if (better_min(a, mn)) mn = a;
    if (better_max(b, mx)) mx = b;
  }
}

__device__ __forceinline__ int block_sum(int v, int *tot, int lane, int warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) tot[warp] = v;
  __syncthreads();
  int t = tot[lane];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  return t;
}

template <int KMAX>
__global__ void __launch_bounds__(kTrainThreads, 1) fastron_train_kernel(const TrainArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Cand slot_min[2][kTrainWarps], slot_max[2][kTrainWarps];
  __shared__ int tot[kTrainWarps];
  double *alpha = reinterpret_cast<double *>(smem_raw);  // [N], owner-private entries

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = (int)a.N;
  double F[KMAX];
  int yv[KMAX];
  int nnz_local = 0;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int j = tid + kTrainThreads * k;
    F[k] = 0.0;
    yv[k] = 1;
    if (j < N) {
      F[k] = a.F[j];
      yv[k] = a.y[j] > 0 ? 1 : -1;
      alpha[j] = a.alpha[j];
      nnz_local += a.alpha[j] != 0.0;
    }
  }
  // |{alpha != 0}|, identical in every thread and updated uniformly below.
  int64_t nnz = block_sum(nnz_local, tot, lane, warp);

  int parity = 0;
  auto reduce_candidates = [&](Cand &mn, Cand &mx) {
    mn = {INFINITY, 0.0, INT_MAX, 1};
    mx = {-INFINITY, 0.0, INT_MAX, 1};
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int j = tid + kTrainThreads * k;
      if (j < N) {
        const double aj = alpha[j];
        const double m = yv[k] > 0 ? F[k] : -F[k];
        if (m < mn.v) mn = {m, aj, j, yv[k]};  // j ascends within a thread
        if (aj != 0.0) {
          const double d = __dsub_rn(F[k], aj);
          const double r = yv[k] > 0 ? d : -d;
          if (r > mx.v) mx = {r, aj, j, yv[k]};
        }
      }
    }
    warp_reduce(mn, mx);
    if (lane == 0) {
      slot_min[parity][warp] = mn;
      slot_max[parity][warp] = mx;
    }
    __syncthreads();
    mn = slot_min[parity][lane];
    mx = slot_max[parity][lane];
    warp_reduce(mn, mx);
    parity ^= 1;
  };

  Cand mn, mx;
  reduce_candidates(mn, mx);
  int64_t iters = 0, adds = 0, removes = 0;
  int converged = 0;
  for (int64_t iter = 1; iter <= a.iter_max; ++iter) {
    int i = -1, kind = 0;
    double coef = 0.0, delta = 0.0;
    if (mn.i != INT_MAX && mn.v <= 0.0 && (nnz < a.s_max || mn.alpha != 0.0)) {
      // add / adjust support point i (Eqs. 6-8)
      i = mn.i;
      kind = 1;
      const double Fi = mn.y > 0 ? mn.v : -mn.v;
      const double by = mn.y > 0 ? a.beta : -1.0;  // b_i y_i, b_i = beta^(0.5 (y_i + 1))
      delta = __dsub_rn(by, Fi);
      coef = delta;
      const double anew = __dadd_rn(mn.alpha, delta);
      nnz += (anew != 0.0) - (mn.alpha != 0.0);
      if ((i & (kTrainThreads - 1)) == tid) alpha[i] = anew;
      ++adds;
    } else if (mx.i != INT_MAX && mx.v > 0.0) {
      // remove redundant support point i
      i = mx.i;
      kind = 2;
      coef = -mx.alpha;
      delta = -mx.alpha;
      if ((i & (kTrainThreads - 1)) == tid) alpha[i] = 0.0;
      --nnz;
      ++removes;
    } else {
      converged = 1;
      break;
    }
    ++iters;
    if (tid == 0 && a.trace_kind) {
      a.trace_kind[iter - 1] = (int8_t)kind;
      a.trace_idx[iter - 1] = i;
      a.trace_delta[iter - 1] = delta;
    }
    const double *row = a.G + (int64_t)i * N;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int j = tid + kTrainThreads * k;
      if (j < N) {
        const double g = row[j];
        // F += delta K e_i (add) or F -= alpha_i K e_i (removal)
        F[k] = kind == 1 ? __dadd_rn(F[k], __dmul_rn(coef, g)) : __dsub_rn(F[k], __dmul_rn(mx.alpha, g));
      }
    }
    reduce_candidates(mn, mx);
  }

  // write back alpha and F (warm starts reuse them)
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int j = tid + kTrainThreads * k;
    if (j < N) {
      a.F[j] = F[k];
      a.alpha[j] = alpha[j];
    }
  }
  // removeNonsupportPoints: ascending indices with alpha != 0
  int base = 0;
  for (int c0 = 0; c0 < N; c0 += kTrainThreads) {
    const int j = c0 + tid;
    const bool keep = j < N && alpha[j] != 0.0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kTrainWarps; ++w) {
      const int t = tot[w];
      before += w < warp ? t : 0;
      total += t;
    }
    if (keep) {
      const int pos = base + before + __popc(bal & ((1u << lane) - 1u));
      a.sup_idx[pos] = j;
      a.sup_alpha[pos] = alpha[j];
    }
    base += total;
    __syncthreads();
  }
  if (tid == 0) {
    a.stats[0] = iters;
    a.stats[1] = adds;
    a.stats[2] = removes;
    a.stats[3] = converged;
    a.stats[4] = base;
  }
}

template <int KMAX>
static cudaError_t launch_k(const TrainArgs &a, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)a.N;
  cudaError_t e =
      cudaFuncSetAttribute(fastron_train_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fastron_train_kernel<KMAX><<<1, kTrainThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fastron_train(const TrainArgs &a, cudaStream_t s) {
  if (a.N <= 1 * kTrainThreads) return launch_k<1>(a, s);
  if (a.N <= 2 * kTrainThreads) return launch_k<2>(a, s);
  if (a.N <= 4 * kTrainThreads) return launch_k<4>(a, s);
  if (a.N <= 8 * kTrainThreads) return launch_k<8>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace fk
