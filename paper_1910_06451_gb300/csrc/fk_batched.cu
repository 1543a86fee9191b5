// Many independent scenes (own chain, own support set, own query batch) in
// one persistent launch.  Work items are (scene, block of queries); the host
// sorts them by cost, |S_scene| x queries, longest first, and CTAs take them
// in that order from an atomic counter, so the long items start first and the
// short ones fill the tail.  Each item stages its scene's chain in shared
// memory and runs the same score_block as the per-call kernel; the band
// queries of every scene are then re-scored in double-float by one launch
// (one warp per band query, the lanes over the scene's support set) and
// those it cannot decide in FP64 by another.  Band sizes stay on the device,
// so the whole sequence is one CUDA graph.
#include <cstring>

#include "df_arith.cuh"
#include "fk_internal.h"
#include "fk_ptx.cuh"
#include "score_core.cuh"

namespace fk {

// Per-scene description in device memory.
struct SceneDev {
  ChainF cf;
  ChainD cd;
  const float4 *rec;
  const float *sdf;    // double-float records [ns][rec_df_len(Mv)]
  const double *cp64;
  const double *alpha;
  int64_t ns;     // support points
  int64_t nrec;   // record halves, 2 rec_pairs(ns)
  const int32_t *npair_pos;  // device: [0] positive-weight pairs, which lead the records; [1] |s|max bits
  double gs;      // coordinate scale sqrt(gamma/2)
  float eps0, eps1;  // the scene's band (see score_band): eps(q) = eps0 + eps1 (|p(q)| + |s|max)
  float cnorm;       // > 0 in every scene of a batch scored in the circle form (score_circle)
  double gamma;
  int64_t q_off;  // first query of the scene in the concatenated batch
  int64_t n;      // its number of queries
};

struct WorkItem {
  int32_t scene;
  int32_t block;  // block of NTHR * Q queries within the scene
};

struct BatchArgs {
  const SceneDev *scenes;
  const WorkItem *items;
  int32_t n_items;
  int32_t *counter;
  const float *q;
  float *f;
  int8_t *label;
  int32_t *band_idx;
  int32_t *band_scene;
  int32_t *band_cnt;
  int32_t *err;
  uint32_t wait_limit;
  int circ;  // every scene's cnorm > 0: the CIRC kernels
};

// MINB: resident CTAs the shape is compiled for (its register budget; 1
// leaves the choice to the compiler).  CIRC: the first control point of
// every scene in the circle form (each scene with its own cnorm).
template <int MV, int Q, int TP, int NTHR, int MINB, bool CIRC>
__global__ void __launch_bounds__(NTHR, MINB) batched_score_kernel(const BatchArgs a) {
  extern __shared__ __align__(128) float4 tiles[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ __align__(16) ChainF cs;
  __shared__ int item_sh;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(a.counter, 1);
    __syncthreads();
    const int it = item_sh;
    if (it >= a.n_items) break;
    const WorkItem w = a.items[it];
    const SceneDev *sc = a.scenes + w.scene;
    {
      const int *src = reinterpret_cast<const int *>(&sc->cf);
      int *dst = reinterpret_cast<int *>(&cs);
      for (int i = tid; i < (int)(sizeof(ChainF) / sizeof(int)); i += NTHR) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t off = sc->q_off;
    const BlockOut o{a.f ? a.f + off : nullptr, a.label + off, sc->eps0, sc->eps1, a.band_idx, a.band_scene, w.scene,
                     off, a.band_cnt, a.err, a.wait_limit, sc->npair_pos, sc->cnorm};
    const double gsd = sc->gs;
    const float gh = __double2float_rn(gsd);
    const bool ok = score_block<MV, Q, TP, NTHR, false, false, 0, CIRC>(cs, sc->rec, sc->nrec, dd{gh, __double2float_rn(gsd - (double)gh)},
                                                 a.q + off * sc->cf.D, sc->n, (int64_t)w.block * (NTHR * Q), o, tiles,
                                                 bar);
    if (!ok) break;   // identical in every thread
    __syncthreads();  // item_sh, cs and the tiles are reused by the next item
  }
}

// Double-float re-score of the band queries of all scenes: one warp per
// entry.  Lane 0 computes the query's control points in FP64; they are split
// into pairs in shared memory; each lane sums the summands (df_rq_term) of
// its share of the support points; a fixed butterfly of two-sums adds the
// lanes.  |f| > eps2 B(q) decides; the rest go to band2 for FP64.
constexpr int kBRescoreWarps = 8;

__global__ void __launch_bounds__(kBRescoreWarps * 32) batched_rescore_df_kernel(const SceneDev *__restrict__ scenes,
                                                                                const float *__restrict__ q,
                                                                                const int32_t *__restrict__ band_idx,
                                                                                const int32_t *__restrict__ band_scene,
                                                                                const int32_t *__restrict__ band_cnt,
                                                                                double eps2, float *__restrict__ f,
                                                                                int8_t *__restrict__ label,
                                                                                int32_t *__restrict__ band2_idx,
                                                                                int32_t *__restrict__ band2_scene,
                                                                                int32_t *__restrict__ band2_cnt) {
  __shared__ double qcp[kBRescoreWarps][FK_MAX_CP][3];
  __shared__ float qd[kBRescoreWarps][FK_MAX_CP][6];  // (h, l) per axis of each configuration-dependent point
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t gw = blockIdx.x * (int64_t)kBRescoreWarps + wl;
  const int64_t nw = (int64_t)gridDim.x * kBRescoreWarps;
  const int64_t cnt = *band_cnt;
  for (int64_t e = gw; e < cnt; e += nw) {
    const int64_t k = band_idx[e];
    const int scene = band_scene[e];
    const SceneDev *sc = scenes + scene;
    const ChainD &c = sc->cd;
    if (lane == 0) {
      PoseD P;
      pose_base(c, P);
      for (int m = 0; m < c.M; ++m)
        if (c.cj[m] == 0) pose_point(P, c.ct[m], qcp[wl][m]);
      for (int i = 0; i < c.D; ++i) {
        pose_step(c, i, (double)q[k * c.D + i], P);
        for (int m = 0; m < c.M; ++m)
          if (c.cj[m] == i + 1) pose_point(P, c.ct[m], qcp[wl][m]);
      }
    }
    __syncwarp();
    const double gs = sqrt(0.5 * sc->gamma);
    for (int i = lane; i < 3 * c.Mv; i += 32) {
      const int v = i / 3, r = i % 3;
      const dfl x = df_from_double(gs * qcp[wl][c.vidx[v]][r]);
      qd[wl][v][2 * r] = x.h;
      qd[wl][v][2 * r + 1] = x.l;
    }
    __syncwarp();
    const int Mv = c.Mv, RL = rec_df_len(Mv);
    const float n_const = (float)c.n_const;
    float fh = 0.f, fl = 0.f, B = 0.f;
    for (int64_t s = lane; s < sc->ns; s += 32) {
      const float *S = sc->sdf + s * RL;
      float kh = n_const, kl = 0.f;
      for (int v = 0; v < Mv; ++v) {
        const float qh[3] = {qd[wl][v][0], qd[wl][v][2], qd[wl][v][4]};
        const float ql[3] = {qd[wl][v][1], qd[wl][v][3], qd[wl][v][5]};
        float rh, rl;
        df_rq_term(qh, ql, S + v * 6, rh, rl);
        const dfl ks = two_sum(kh, rh);
        kh = ks.h;
        kl += ks.l + rl;
      }
      const float wh = S[6 * Mv], wlo = S[6 * Mv + 1];
      const float ph = wh * kh;
      const float pe = fmaf(wh, kl, fmaf(wlo, kh, fmaf(wh, kh, -ph)));
      const dfl fs = two_sum(fh, ph);
      fh = fs.h;
      fl += fs.l + pe;
      B = fmaf(S[6 * Mv + 2], kh, B);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, fh, o), ol = __shfl_xor_sync(0xffffffffu, fl, o);
      const float ob = __shfl_xor_sync(0xffffffffu, B, o);
      // the same operands in the same order in both lanes of a pair (lower lane first)
      const bool low = (lane & o) == 0;
      const dfl t = two_sum(low ? fh : oh, low ? oh : fh);
      fl = t.l + (low ? fl + ol : ol + fl);
      fh = t.h;
      B = low ? B + ob : ob + B;
    }
    if (lane == 0) {
      const double fv = (double)fh + (double)fl;
      if (fabs(fv) > eps2 * (double)B) {
        if (f) f[k] = (float)fv;
        label[k] = fv >= 0.0 ? 1 : -1;
      } else {
        const int pos = atomicAdd(band2_cnt, 1);
        band2_idx[pos] = (int32_t)k;
        band2_scene[pos] = scene;
      }
    }
    __syncwarp();
  }
}

// FP64 re-score of the entries the double-float pass left: one warp per entry.

__global__ void __launch_bounds__(kBRescoreWarps * 32) batched_rescore_kernel(const SceneDev *__restrict__ scenes,
                                                                             const float *__restrict__ q,
                                                                             const int32_t *__restrict__ band_idx,
                                                                             const int32_t *__restrict__ band_scene,
                                                                             const int32_t *__restrict__ band_cnt,
                                                                             float *__restrict__ f,
                                                                             int8_t *__restrict__ label) {
  __shared__ double qcp[kBRescoreWarps][FK_MAX_CP][3];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t gw = blockIdx.x * (int64_t)kBRescoreWarps + wl;
  const int64_t nw = (int64_t)gridDim.x * kBRescoreWarps;
  const int64_t cnt = *band_cnt;
  for (int64_t e = gw; e < cnt; e += nw) {
    const int64_t k = band_idx[e];
    const SceneDev *sc = scenes + band_scene[e];
    const ChainD &c = sc->cd;
    if (lane == 0) {
      PoseD P;
      pose_base(c, P);
      for (int m = 0; m < c.M; ++m)
        if (c.cj[m] == 0) pose_point(P, c.ct[m], qcp[wl][m]);
      for (int i = 0; i < c.D; ++i) {
        pose_step(c, i, (double)q[k * c.D + i], P);
        for (int m = 0; m < c.M; ++m)
          if (c.cj[m] == i + 1) pose_point(P, c.ct[m], qcp[wl][m]);
      }
    }
    __syncwarp();
    const double hg = 0.5 * sc->gamma, invM = 1.0 / c.M;
    const int64_t ns = sc->ns;
    double acc = 0.0;
    for (int64_t s = lane; s < ns; s += 32) {
      double ks = (double)c.n_const;
      for (int v = 0; v < c.Mv; ++v) {
        const int m = c.vidx[v];
        const double sp[3] = {sc->cp64[(m * 3 + 0) * ns + s], sc->cp64[(m * 3 + 1) * ns + s],
                              sc->cp64[(m * 3 + 2) * ns + s]};
        ks += k_rq_f64(hg, sp, qcp[wl][m]);
      }
      acc = fma(sc->alpha[s] * invM, ks, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (f) f[k] = (float)acc;
      label[k] = acc >= 0.0 ? 1 : -1;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- variants ---
// Tile shapes the autotuner chooses among: queries per thread, support pairs
// per shared-memory tile, threads per CTA, CTAs per SM compiled for (the last
// shape: one query per thread with the register budget of 3 CTAs per SM).
struct Variant {
  int Q, TP, NTHR, MINB;
};
constexpr Variant kVariants[] = {{2, 64, 256, 1}, {1, 64, 256, 1}, {2, 32, 256, 1},
                                 {2, 128, 256, 1}, {1, 32, 128, 1}, {1, 64, 256, 3}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int batched_num_variants() { return kNumVariants; }
int batched_block_queries(int v) { return kVariants[v].Q * kVariants[v].NTHR; }

template <int MV, int Q, int TP, int NTHR, int MINB>
static cudaError_t launch_bv(const BatchArgs &a, cudaStream_t s, bool prepare_only) {
  // the circle form is compiled for 7 and 11 points (the 3-point arms'
  // scenes take the direct form)
  constexpr bool kCirc = MV == 7 || MV == 11;
  auto kern = kCirc && a.circ ? batched_score_kernel<MV, Q, TP, NTHR, MINB, kCirc>
                              : batched_score_kernel<MV, Q, TP, NTHR, MINB, false>;
  const size_t smem = 2 * (size_t)TP * rec_len(MV) * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess || prepare_only) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTHR, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > a.n_items) grid = a.n_items > 0 ? a.n_items : 1;
  kern<<<grid, NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MV>
static cudaError_t launch_bmv(int v, const BatchArgs &a, cudaStream_t s, bool prep) {
  switch (v) {
    case 0: return launch_bv<MV, 2, 64, 256, 1>(a, s, prep);
    case 1: return launch_bv<MV, 1, 64, 256, 1>(a, s, prep);
    case 2: return launch_bv<MV, 2, 32, 256, 1>(a, s, prep);
    case 3: return launch_bv<MV, 2, 128, 256, 1>(a, s, prep);
    case 4: return launch_bv<MV, 1, 32, 128, 1>(a, s, prep);
    case 5: return launch_bv<MV, 1, 64, 256, 3>(a, s, prep);
    default: return cudaErrorInvalidValue;
  }
}

bool batched_supported(int mv) { return mv == 3 || mv == 7 || mv == 11; }

cudaError_t launch_batched_score(int mv, int variant, const BatchArgs &a, cudaStream_t s, bool prepare_only) {
  switch (mv) {
    case 3: return launch_bmv<3>(variant, a, s, prepare_only);
    case 7: return launch_bmv<7>(variant, a, s, prepare_only);
    case 11: return launch_bmv<11>(variant, a, s, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batched_rescore_df(const SceneDev *scenes, const float *q, const int32_t *band_idx,
                                      const int32_t *band_scene, const int32_t *band_cnt, double eps2, float *f,
                                      int8_t *label, int32_t *band2_idx, int32_t *band2_scene, int32_t *band2_cnt,
                                      cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  batched_rescore_df_kernel<<<(unsigned)(sms > 0 ? 4 * sms : 608), kBRescoreWarps * 32, 0, s>>>(
      scenes, q, band_idx, band_scene, band_cnt, eps2, f, label, band2_idx, band2_scene, band2_cnt);
  return cudaGetLastError();
}

cudaError_t launch_batched_rescore(const SceneDev *scenes, const float *q, const int32_t *band_idx,
                                   const int32_t *band_scene, const int32_t *band_cnt, float *f, int8_t *label,
                                   cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  batched_rescore_kernel<<<(unsigned)(sms > 0 ? 2 * sms : 304), kBRescoreWarps * 32, 0, s>>>(
      scenes, q, band_idx, band_scene, band_cnt, f, label);
  return cudaGetLastError();
}

size_t scene_dev_size() { return sizeof(SceneDev); }
size_t work_item_size() { return sizeof(WorkItem); }

// Host-side filling of a SceneDev record (the layout stays private to this file).
void fill_scene_dev(void *dst, const ChainF &cf, const ChainD &cd, const void *rec, const float *sdf,
                    const double *cp64, const double *alpha, int64_t ns, const int32_t *npair_pos, double gamma,
                    float eps0, float eps1, float cnorm, int64_t q_off, int64_t n) {
  SceneDev d;
  memset(&d, 0, sizeof d);
  d.cf = cf;
  d.cd = cd;
  d.rec = static_cast<const float4 *>(rec);
  d.sdf = sdf;
  d.cp64 = cp64;
  d.alpha = alpha;
  d.ns = ns;
  d.nrec = 2 * rec_pairs(ns);
  d.npair_pos = npair_pos;
  d.gs = sqrt(0.5 * gamma);
  d.eps0 = eps0;
  d.eps1 = eps1;
  d.cnorm = cnorm;
  d.gamma = gamma;
  d.q_off = q_off;
  d.n = n;
  memcpy(dst, &d, sizeof d);
}

void fill_work_item(void *dst, int32_t scene, int32_t block) {
  WorkItem w{scene, block};
  memcpy(dst, &w, sizeof w);
}

cudaError_t launch_batched_score_args(int mv, int variant, const void *scenes, const void *items, int32_t n_items,
                                      int32_t *counter, const float *q, float *f, int8_t *label,
                                      int32_t *band_idx, int32_t *band_scene, int32_t *band_cnt, int32_t *err,
                                      uint32_t wait_limit, int circ, cudaStream_t s, bool prepare_only) {
  BatchArgs a{static_cast<const SceneDev *>(scenes), static_cast<const WorkItem *>(items), n_items, counter, q, f,
              label, band_idx, band_scene, band_cnt, err, wait_limit, circ};
  return launch_batched_score(mv, variant, a, s, prepare_only);
}

cudaError_t launch_batched_rescore_df_args(const void *scenes, const float *q, const int32_t *band_idx,
                                           const int32_t *band_scene, const int32_t *band_cnt, double eps2, float *f,
                                           int8_t *label, int32_t *band2_idx, int32_t *band2_scene,
                                           int32_t *band2_cnt, cudaStream_t s) {
  return launch_batched_rescore_df(static_cast<const SceneDev *>(scenes), q, band_idx, band_scene, band_cnt, eps2, f,
                                   label, band2_idx, band2_scene, band2_cnt, s);
}

cudaError_t launch_batched_rescore_args(const void *scenes, const float *q, const int32_t *band_idx,
                                        const int32_t *band_scene, const int32_t *band_cnt, float *f, int8_t *label,
                                        cudaStream_t s) {
  return launch_batched_rescore(static_cast<const SceneDev *>(scenes), q, band_idx, band_scene, band_cnt, f, label,
                                s);
}

}  // namespace fk
