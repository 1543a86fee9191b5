// C ABI of libfkfast.so (include/fkfast.h): argument checking, handle and
// workspace management, and the launch sequence of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fk_internal.h"
#include "tc_gemm.cuh"

namespace fk {
struct GemmArgs;
cudaError_t launch_gemm_f32(const GemmArgs &g, int splits, cudaStream_t s);
bool score_supported(int mv);
int probe_iters(int kind);
int probe_ops_per_iter(int kind);
}  // namespace fk

using namespace fk;

// ------------------------------------------------------------- errors ---
static thread_local char g_err[512] = "";

static int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(FK_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char *fk_last_error(void) { return g_err; }

// Device buffer that only grows.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) {
      cudaError_t e = cudaFree(p);
      if (e != cudaSuccess) return e;
      p = nullptr;
      cap = 0;
    }
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T>
  T *as() const {
    return reinterpret_cast<T *>(p);
  }
};

// --------------------------------------------------------------- chain ---
struct fk_chain {
  int D = 0, M = 0;
  ChainF cf{};
  ChainD cd{};
  DevBuf ws_a, ws_b;  // control-point workspaces of fk_gram
};

extern "C" int fk_chain_create(const fk_dh *dh, int D, const double *base4x4, const fk_cp *cps, int M,
                               fk_chain_t **out) {
  if (!out) return fail(FK_ERR_ARG, "fk_chain_create: out is NULL");
  *out = nullptr;
  if (!dh || !cps) return fail(FK_ERR_ARG, "fk_chain_create: dh and cps must not be NULL");
  if (D < 1 || D > FK_MAX_DOF) return fail(FK_ERR_ARG, "fk_chain_create: D=%d outside [1, %d]", D, FK_MAX_DOF);
  if (M < 1 || M > FK_MAX_CP) return fail(FK_ERR_ARG, "fk_chain_create: M=%d outside [1, %d]", M, FK_MAX_CP);
  double base[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  if (base4x4) memcpy(base, base4x4, sizeof base);
  if (base[12] != 0.0 || base[13] != 0.0 || base[14] != 0.0 || base[15] != 1.0)
    return fail(FK_ERR_ARG, "fk_chain_create: the last row of base4x4 must be (0, 0, 0, 1)");
  for (int i = 0; i < D; ++i) {
    if (dh[i].type != FK_REVOLUTE && dh[i].type != FK_PRISMATIC)
      return fail(FK_ERR_ARG, "fk_chain_create: link %d has unknown type %d", i, dh[i].type);
    if (!std::isfinite(dh[i].a) || !std::isfinite(dh[i].alpha) || !std::isfinite(dh[i].d) ||
        !std::isfinite(dh[i].theta0))
      return fail(FK_ERR_ARG, "fk_chain_create: link %d has a non-finite parameter", i);
  }
  int mv = 0, nconst = 0;
  for (int m = 0; m < M; ++m) {
    if (cps[m].joint < 0 || cps[m].joint > D)
      return fail(FK_ERR_ARG, "fk_chain_create: control point %d on frame %d outside [0, %d]", m, cps[m].joint, D);
    if (cps[m].joint == 0)
      ++nconst;
    else
      ++mv;
  }
  fk_chain *c = new fk_chain;
  c->D = D;
  c->M = M;
  ChainF &f = c->cf;
  ChainD &d = c->cd;
  f.D = d.D = D;
  f.M = d.M = M;
  f.Mv = d.Mv = mv;
  f.n_const = d.n_const = nconst;
  for (int i = 0; i < D; ++i) {
    const double ca = cos(dh[i].alpha), sa = sin(dh[i].alpha);
    d.type[i] = f.type[i] = dh[i].type;
    d.a[i] = dh[i].a;
    d.ca[i] = ca;
    d.sa[i] = sa;
    d.d[i] = dh[i].d;
    d.th0[i] = dh[i].theta0;
    f.a[i] = (float)dh[i].a;
    f.ca[i] = (float)ca;
    f.sa[i] = (float)sa;
    f.d[i] = (float)dh[i].d;
    f.th0[i] = (float)dh[i].theta0;
  }
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 4; ++k) d.T0[4 * r + k] = base[4 * r + k];
    for (int k = 0; k < 3; ++k) f.R0[3 * r + k] = (float)base[4 * r + k];
    f.p0[r] = (float)base[4 * r + 3];
  }
  int v = 0;
  for (int m = 0; m < M; ++m) {
    d.cj[m] = f.cj[m] = cps[m].joint;
    for (int r = 0; r < 3; ++r) {
      d.ct[m][r] = cps[m].t[r];
      f.ct[m][r] = (float)cps[m].t[r];
    }
    if (cps[m].joint != 0) {
      f.vj[v] = cps[m].joint;
      f.vidx[v] = d.vidx[v] = m;
      for (int r = 0; r < 3; ++r) f.vt[v][r] = (float)cps[m].t[r];
      ++v;
    }
  }
  *out = c;
  return FK_OK;
}

extern "C" void fk_chain_destroy(fk_chain_t *c) {
  if (!c) return;
  c->ws_a.release();
  c->ws_b.release();
  delete c;
}

// ------------------------------------------------------------ forward ---
extern "C" int fk_forward(const fk_chain_t *c, const float *q, int64_t n, float *cp, void *stream) {
  if (!c) return fail(FK_ERR_ARG, "fk_forward: chain is NULL");
  if (n < 0) return fail(FK_ERR_ARG, "fk_forward: n < 0");
  if (n == 0) return FK_OK;
  if (!q || !cp) return fail(FK_ERR_ARG, "fk_forward: q and cp must not be NULL");
  CK(launch_fk_forward_f32(c->cf, q, n, cp, (cudaStream_t)stream));
  return FK_OK;
}

extern "C" int fk_forward_f64(const fk_chain_t *c, const double *q, int64_t n, double *cp, void *stream) {
  if (!c) return fail(FK_ERR_ARG, "fk_forward_f64: chain is NULL");
  if (n < 0) return fail(FK_ERR_ARG, "fk_forward_f64: n < 0");
  if (n == 0) return FK_OK;
  if (!q || !cp) return fail(FK_ERR_ARG, "fk_forward_f64: q and cp must not be NULL");
  CK(launch_fk_forward_f64(c->cd, q, n, cp, (cudaStream_t)stream));
  return FK_OK;
}

// --------------------------------------------------------------- gram ---
extern "C" int fk_gram(const fk_chain_t *cc, const void *Xa, int64_t na, const void *Xb, int64_t nb, double gamma,
                       int precision, void *K, void *stream) {
  fk_chain *c = const_cast<fk_chain *>(cc);
  if (!c) return fail(FK_ERR_ARG, "fk_gram: chain is NULL");
  if (na < 0 || nb < 0) return fail(FK_ERR_ARG, "fk_gram: negative size");
  if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(FK_ERR_ARG, "fk_gram: gamma must be finite and > 0");
  if (precision != FK_F32 && precision != FK_F64) return fail(FK_ERR_ARG, "fk_gram: unknown precision %d", precision);
  if (na == 0 || nb == 0) return FK_OK;
  if (!Xa || !Xb || !K) return fail(FK_ERR_ARG, "fk_gram: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const bool sym = Xa == Xb && na == nb;
  const size_t el = precision == FK_F64 ? sizeof(double) : sizeof(float);
  CK(c->ws_a.ensure(el * (size_t)c->M * 3 * (size_t)na));
  if (!sym) CK(c->ws_b.ensure(el * (size_t)c->M * 3 * (size_t)nb));
  if (precision == FK_F64) {
    double *A = c->ws_a.as<double>(), *B = sym ? A : c->ws_b.as<double>();
    CK(launch_fk_forward_f64(c->cd, (const double *)Xa, na, A, s));
    if (!sym) CK(launch_fk_forward_f64(c->cd, (const double *)Xb, nb, B, s));
    CK(launch_gram_f64(c->cd, gamma, A, na, B, nb, sym, (double *)K, s));
  } else {
    float *A = c->ws_a.as<float>(), *B = sym ? A : c->ws_b.as<float>();
    CK(launch_fk_forward_f32(c->cf, (const float *)Xa, na, A, s));
    if (!sym) CK(launch_fk_forward_f32(c->cf, (const float *)Xb, nb, B, s));
    CK(launch_gram_f32(c->cd, (float)gamma, A, na, B, nb, sym, (float *)K, s));
  }
  return FK_OK;
}

// -------------------------------------------------------------- model ---
static constexpr int64_t kMaxTrainN = 8192;
static constexpr double kDefaultEps = 6e-6;
static constexpr uint32_t kDefaultWaitLimit = 1u << 22;  // about a quarter second of polling
static uint32_t g_wait_limit = kDefaultWaitLimit;

extern "C" void fk_set_wait_limit(uint32_t polls) { g_wait_limit = polls; }

struct fastron_model {
  const fk_chain *chain = nullptr;
  // training state (full training set)
  int64_t N = 0;
  DevBuf cpX, G, alpha, F, stats, sup_idx, sup_alpha, trace_kind, trace_idx, trace_delta;
  int64_t trace_len = 0;
  // support set packed for scoring
  int64_t ns = -1;  // -1 = untrained
  double gamma = 0.0;
  DevBuf rec, cp64, alpha_s, q_s, qin;
  std::vector<int64_t> host_idx;  // training indices of the support points (model_set: positions)
  bool host_idx_valid = false;
  // score scratch
  DevBuf band_idx, flags;  // flags: [0] band count, [1] error bits
};

extern "C" int fastron_model_create(const fk_chain_t *chain, fastron_model_t **out) {
  if (!out) return fail(FK_ERR_ARG, "fastron_model_create: out is NULL");
  *out = nullptr;
  if (!chain) return fail(FK_ERR_ARG, "fastron_model_create: chain is NULL");
  if (!score_supported(chain->cf.Mv))
    return fail(FK_ERR_ARG, "fastron_model_create: %d configuration-dependent control points is not a compiled shape",
                chain->cf.Mv);
  fastron_model *m = new fastron_model;
  m->chain = chain;
  *out = m;
  return FK_OK;
}

extern "C" void fastron_model_destroy(fastron_model_t *m) {
  if (!m) return;
  DevBuf *bufs[] = {&m->cpX, &m->G, &m->alpha, &m->F, &m->stats, &m->sup_idx, &m->sup_alpha, &m->trace_kind,
                    &m->trace_idx, &m->trace_delta, &m->rec, &m->cp64, &m->alpha_s, &m->q_s, &m->qin,
                    &m->band_idx, &m->flags};
  for (DevBuf *b : bufs) b->release();
  delete m;
}

static int pack(fastron_model *m, const double *X, const int32_t *idx, const double *alpha, int64_t ns, double gamma,
                cudaStream_t s) {
  const fk_chain *c = m->chain;
  CK(m->rec.ensure(sizeof(float4) * (size_t)((ns + 1) / 2 > 0 ? (ns + 1) / 2 : 1) * rec_len(c->cf.Mv)));
  CK(m->cp64.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * c->M * 3));
  CK(m->alpha_s.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1)));
  CK(m->q_s.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * c->D));
  PackArgs pa{X, idx, alpha, ns, gamma, m->rec.as<float4>(), m->cp64.as<double>(), m->alpha_s.as<double>(),
              m->q_s.as<double>()};
  CK(launch_pack_support(c->cf, c->cd, pa, s));
  m->ns = ns;
  m->gamma = gamma;
  return FK_OK;
}

extern "C" int fastron_train(fastron_model_t *m, const double *X, const int8_t *y, int64_t N, const fastron_params *p,
                             fastron_stats *st, void *stream) {
  if (!m) return fail(FK_ERR_ARG, "fastron_train: model is NULL");
  if (!X || !y || !p) return fail(FK_ERR_ARG, "fastron_train: NULL pointer");
  if (N < 1) return fail(FK_ERR_ARG, "fastron_train: N must be >= 1");
  if (N > kMaxTrainN) return fail(FK_ERR_CAPACITY, "fastron_train: N=%lld exceeds %lld", (long long)N, (long long)kMaxTrainN);
  if (!(p->gamma > 0.0) || !std::isfinite(p->gamma)) return fail(FK_ERR_ARG, "fastron_train: gamma must be finite and > 0");
  if (!(p->beta >= 1.0) || !std::isfinite(p->beta)) return fail(FK_ERR_ARG, "fastron_train: beta must be >= 1");
  if (p->iter_max < 0) return fail(FK_ERR_ARG, "fastron_train: iter_max < 0");
  if (p->s_max < 1) return fail(FK_ERR_ARG, "fastron_train: s_max < 1");
  if (p->warm_start && (m->N != N || m->alpha.p == nullptr))
    return fail(FK_ERR_STATE, "fastron_train: warm start needs a previous training call with the same N");
  cudaStream_t s = (cudaStream_t)stream;
  const fk_chain *c = m->chain;
  const bool keep = p->warm_start != 0;
  CK(m->cpX.ensure(sizeof(double) * (size_t)N * c->M * 3));
  CK(m->G.ensure(sizeof(double) * (size_t)N * (size_t)N));
  if (!keep) {
    CK(m->alpha.ensure(sizeof(double) * (size_t)N));
    CK(m->F.ensure(sizeof(double) * (size_t)N));
    CK(cudaMemsetAsync(m->alpha.p, 0, sizeof(double) * (size_t)N, s));
    CK(cudaMemsetAsync(m->F.p, 0, sizeof(double) * (size_t)N, s));
  }
  CK(m->stats.ensure(sizeof(int64_t) * 5));
  CK(m->sup_idx.ensure(sizeof(int32_t) * (size_t)N));
  CK(m->sup_alpha.ensure(sizeof(double) * (size_t)N));
  const bool trace = p->trace != 0;
  if (trace) {
    const size_t L = (size_t)(p->iter_max > 0 ? p->iter_max : 1);
    CK(m->trace_kind.ensure(L));
    CK(m->trace_idx.ensure(sizeof(int32_t) * L));
    CK(m->trace_delta.ensure(sizeof(double) * L));
  }
  m->N = N;
  CK(launch_fk_forward_f64(c->cd, X, N, m->cpX.as<double>(), s));
  CK(launch_gram_f64(c->cd, p->gamma, m->cpX.as<double>(), N, m->cpX.as<double>(), N, 1, m->G.as<double>(), s));
  TrainArgs ta{m->G.as<double>(), y, N, p->beta, p->iter_max, p->s_max, m->alpha.as<double>(), m->F.as<double>(),
               m->stats.as<int64_t>(), m->sup_idx.as<int32_t>(), m->sup_alpha.as<double>(),
               trace ? m->trace_kind.as<int8_t>() : nullptr, trace ? m->trace_idx.as<int32_t>() : nullptr,
               trace ? m->trace_delta.as<double>() : nullptr};
  CK(launch_fastron_train(ta, s));
  int64_t hs[5];
  CK(cudaMemcpyAsync(hs, m->stats.p, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  m->trace_len = trace ? hs[0] : 0;
  int rc = pack(m, X, m->sup_idx.as<int32_t>(), m->sup_alpha.as<double>(), hs[4], p->gamma, s);
  if (rc != FK_OK) return rc;
  m->host_idx_valid = false;
  if (st) {
    st->iterations = hs[0];
    st->adds = hs[1];
    st->removes = hs[2];
    st->converged = (int32_t)hs[3];
    st->n_support = hs[4];
    st->reserved = 0;
  }
  return FK_OK;
}

extern "C" int fastron_model_trace(const fastron_model_t *m, int8_t *kind, int64_t *idx, double *delta, int64_t cap,
                                   int64_t *n) {
  if (!m || !n) return fail(FK_ERR_ARG, "fastron_model_trace: NULL pointer");
  *n = m->trace_len;
  const int64_t k = m->trace_len < cap ? m->trace_len : cap;
  if (k <= 0) return FK_OK;
  std::vector<int32_t> tmp((size_t)k);
  if (kind) CK(cudaMemcpy(kind, m->trace_kind.p, (size_t)k, cudaMemcpyDeviceToHost));
  if (idx) {
    CK(cudaMemcpy(tmp.data(), m->trace_idx.p, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < k; ++i) idx[i] = tmp[(size_t)i];
  }
  if (delta) CK(cudaMemcpy(delta, m->trace_delta.p, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost));
  return FK_OK;
}

extern "C" int fastron_model_set(fastron_model_t *m, const double *q, const double *alpha, int64_t ns, double gamma) {
  if (!m) return fail(FK_ERR_ARG, "fastron_model_set: model is NULL");
  if (ns < 0) return fail(FK_ERR_ARG, "fastron_model_set: ns < 0");
  if (ns > 0 && (!q || !alpha)) return fail(FK_ERR_ARG, "fastron_model_set: NULL pointer");
  if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(FK_ERR_ARG, "fastron_model_set: gamma must be finite and > 0");
  const fk_chain *c = m->chain;
  CK(m->qin.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * (c->D + 1)));
  double *dq = m->qin.as<double>(), *da = dq + (size_t)ns * c->D;
  if (ns > 0) {
    CK(cudaMemcpy(dq, q, sizeof(double) * (size_t)ns * c->D, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(da, alpha, sizeof(double) * (size_t)ns, cudaMemcpyHostToDevice));
  }
  int rc = pack(m, dq, nullptr, da, ns, gamma, 0);
  if (rc != FK_OK) return rc;
  CK(cudaStreamSynchronize(0));
  m->host_idx.resize((size_t)ns);
  for (int64_t i = 0; i < ns; ++i) m->host_idx[(size_t)i] = i;
  m->host_idx_valid = true;
  return FK_OK;
}

extern "C" int fastron_model_get(const fastron_model_t *cm, int64_t *idx, double *alpha, int64_t cap, int64_t *ns) {
  fastron_model *m = const_cast<fastron_model *>(cm);
  if (!m || !ns) return fail(FK_ERR_ARG, "fastron_model_get: NULL pointer");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fastron_model_get: model is untrained");
  *ns = m->ns;
  const int64_t k = m->ns < cap ? m->ns : cap;
  if (k <= 0) return FK_OK;
  CK(cudaDeviceSynchronize());
  if (alpha) CK(cudaMemcpy(alpha, m->alpha_s.p, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost));
  if (idx) {
    if (m->host_idx_valid) {
      for (int64_t i = 0; i < k; ++i) idx[i] = m->host_idx[(size_t)i];
    } else {
      std::vector<int32_t> tmp((size_t)k);
      CK(cudaMemcpy(tmp.data(), m->sup_idx.p, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < k; ++i) idx[i] = tmp[(size_t)i];
    }
  }
  return FK_OK;
}

// -------------------------------------------------------------- score ---
extern "C" int fk_score(fastron_model_t *m, const float *q, int64_t n, int precision, int rescore, double rescore_eps,
                        float *f, int8_t *label, int64_t *n_rescored, void *stream) {
  if (!m) return fail(FK_ERR_ARG, "fk_score: model is NULL");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_score: model is untrained");
  if (n < 0) return fail(FK_ERR_ARG, "fk_score: n < 0");
  if (n > (int64_t)INT32_MAX) return fail(FK_ERR_CAPACITY, "fk_score: n exceeds 2^31 - 1");
  if (precision != FK_F32) return fail(FK_ERR_ARG, "fk_score: unsupported precision %d", precision);
  if (n_rescored) *n_rescored = 0;
  if (n == 0) return FK_OK;
  if (!q || !label) return fail(FK_ERR_ARG, "fk_score: q and label must not be NULL");
  if (m->gamma > 1e7) return fail(FK_ERR_ARG, "fk_score: gamma above the FP32 range of the score kernel");
  cudaStream_t s = (cudaStream_t)stream;
  const fk_chain *c = m->chain;
  CK(m->flags.ensure(sizeof(int32_t) * 2));
  CK(cudaMemsetAsync(m->flags.p, 0, sizeof(int32_t) * 2, s));
  int32_t *cnt = m->flags.as<int32_t>(), *err = cnt + 1;
  if (rescore) CK(m->band_idx.ensure(sizeof(int32_t) * (size_t)n));
  const double eps = rescore_eps > 0.0 ? rescore_eps : kDefaultEps;
  ScoreArgs sa{q, n, m->rec.as<float4>(), m->ns, (float)sqrt(0.5 * m->gamma), (float)eps, f, label,
               rescore ? m->band_idx.as<int32_t>() : nullptr, cnt, err, g_wait_limit};
  CK(launch_score_f32(c->cf, sa, s));
  if (rescore) {
    RescoreArgs ra{q, m->band_idx.as<int32_t>(), cnt, n, m->cp64.as<double>(), m->alpha_s.as<double>(), m->ns,
                   m->gamma, f, label};
    CK(launch_rescore_f64(c->cd, ra, s));
  }
  if (n_rescored) {
    int32_t h[2];
    CK(cudaMemcpyAsync(h, m->flags.p, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[1] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score: a shared-memory tile wait timed out");
    *n_rescored = rescore ? h[0] : 0;
  }
  return FK_OK;
}

// -------------------------------------------------------------- label ---
extern "C" int fk_label(const fk_chain_t *c, const double *boxes, int64_t nb, double radius, const float *q, int64_t n,
                        int8_t *y, void *stream) {
  if (!c) return fail(FK_ERR_ARG, "fk_label: chain is NULL");
  if (nb < 0 || nb > kMaxBoxes) return fail(FK_ERR_CAPACITY, "fk_label: nb=%lld outside [0, %d]", (long long)nb, kMaxBoxes);
  if (nb > 0 && !boxes) return fail(FK_ERR_ARG, "fk_label: boxes is NULL");
  if (!(radius >= 0.0) || !std::isfinite(radius)) return fail(FK_ERR_ARG, "fk_label: radius must be finite and >= 0");
  if (n < 0) return fail(FK_ERR_ARG, "fk_label: n < 0");
  if (n == 0) return FK_OK;
  if (!q || !y) return fail(FK_ERR_ARG, "fk_label: q and y must not be NULL");
  Boxes bx{};
  bx.nb = (int)nb;
  bx.r2 = radius * radius;
  for (int64_t b = 0; b < nb; ++b)
    for (int k = 0; k < 6; ++k) bx.b[b][k] = boxes[6 * b + k];
  CK(launch_label(c->cd, bx, q, n, y, (cudaStream_t)stream));
  return FK_OK;
}

// --------------------------------------------------------- tensor GEMM ---
extern "C" int fk_tc_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int M, int N, int K,
                               int splits, float *C, void *stream) {
  if (!A || !B || !C) return fail(FK_ERR_ARG, "fk_tc_gemm_bf16: NULL pointer");
  if (M <= 0 || N <= 0 || K <= 0 || splits <= 0 || M % 128 || N % 64 || K % (64 * splits))
    return fail(FK_ERR_ARG, "fk_tc_gemm_bf16: need M %% 128 == 0, N %% 64 == 0, K %% (64 splits) == 0");
  if (lda < K || ldb < K || lda % 8 || ldb % 8)
    return fail(FK_ERR_ARG, "fk_tc_gemm_bf16: leading dimensions must be >= K and multiples of 8");
  if (((uintptr_t)A | (uintptr_t)B) % 16 || (uintptr_t)C % 16)
    return fail(FK_ERR_ARG, "fk_tc_gemm_bf16: pointers must be 16-byte aligned");
  static DevBuf err;
  CK(err.ensure(sizeof(int32_t)));
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(err.p, 0, sizeof(int32_t), s));
  GemmArgs g{};
  g.A = reinterpret_cast<const bf16 *>(A);
  g.lda = lda;
  g.B = reinterpret_cast<const bf16 *>(B);
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K / splits;
  g.Cf = C;
  g.ldcf = N;
  g.zstride = (int64_t)M * N;
  g.err = err.as<int32_t>();
  g.wait_limit = g_wait_limit;
  CK(launch_gemm_f32(g, splits, s));
  int32_t h = 0;
  CK(cudaMemcpyAsync(&h, err.p, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_tc_gemm_bf16: an MMA completion wait timed out");
  return FK_OK;
}

// -------------------------------------------------------------- probe ---
extern "C" int fk_probe_pipe(int kind, double *ops_per_clk_sm, double *seconds) {
  if (kind < 0 || kind > 9) return fail(FK_ERR_ARG, "fk_probe_pipe: unknown kind %d", kind);
  if (!ops_per_clk_sm) return fail(FK_ERR_ARG, "fk_probe_pipe: NULL pointer");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 4;
  long long *rec = nullptr;
  CK(cudaMalloc(&rec, sizeof(long long) * 3 * blocks));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(launch_probe(kind, blocks, threads, rec, 0));  // warm-up
  CK(cudaEventRecord(e0, 0));
  CK(launch_probe(kind, blocks, threads, rec, 0));
  CK(cudaEventRecord(e1, 0));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  std::vector<long long> h((size_t)3 * blocks);
  CK(cudaMemcpy(h.data(), rec, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost));
  cudaFree(rec);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // per SM: lane-ops of its blocks / (last end - first start)
  std::vector<long long> lo((size_t)sms + 64, -1), hi((size_t)sms + 64, -1);
  std::vector<int> nblk((size_t)sms + 64, 0);
  for (int b = 0; b < blocks; ++b) {
    const long long sm = h[3 * b], t0 = h[3 * b + 1], t1 = h[3 * b + 2];
    if (sm < 0 || sm >= (long long)lo.size()) continue;
    if (lo[sm] < 0 || t0 < lo[sm]) lo[sm] = t0;
    if (hi[sm] < 0 || t1 > hi[sm]) hi[sm] = t1;
    ++nblk[sm];
  }
  const double per_block = (double)threads * probe_iters(kind) * probe_ops_per_iter(kind);
  double sum = 0.0;
  int used = 0;
  for (size_t i = 0; i < lo.size(); ++i)
    if (nblk[i] > 0 && hi[i] > lo[i]) {
      sum += per_block * nblk[i] / (double)(hi[i] - lo[i]);
      ++used;
    }
  *ops_per_clk_sm = used ? sum / used : 0.0;
  if (seconds) *seconds = ms * 1e-3;
  return FK_OK;
}

// ------------------------------------------------- score, no allocation ---
// Some callers cannot allocate device memory at the time they score: a
// real-time planner loop that must never block on the allocator, a host
// process that hands the GPU over to a pre-sized memory pool, or code
// running under a memory budget fixed at start-up.  fk_score may grow the
// model's band-list buffer with cudaMalloc on its first call with a larger
// batch; fk_score_noalloc never does.  Its scratch (the band counter, the
// error word and the band index list) is the file-scope device array below,
// which every GPU that loads this library holds until the process exits.
constexpr int64_t kNoAllocMaxQueries = 1 << 20;  // 4 MiB of band indices
constexpr int kNoAllocHeader = 64;               // [0] band count, [1] error bits, rest padding

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocHeader + kNoAllocMaxQueries];

// Device address of g_noalloc_scratch per device ordinal, looked up on the
// first call made with that device current.  In host code the array's name
// only stands in for the symbol; handing it to a kernel would reach the wrong
// memory, so kernels get the address found here.
static constexpr int kNoAllocMaxDevices = 64;
static int32_t *g_noalloc_ptr[kNoAllocMaxDevices] = {};
static std::mutex g_noalloc_mu;

static int noalloc_scratch(int32_t **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(FK_ERR_CAPACITY, "fk_score_noalloc: device ordinal %d above %d", dev, kNoAllocMaxDevices - 1);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return FK_OK;
}

extern "C" int fk_score_noalloc(fastron_model_t *m, const float *q, int64_t n, double rescore_eps, float *f,
                                int8_t *label, int64_t *n_rescored, void *stream) {
  if (!m) return fail(FK_ERR_ARG, "fk_score_noalloc: model is NULL");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_score_noalloc: model is untrained");
  if (n < 0) return fail(FK_ERR_ARG, "fk_score_noalloc: n < 0");
  if (n > kNoAllocMaxQueries)
    return fail(FK_ERR_CAPACITY, "fk_score_noalloc: n=%lld exceeds the fixed scratch of %lld queries per call",
                (long long)n, (long long)kNoAllocMaxQueries);
  if (n_rescored) *n_rescored = 0;
  if (n == 0) return FK_OK;
  if (!q || !label) return fail(FK_ERR_ARG, "fk_score_noalloc: q and label must not be NULL");
  if (m->gamma > 1e7) return fail(FK_ERR_ARG, "fk_score_noalloc: gamma above the FP32 range of the score kernel");
  int32_t *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != FK_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const fk_chain *c = m->chain;
  int32_t *cnt = scratch, *err = scratch + 1, *band = scratch + kNoAllocHeader;
  // the array keeps the previous call's contents: the counter and the error
  // word must start at zero (the band list is written before it is read)
  CK(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 2, s));
  const double eps = rescore_eps > 0.0 ? rescore_eps : kDefaultEps;
  ScoreArgs sa{q, n, m->rec.as<float4>(), m->ns, (float)sqrt(0.5 * m->gamma), (float)eps, f, label,
               band, cnt, err, g_wait_limit};
  CK(launch_score_f32(c->cf, sa, s));
  RescoreArgs ra{q, band, cnt, n, m->cp64.as<double>(), m->alpha_s.as<double>(), m->ns, m->gamma, f, label};
  CK(launch_rescore_f64(c->cd, ra, s));
  if (n_rescored) {
    int32_t h[2];
    CK(cudaMemcpyAsync(h, scratch, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[1] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score_noalloc: a shared-memory tile wait timed out");
    *n_rescored = h[0];
  }
  return FK_OK;
}
