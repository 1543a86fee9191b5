// C ABI of libfkfast.so (include/fkfast.h): argument checking, handle and
// workspace management, and the launch sequence of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "fk_internal.h"
#include "surr_step.h"
#include "tc_gemm.cuh"

namespace fk {
cudaError_t launch_score_f16(const ChainF &c, const ScoreArgs &a, cudaStream_t s);
bool score_f16_supported(int mv);
cudaError_t launch_gather_rows(const float *q, int D, const int32_t *idx, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_scatter_labels(const int8_t *src, const float *fsrc, const int32_t *idx, int64_t n, int8_t *label,
                                  float *pred, cudaStream_t s);
struct GemmArgs;
cudaError_t launch_gemm_f32(const GemmArgs &g, int splits, cudaStream_t s);
bool score_supported(int mv);
bool score_gauss_supported(int mv);
int probe_iters(int kind);
int probe_ops_per_iter(int kind);
cudaError_t launch_check_rcp(int e_lo, int e_hi, unsigned long long *out, cudaStream_t s);
cudaError_t launch_check_sincos(float hi, double th0, unsigned long long *out, cudaStream_t s);
cudaError_t launch_forward_dd(const ChainF &c, const float *q, int64_t n, double scale, float *cp, cudaStream_t s);
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
  DevBuf ws_a, ws_b;    // control-point workspaces of fk_gram
  DevBuf ws_da, ws_db;  // their double-float splits
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
  f.summand = d.summand = FK_SUMMAND_RQ;
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
    f.a_l[i] = (float)(dh[i].a - (double)f.a[i]);
    f.ca_l[i] = (float)(ca - (double)f.ca[i]);
    f.sa_l[i] = (float)(sa - (double)f.sa[i]);
    f.d_l[i] = (float)(dh[i].d - (double)f.d[i]);
    f.th0_l[i] = (float)(dh[i].theta0 - (double)f.th0[i]);
    f.quarter[i] = fabs((double)f.sa[i]) == 1.0 && fabs(ca) < 0x1p-20;
  }
  double p0n = 0.0, tmax = 0.0;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 4; ++k) d.T0[4 * r + k] = base[4 * r + k];
    for (int k = 0; k < 3; ++k) {
      f.R0[3 * r + k] = (float)base[4 * r + k];
      f.R0_l[3 * r + k] = (float)(base[4 * r + k] - (double)f.R0[3 * r + k]);
    }
    f.p0[r] = (float)base[4 * r + 3];
    f.p0_l[r] = (float)(base[4 * r + 3] - (double)f.p0[r]);
    p0n += base[4 * r + 3] * base[4 * r + 3];
  }
  // lever-arm bound of the chain (metres): base offset, every link's |a| +
  // |d| (a prismatic joint's travel counted up to 2^10), the largest offset
  double reach = sqrt(p0n);
  for (int i = 0; i < D; ++i) reach += fabs(dh[i].a) + fabs(dh[i].d) + (dh[i].type == FK_PRISMATIC ? 1024.0 : 0.0);
  for (int m = 0; m < M; ++m)
    tmax = fmax(tmax, sqrt(cps[m].t[0] * cps[m].t[0] + cps[m].t[1] * cps[m].t[1] + cps[m].t[2] * cps[m].t[2]));
  f.reach = (float)((reach + tmax) * (1.0 + 1e-6));
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
      f.vt_nz[v] = 0;
      for (int r = 0; r < 3; ++r) {
        f.vt[v][r] = (float)cps[m].t[r];
        f.vt_l[v][r] = (float)(cps[m].t[r] - (double)f.vt[v][r]);
        f.vt_nz[v] |= cps[m].t[r] != 0.0;
      }
      if (cps[m].joint == D && f.vt_nz[v]) f.rot_last = 1;
      ++v;
    }
  }
  // Point 0 on frame 1 of a revolute joint 1: its position is
  // p0 + R0 Rz(theta) u with the constant u = (a, 0, d) + Rx(alpha) t (Eq. 1
  // for link 1, then Eq. 2), so it lies on a circle of radius
  // rho = |(u_x, u_y)| about the joint's axis and |p - s| = 2 rho
  // |sin((theta - theta_s) / 2)| for two configurations.
  f.circ = d.circ = 0;
  d.circ_rho = 0.0;
  if (mv > 0 && dh[0].type == FK_REVOLUTE && f.vj[0] == 1) {
    const double *t = cps[f.vidx[0]].t;
    f.circ = d.circ = 1;
    d.circ_rho = hypot(dh[0].a + t[0], d.ca[0] * t[1] - d.sa[0] * t[2]);
  }
  *out = c;
  return FK_OK;
}

extern "C" int fk_chain_set_summand(fk_chain_t *c, int summand) {
  if (!c) return fail(FK_ERR_ARG, "fk_chain_set_summand: chain is NULL");
  if (summand != FK_SUMMAND_RQ && summand != FK_SUMMAND_GAUSS)
    return fail(FK_ERR_ARG, "fk_chain_set_summand: unknown summand %d", summand);
  if (summand == FK_SUMMAND_GAUSS && !score_gauss_supported(c->cf.Mv))
    return fail(FK_ERR_ARG, "fk_chain_set_summand: no Gaussian score kernel for %d control points", c->cf.Mv);
  c->cf.summand = c->cd.summand = summand;
  return FK_OK;
}

extern "C" void fk_chain_destroy(fk_chain_t *c) {
  if (!c) return;
  c->ws_a.release();
  c->ws_b.release();
  c->ws_da.release();
  c->ws_db.release();
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
  if (precision != FK_F32 && precision != FK_F64 && precision != FK_DF64 && precision != FK_DF32)
    return fail(FK_ERR_ARG, "fk_gram: unknown precision %d", precision);
  if (c->cd.summand != FK_SUMMAND_RQ && (precision == FK_DF64 || precision == FK_DF32))
    return fail(FK_ERR_ARG, "fk_gram: the Gaussian summand has no double-float form (use FK_F64 or FK_F32)");
  if (na == 0 || nb == 0) return FK_OK;
  if (!Xa || !Xb || !K) return fail(FK_ERR_ARG, "fk_gram: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const bool sym = Xa == Xb && na == nb;
  const size_t el = precision == FK_F32 ? sizeof(float) : sizeof(double);
  CK(c->ws_a.ensure(el * (size_t)c->M * 3 * (size_t)na));
  if (!sym) CK(c->ws_b.ensure(el * (size_t)c->M * 3 * (size_t)nb));
  if (precision == FK_F64 || precision == FK_DF64 || precision == FK_DF32) {
    double *A = c->ws_a.as<double>(), *B = sym ? A : c->ws_b.as<double>();
    CK(launch_fk_forward_f64(c->cd, (const double *)Xa, na, A, s));
    if (!sym) CK(launch_fk_forward_f64(c->cd, (const double *)Xb, nb, B, s));
    if (precision == FK_F64)
      CK(launch_gram_f64(c->cd, gamma, A, na, B, nb, sym, (double *)K, s));
    else {
      CK(c->ws_da.ensure(sizeof(float2) * (size_t)(c->cd.Mv > 0 ? c->cd.Mv : 1) * 3 * (size_t)na));
      if (!sym) CK(c->ws_db.ensure(sizeof(float2) * (size_t)(c->cd.Mv > 0 ? c->cd.Mv : 1) * 3 * (size_t)nb));
      float2 *wa = c->ws_da.as<float2>(), *wb = sym ? wa : c->ws_db.as<float2>();
      if (precision == FK_DF32)
        CK(launch_gram_df32(c->cd, gamma, A, na, B, nb, sym, (float *)K, wa, wb, s));
      else
        CK(launch_gram_df(c->cd, gamma, A, na, B, nb, sym, (double *)K, wa, wb, s));
    }
  } else {
    float *A = c->ws_a.as<float>(), *B = sym ? A : c->ws_b.as<float>();
    CK(launch_fk_forward_f32(c->cf, (const float *)Xa, na, A, s));
    if (!sym) CK(launch_fk_forward_f32(c->cf, (const float *)Xb, nb, B, s));
    CK(launch_gram_f32(c->cd, (float)gamma, A, na, B, nb, sym, (float *)K, s));
  }
  return FK_OK;
}

// -------------------------------------------------------------- model ---
static constexpr int64_t kMaxTrainN = 65536;
static constexpr double kDefaultEpsDf = 1e-9;  // band of the double-float re-score, relative to B(q)
// Gaussian summand (not the paper's): per-query bands relative to B(q), set
// from measurement, not derived: the measured worst |f - f64| / B(q) over
// 200k queries of the 3- and 7-DOF models is 7.3e-8 (FP32, MUFU or
// polynomial) and 1.8e-4 (half)
static constexpr double kDefaultEpsGauss = 6e-6;
static constexpr double kDefaultEpsF16Gauss = 2e-3;

// ---- the band of the score kernel: a bound on its whole error -----------
// Relative error bound of MUFU rcp.approx.ftz.f32 on normal inputs (one ulp:
// |r x - 1| <= 2^-23), the premise the derivation takes from the PTX ISA;
// a GPU test checks it on every FP32 mantissa over the exponent range the
// kernel uses.
static constexpr double kRcpRel = 0x1p-23;

// The score kernel (score_core.cuh, summand RQ) returns f~ and B~ for f =
// sum_s w_s sum_m k_sm (w_s = alpha_s / M, k = t^-2, t = 1 + |p_m - s_m|^2
// in coordinates scaled by g = sqrt(gamma/2)) and B = sum_s |w_s| sum_m k_sm,
// and it sends a query to the re-score when |f~| <= eps(q) B~, with
// eps(q) = eps0 + eps1 (|p~| + |s~|max): |p~| the largest norm of the
// query's scaled FP32 control points, |s~|max that of the support set's.
// This function returns eps0 and eps1 such that |f~ - f| <= eps(q) B; then
// |f~| > eps(q) B~ implies that f~ has the sign of f (and f != 0), so every
// label decided in FP32 is the label of the exact f.  With u = 2^-24:
//
// (1) Control points.  The query's points come from pair-arithmetic
//     kinematics (fk_dfk.cuh, absolute error e_fk <= 2^-32 (1 + g reach))
//     rounded once to FP32; the support's from FP64 kinematics rounded once.
//     So e = (p~ - s~) - (p - s) has |e| <= u (1 + u) (|p~| + |s~|max) +
//     2 e_fk.  Since t = 1 + |d|^2, t(d + e) / t(d) - 1 = (2 d.e + |e|^2) /
//     (1 + |d|^2) and 2 |d| / (1 + |d|^2) <= 1: t is off by a factor 1 + x
//     with |x| <= |e| + |e|^2, and k = t^-2 by at most 2 |x| (1 + 3 |x|),
//     relative.  Every summand of every support point: 2 |e| to first order.
// (2) Summands, from the FP32 inputs (t* = 1 + |p~ - s~|^2 exactly).  Each
//     difference is rounded once (relative u), squared inside an FMA, and t
//     is a chain of three FMAs over non-negative terms: t~ = t* (1 + eta),
//     |eta| <= 5u, so 1/t~^2 is within 10u of 1/t*^2.  A shared pair
//     (t1^2 + t2^2) / (t1 t2)^2: products t1 t2, its square, t2^2 and the
//     numerator's FMA are rounded once each (u each, but the numerator's two
//     roundings act on a sum of positive terms: 1u + 1u), the reciprocal
//     rho = 2^-23: 5u + rho beside the 10u of the t's.  A single 1/t^2 = r r
//     with r = rcp(t): 2 rho + 10u.  The Mv - NP summands (NP pairs) of a
//     support point are added by FMAs to the exact constant count of base
//     points: (Mv - NP) u more; the weight alpha_s / M rounded to FP32: u.
//     So each term w_s acc_s is within A u of its value from the FP32
//     inputs, A = max(15 + rho/u, 10 + 2 rho/u) + Mv - NP + 1.
// (3) Accumulation.  Per packed half, the terms of one sign are summed in
//     FP32 kFoldPairs at a time (that many roundings, each at most u times a partial
//     sum of same-sign terms), each partial folded into a pair by two-sum
//     (exact; the low word's own roundings add at most n_c^2 u^2 / 2 for n_c
//     partials), the pair rounded once (u), the two halves added (u), and
//     f = P + N (u): (kFoldPairs + 3) u + n_c^2 u^2 / 2 of sum |terms| = B.
// B~ is bounded the same way, so dividing by B~ instead of B costs a
// factor 1 + O(1e-5); the FP32 evaluation of eps(q) and of eps(q) B~ a few
// u relative.  All first-order terms add up to below 1e-5, so their
// products are below 1e-10: the factor 1 + 2^-10 on eps0 and eps1 covers
// every such term.
//
// The half-precision kernel (FK_F16): coordinates and differences rounded
// to FP16 (uh = 2^-11), t by three HFMA2: (1) with (uh + u) in place of u
// and an absolute 2^-25 per coordinate below the FP16 normal range; (2)
// with 10 uh for the t's; the rest in FP32 as above; factor 1 + 1/16.
//
// A caller-given eps (rescore_eps > 0) replaces the bound: eps0 = eps,
// eps1 = 0.  The Gaussian summand uses measured bands (kDefaultEpsGauss,
// kDefaultEpsF16Gauss), eps1 = 0.
static void score_band(const ChainF &cf, int summand, double gamma, int64_t ns, bool half, double user_eps,
                       float *eps0, float *eps1) {
  if (user_eps > 0.0) {
    *eps0 = (float)user_eps;
    *eps1 = 0.f;
    return;
  }
  if (summand == FK_SUMMAND_GAUSS) {
    *eps0 = (float)(half ? kDefaultEpsF16Gauss : kDefaultEpsGauss);
    *eps1 = 0.f;
    return;
  }
  const double u = 0x1p-24, uh = 0x1p-11, rho = kRcpRel;
  const int Mv = cf.Mv, NP = (Mv + 5) / 14;  // RcpPlan<Mv>::NP of score_core.cuh
  const double g = sqrt(0.5 * gamma);
  const double t_err = half ? 10.0 * uh : 10.0 * u;
  const double pair = NP > 0 ? t_err + 5.0 * u + rho : 0.0;
  const double single = Mv > 2 * NP ? t_err + 2.0 * rho : 0.0;
  const double term = (pair > single ? pair : single) + (Mv - NP + 1) * u;
  const double npair = (double)((ns + 1) / 2 + 1);
  const double nc = npair / kFoldPairs + npair / kMinTilePairs + 2.0;
  const double acc = (kFoldPairs + 3) * u + 0.5 * nc * nc * u * u;
  const double efk = 0x1p-32 * (1.0 + g * cf.reach);
  const double pos_abs = half ? 2.0 * 2.0 * sqrt(3.0) * 0x1p-25 : 0.0;
  const double factor = half ? 1.0 + 1.0 / 16 : 1.0 + 0x1p-10;
  *eps0 = (float)((term + acc + 4.0 * efk + pos_abs) * factor);
  *eps1 = (float)(2.0 * ((half ? uh : 0.0) + u) * (1.0 + u) * factor);
}
// The circle form of point 0 in the FP32 RQ score (score_core.cuh, CIRC).
// Its summand t = 1 + D^2, D = fl(sg C + fl(-cg S)): sg, cg the query's sine
// and cosine of theta / 2 (pair arithmetic, error e_sc ~ 2^-44, rounded once),
// C, S the support's 2 rho g (cos, sin)(theta_s / 2) from FP64, rounded once.
// (1) Inputs.  |sin a cos b| + |cos a sin b| <= 1, so the exact products
//     from the rounded inputs move D by at most (2u + u^2) 2 rho g + 4 rho g
//     e_sc; as in (1) above, t moves by a factor 1 + x with |x| <= |e| + e^2
//     and k = t^-2 by 2|e| to first order: 8 u (1 + u) rho g, plus 8 rho g
//     e_sc, which is far below the 4 e_fk of eps0.
// (2) Arithmetic.  fl(cg S) and the FMA for D round once each, t's FMA once:
//     t~ / t* - 1 <= u |cg S| 2|D| / (1 + D^2) + 2u D^2 / (1 + D^2) + u
//     <= 2 u (1 + u) rho g + 3u, so k is within 4 u (1 + u) rho g + 6u; the
//     reciprocal and the sums as for the other points.
// Together 12 u (1 + u) rho g + 6u + 2 rho_rcp: within 10u + 2 rho_rcp (A u)
// plus eps1 times cnorm = 6 rho g.  So the kernel takes max(|p~| + |s~|max,
// cnorm) in eps(q), and every summand of every point stays within eps(q).  The
// form is used for rho g <= 4 (first-order terms below 1e-5, as above) and
// from kCircleMinSupport support points up: it saves three packed operations
// per support pair and costs a pair-arithmetic sine and cosine per query
// (3-DOF arm, 49 points: 0.40 against 0.39 ms; 7-DOF, 800 points: 5.26
// against 5.49 ms).
static bool g_circle = true;
constexpr int64_t kCircleMinSupport = 128;

static float score_circle(const fk_chain *c, int summand, double gamma, int64_t ns) {
  if (!g_circle || !c->cd.circ || summand != FK_SUMMAND_RQ || ns < kCircleMinSupport) return 0.f;
  const double rg = c->cd.circ_rho * sqrt(0.5 * gamma);
  if (!(rg > 0.0) || rg > 4.0) return 0.f;
  return nextafterf((float)(6.0 * rg * (1.0 + 0x1p-20)), INFINITY);
}

extern "C" int fk_set_circle_form(int on) {
  g_circle = on != 0;
  return FK_OK;
}

static int g_gauss_poly = 0;  // control points per support point on the FMA polynomial

extern "C" int fk_set_gauss_poly(int points) {
  if (points < 0 || points > 2) return fail(FK_ERR_ARG, "fk_set_gauss_poly: points must be 0, 1 or 2");
  g_gauss_poly = points;
  return FK_OK;
}
static constexpr uint32_t kDefaultWaitLimit = 1u << 22;  // about a quarter second of polling
static uint32_t g_wait_limit = kDefaultWaitLimit;

extern "C" void fk_set_wait_limit(uint32_t polls) { g_wait_limit = polls; }

struct fastron_model {
  const fk_chain *chain = nullptr;
  // training state (full training set)
  int64_t N = 0;
  int gram = -1;  // arithmetic/storage of G for the training set of the last call (-1: none)
  const double *gram_X = nullptr;  // the device buffer G was built from
  int gram_summand = FK_SUMMAND_RQ;  // the summand G was built with
  DevBuf cpX, cpdf, G, alpha, F, stats, sup_idx, sup_alpha, trace_kind, trace_idx, trace_delta;
  int64_t trace_len = 0;
  // support set packed for scoring
  int64_t ns = -1;  // -1 = untrained
  double gamma = 0.0;
  int summand = FK_SUMMAND_RQ;  // the chain's summand when the support set was packed
  DevBuf rec, cp64, alpha_s, q_s, qin, sdf;
  DevBuf slot, npos;  // record slot of each support point; [0] positive-weight pairs, [1] |s|max bits (device)
  std::vector<int64_t> host_idx;  // training indices of the support points (model_set: positions)
  bool host_idx_valid = false;
  // score scratch
  DevBuf band_idx, flags;  // flags: [0] band count, [1] error bits, [2] FP64 band count
  DevBuf qdf, part, band2_idx;  // double-float re-score scratch
  DevBuf fb_idx, fb_q, fb_lab, fb_f;  // band of the half pass, re-scored by the FP32 path
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
  DevBuf *bufs[] = {&m->cpX, &m->cpdf, &m->G, &m->alpha, &m->F, &m->stats, &m->sup_idx, &m->sup_alpha, &m->trace_kind,
                    &m->trace_idx, &m->trace_delta, &m->rec, &m->cp64, &m->alpha_s, &m->q_s, &m->qin, &m->sdf,
                    &m->qdf, &m->part, &m->band2_idx, &m->slot, &m->npos,
                    &m->band_idx, &m->flags, &m->fb_idx, &m->fb_q, &m->fb_lab, &m->fb_f};
  for (DevBuf *b : bufs) b->release();
  delete m;
}

static int pack(fastron_model *m, const double *X, const int32_t *idx, const double *alpha, int64_t ns, double gamma,
                cudaStream_t s) {
  const fk_chain *c = m->chain;
  CK(m->rec.ensure(sizeof(float4) * (size_t)rec_pairs(ns) * rec_len(c->cf.Mv)));
  CK(m->slot.ensure(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1)));
  CK(m->npos.ensure(sizeof(int32_t) * 2));
  CK(m->cp64.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * c->M * 3));
  CK(m->alpha_s.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1)));
  CK(m->q_s.ensure(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * c->D));
  CK(m->sdf.ensure(sizeof(float) * (size_t)(ns > 0 ? ns : 1) * rec_df_len(c->cf.Mv)));
  const int summand = c->cf.summand;
  // coordinates scaled so that the summand is (1 + |d|^2)^-2 (RQ) or
  // 2^(-|d|^2) (Gaussian), in the FP32 and the double-float records alike
  const double scale = sqrt(summand == FK_SUMMAND_GAUSS ? 0.5 * gamma * M_LOG2E : 0.5 * gamma);
  PackArgs pa{X, idx, alpha, ns, gamma, m->rec.as<float4>(), m->cp64.as<double>(), m->alpha_s.as<double>(),
              m->q_s.as<double>(), m->sdf.as<float>(), scale, m->slot.as<int32_t>(), m->npos.as<int32_t>()};
  CK(launch_pack_support(c->cf, c->cd, pa, s));
  m->ns = ns;
  m->gamma = gamma;
  m->summand = summand;
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
  const bool gauss = m->chain->cd.summand == FK_SUMMAND_GAUSS;
  const int gram = p->gram == 0 ? (gauss ? FK_F64 : FK_DF64) : p->gram;
  if (gram != FK_F64 && gram != FK_DF64 && gram != FK_DF32)
    return fail(FK_ERR_ARG, "fastron_train: gram must be FK_DF64, FK_F64 or FK_DF32");
  if (gauss && gram != FK_F64)
    return fail(FK_ERR_ARG, "fastron_train: the Gaussian summand's kernel matrix is built in FP64 (gram FK_F64 or 0)");
  if (p->warm_start < 0 || p->warm_start > 2) return fail(FK_ERR_ARG, "fastron_train: warm_start must be 0, 1 or 2");
  if (p->warm_start == 1 && (m->N != N || m->alpha.p == nullptr))
    return fail(FK_ERR_STATE, "fastron_train: warm start needs a previous training call with the same N");
  const int64_t ns_carry = m->ns;
  if (p->warm_start == 2 && (ns_carry < 0 || ns_carry > N))
    return fail(FK_ERR_STATE, "fastron_train: carrying the support set needs a trained model with |S| <= N");
  if (p->warm_start == 2 && p->reuse_gram)
    return fail(FK_ERR_ARG, "fastron_train: a carried support set means a new training set: reuse_gram must be 0");
  if (p->reuse_gram && (m->N != N || m->gram != gram || m->gram_X != X || m->gram_summand != m->chain->cd.summand))
    return fail(FK_ERR_STATE, "fastron_train: reuse_gram needs a previous call on the same X buffer with the same N "
                              "and gram");
  cudaStream_t s = (cudaStream_t)stream;
  const fk_chain *c = m->chain;
  const bool keep = p->warm_start == 1;
  const bool reuse = p->reuse_gram != 0;
  CK(m->cpX.ensure(sizeof(double) * (size_t)N * c->M * 3));
  if (!reuse) m->gram = -1;  // the stored matrix is invalid until rebuilt below
  CK(m->G.ensure((gram == FK_DF32 ? sizeof(float) : sizeof(double)) * (size_t)N * (size_t)N));
  if (!keep) {
    CK(m->alpha.ensure(sizeof(double) * (size_t)N));
    CK(m->F.ensure(sizeof(double) * (size_t)N));
    CK(cudaMemsetAsync(m->alpha.p, 0, sizeof(double) * (size_t)N, s));
    CK(cudaMemsetAsync(m->F.p, 0, sizeof(double) * (size_t)N, s));
  }
  CK(m->stats.ensure(sizeof(int64_t) * 6));
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
  if (!reuse) {
    CK(launch_fk_forward_f64(c->cd, X, N, m->cpX.as<double>(), s));
    const double *cp = m->cpX.as<double>();
    if (gram == FK_F64)
      CK(launch_gram_f64(c->cd, p->gamma, cp, N, cp, N, 1, m->G.as<double>(), s));
    else {
      CK(m->cpdf.ensure(sizeof(float2) * (size_t)(c->cd.Mv > 0 ? c->cd.Mv : 1) * 3 * (size_t)N));
      float2 *w = m->cpdf.as<float2>();
      if (gram == FK_DF32)
        CK(launch_gram_df32(c->cd, p->gamma, cp, N, cp, N, 1, m->G.as<float>(), w, w, s));
      else
        CK(launch_gram_df(c->cd, p->gamma, cp, N, cp, N, 1, m->G.as<double>(), w, w, s));
    }
    m->gram = gram;
    m->gram_X = X;
    m->gram_summand = c->cd.summand;
  }
  if (p->warm_start == 2) {
    // loadPreviousModel on a changed training set: the first ns rows are the
    // previous support points with their weights; F = K alpha
    if (ns_carry > 0)
      CK(cudaMemcpyAsync(m->alpha.p, m->alpha_s.p, sizeof(double) * (size_t)ns_carry, cudaMemcpyDeviceToDevice, s));
    CK(launch_margins(m->G.p, gram == FK_DF32 ? 1 : 0, N, m->alpha.as<double>(), ns_carry, m->F.as<double>(), s));
  }
  TrainArgs ta{m->G.p, gram == FK_DF32 ? 1 : 0, y, N, p->beta, p->iter_max, p->s_max, m->alpha.as<double>(), m->F.as<double>(),
               m->stats.as<int64_t>(), m->sup_idx.as<int32_t>(), m->sup_alpha.as<double>(),
               trace ? m->trace_kind.as<int8_t>() : nullptr, trace ? m->trace_idx.as<int32_t>() : nullptr,
               trace ? m->trace_delta.as<double>() : nullptr, g_wait_limit};
  CK(cudaMemsetAsync(m->stats.p, 0, sizeof(int64_t) * 6, s));
  CK(launch_fastron_train(ta, s));
  int64_t hs[6];
  CK(cudaMemcpyAsync(hs, m->stats.p, sizeof hs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs[5] != 0) {  // alpha and F are incomplete: no warm start or matrix reuse from them
    m->N = 0;
    m->gram = -1;
    m->trace_len = 0;
    return fail(FK_ERR_TIMEOUT, "fastron_train: a cluster exchange wait timed out");
  }
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

extern "C" int fastron_model_copy(fastron_model_t *dst, const fastron_model_t *cs, void *stream) {
  fastron_model *src = const_cast<fastron_model *>(cs);
  if (!dst || !src) return fail(FK_ERR_ARG, "fastron_model_copy: model is NULL");
  if (dst == src) return fail(FK_ERR_ARG, "fastron_model_copy: dst and src are the same model");
  if (dst->chain != src->chain) return fail(FK_ERR_ARG, "fastron_model_copy: the models have different chains");
  if (src->ns < 0) return fail(FK_ERR_STATE, "fastron_model_copy: src is untrained");
  const fk_chain *c = src->chain;
  const int64_t ns = src->ns, n1 = ns > 0 ? ns : 1;
  cudaStream_t s = (cudaStream_t)stream;
  // the buffers pack() fills, at the sizes it gives them
  const size_t bytes[] = {sizeof(float4) * (size_t)rec_pairs(ns) * rec_len(c->cf.Mv), sizeof(int32_t) * (size_t)n1,
                          sizeof(int32_t) * 2, sizeof(double) * (size_t)n1 * c->M * 3, sizeof(double) * (size_t)n1,
                          sizeof(double) * (size_t)n1 * c->D, sizeof(float) * (size_t)n1 * rec_df_len(c->cf.Mv),
                          sizeof(int32_t) * (size_t)n1};
  DevBuf *from[] = {&src->rec, &src->slot, &src->npos, &src->cp64, &src->alpha_s, &src->q_s, &src->sdf, &src->sup_idx};
  DevBuf *to[] = {&dst->rec, &dst->slot, &dst->npos, &dst->cp64, &dst->alpha_s, &dst->q_s, &dst->sdf, &dst->sup_idx};
  const int nbuf = src->host_idx_valid ? 7 : 8;  // the training indices live on the device after fastron_train
  for (int i = 0; i < nbuf; ++i) {
    CK(to[i]->ensure(bytes[i]));
    CK(cudaMemcpyAsync(to[i]->p, from[i]->p, bytes[i], cudaMemcpyDeviceToDevice, s));
  }
  dst->ns = ns;
  dst->gamma = src->gamma;
  dst->summand = src->summand;
  dst->host_idx = src->host_idx;
  dst->host_idx_valid = src->host_idx_valid;
  // dst holds no training state of its own
  dst->N = 0;
  dst->gram = -1;
  dst->trace_len = 0;
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

// ---------------------------------------------------- active learning ---
extern "C" int fk_active_samples(const fastron_model_t *m, int32_t k_near, double sigma, int64_t n_uniform,
                                 double qlim, uint64_t seed, double *X, float *X32, int64_t cap, int64_t *n_out,
                                 void *stream) {
  if (!m || !n_out) return fail(FK_ERR_ARG, "fk_active_samples: NULL pointer");
  *n_out = 0;
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_active_samples: model is untrained");
  if (k_near < 0 || n_uniform < 0) return fail(FK_ERR_ARG, "fk_active_samples: negative count");
  if (!(sigma >= 0.0) || !std::isfinite(sigma) || !(qlim > 0.0) || !std::isfinite(qlim))
    return fail(FK_ERR_ARG, "fk_active_samples: sigma must be >= 0 and qlim > 0, both finite");
  const int64_t rows = m->ns * (1 + (int64_t)k_near) + n_uniform;
  *n_out = rows;
  if (rows > cap) return fail(FK_ERR_CAPACITY, "fk_active_samples: %lld rows exceed cap %lld", (long long)rows,
                              (long long)cap);
  if (rows == 0) return FK_OK;
  if (!X) return fail(FK_ERR_ARG, "fk_active_samples: X is NULL");
  ActiveArgs aa{m->q_s.as<double>(), m->ns, m->chain->D, k_near, sigma, qlim, n_uniform, seed, X, X32};
  CK(launch_active_samples(aa, (cudaStream_t)stream));
  return FK_OK;
}

// -------------------------------------------------------------- score ---
extern "C" int fk_score(fastron_model_t *m, const float *q, int64_t n, int precision, int rescore, double rescore_eps,
                        float *f, int8_t *label, int64_t *n_rescored, void *stream) {
  if (!m) return fail(FK_ERR_ARG, "fk_score: model is NULL");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_score: model is untrained");
  if (n < 0) return fail(FK_ERR_ARG, "fk_score: n < 0");
  if (n > (int64_t)INT32_MAX) return fail(FK_ERR_CAPACITY, "fk_score: n exceeds 2^31 - 1");
  if (precision != FK_F32 && precision != FK_F16) return fail(FK_ERR_ARG, "fk_score: unsupported precision %d", precision);
  if (n_rescored) *n_rescored = 0;
  if (n == 0) return FK_OK;
  if (!q || !label) return fail(FK_ERR_ARG, "fk_score: q and label must not be NULL");
  if (m->gamma > 1e7) return fail(FK_ERR_ARG, "fk_score: gamma above the FP32 range of the score kernel");
  cudaStream_t s = (cudaStream_t)stream;
  const fk_chain *c = m->chain;
  // the summand the support set was packed with (a later change of the
  // chain's summand does not apply to this model)
  const bool gauss = m->summand == FK_SUMMAND_GAUSS;
  ChainF cf = c->cf;
  ChainD cd = c->cd;
  cf.summand = cd.summand = m->summand;
  const double gs = sqrt(gauss ? 0.5 * m->gamma * M_LOG2E : 0.5 * m->gamma);
  float eps0 = 0.f, eps1 = 0.f;
  if (precision == FK_F16) {
    if (!score_f16_supported(c->cf.Mv))
      return fail(FK_ERR_ARG, "fk_score: no half-precision kernel for %d control points", c->cf.Mv);
    CK(m->flags.ensure(sizeof(int32_t) * 2));
    CK(cudaMemsetAsync(m->flags.p, 0, sizeof(int32_t) * 2, s));
    if (rescore) CK(m->band_idx.ensure(sizeof(int32_t) * (size_t)n));
    if (!gauss && sqrt(0.5 * m->gamma) * c->cf.reach > 64.0)
      return fail(FK_ERR_ARG, "fk_score: scaled reach %.1f too large for the half-precision differences",
                  sqrt(0.5 * m->gamma) * c->cf.reach);
    score_band(c->cf, m->summand, m->gamma, m->ns, true, rescore_eps, &eps0, &eps1);
    ScoreArgs sa{q, n, m->rec.as<float4>(), 2 * rec_pairs(m->ns), gs, eps0, eps1, f, label,
                 rescore ? m->band_idx.as<int32_t>() : nullptr, m->flags.as<int32_t>(), m->flags.as<int32_t>() + 1,
                 g_wait_limit, 0, m->npos.as<int32_t>()};
    CK(launch_score_f16(cf, sa, s));
    int32_t h[2] = {0, 0};
    if (rescore || n_rescored) {
      CK(cudaMemcpyAsync(h, m->flags.p, sizeof h, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h[1] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score: a shared-memory tile wait timed out");
    }
    if (!rescore) return FK_OK;
    const int64_t nb = h[0];
    if (nb > 0) {
      // the half pass's band goes through the FP32 score and its FP64 re-score
      CK(m->fb_idx.ensure(sizeof(int32_t) * (size_t)nb));
      CK(m->fb_q.ensure(sizeof(float) * (size_t)nb * c->D));
      CK(m->fb_lab.ensure((size_t)nb));
      CK(m->fb_f.ensure(sizeof(float) * (size_t)nb));
      CK(cudaMemcpyAsync(m->fb_idx.p, m->band_idx.p, sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToDevice, s));
      CK(launch_gather_rows(q, c->D, m->fb_idx.as<int32_t>(), nb, m->fb_q.as<float>(), s));
      int rc = fk_score(m, m->fb_q.as<float>(), nb, FK_F32, 1, 0.0, m->fb_f.as<float>(), m->fb_lab.as<int8_t>(),
                        nullptr, stream);
      if (rc != FK_OK) return rc;
      CK(launch_scatter_labels(m->fb_lab.as<int8_t>(), m->fb_f.as<float>(), m->fb_idx.as<int32_t>(), nb, label, f, s));
    }
    if (n_rescored) *n_rescored = nb;
    return FK_OK;
  }
  CK(m->flags.ensure(sizeof(int32_t) * 4));
  CK(cudaMemsetAsync(m->flags.p, 0, sizeof(int32_t) * 4, s));
  int32_t *cnt = m->flags.as<int32_t>(), *err = cnt + 1, *cnt2 = cnt + 2;
  if (rescore) CK(m->band_idx.ensure(sizeof(int32_t) * (size_t)n));
  score_band(c->cf, m->summand, m->gamma, m->ns, false, rescore_eps, &eps0, &eps1);
  ScoreArgs sa{q, n, m->rec.as<float4>(), 2 * rec_pairs(m->ns), gs, eps0, eps1, f, label,
               rescore ? m->band_idx.as<int32_t>() : nullptr, cnt, err, g_wait_limit, gauss ? g_gauss_poly : 0,
               m->npos.as<int32_t>(), score_circle(c, m->summand, m->gamma, m->ns)};
  CK(launch_score_f32(cf, sa, s));
  if (!rescore && !n_rescored) return FK_OK;
  int32_t h[2];
  CK(cudaMemcpyAsync(h, m->flags.p, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h[1] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score: a shared-memory tile wait timed out");
  if (n_rescored) *n_rescored = rescore ? h[0] : 0;
  if (!rescore || h[0] == 0) return FK_OK;
  // the band: double-float first, FP64 for what it cannot decide
  const int64_t nb = h[0];
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int chunks = rescore_df_chunks(nb, m->ns, sms);
  CK(m->qdf.ensure(sizeof(float2) * (size_t)nb * c->cf.Mv * 3));
  CK(m->part.ensure(sizeof(float4) * (size_t)nb * chunks));
  CK(m->band2_idx.ensure(sizeof(int32_t) * (size_t)nb));
  DfRescoreArgs da{q, m->band_idx.as<int32_t>(), nb, m->sdf.as<float>(), m->ns, c->cd.n_const,
                   sqrt(gauss ? 0.5 * m->gamma * M_LOG2E : 0.5 * m->gamma), m->qdf.as<float2>(), m->part.as<float4>(),
                   chunks,
                   (m->ns + chunks - 1) / chunks, kDefaultEpsDf, f, label, m->band2_idx.as<int32_t>(), cnt2};
  CK(launch_rescore_df(cd, da, s));
  RescoreArgs ra{q, m->band2_idx.as<int32_t>(), cnt2, n, m->cp64.as<double>(), m->alpha_s.as<double>(), m->ns,
                 m->gamma, f, label};
  CK(launch_rescore_f64(cd, ra, s));
  return FK_OK;
}

extern "C" int fk_score_band(const fastron_model_t *m, int precision, double *eps0, double *eps1) {
  if (!m || !eps0 || !eps1) return fail(FK_ERR_ARG, "fk_score_band: NULL pointer");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_score_band: model is untrained");
  if (precision != FK_F32 && precision != FK_F16) return fail(FK_ERR_ARG, "fk_score_band: unsupported precision");
  float e0 = 0.f, e1 = 0.f;
  score_band(m->chain->cf, m->summand, m->gamma, m->ns, precision == FK_F16, 0.0, &e0, &e1);
  *eps0 = e0;
  *eps1 = e1;
  return FK_OK;
}

extern "C" int fk_score_circle(const fastron_model_t *m, double *cnorm) {
  if (!m || !cnorm) return fail(FK_ERR_ARG, "fk_score_circle: NULL pointer");
  if (m->ns < 0) return fail(FK_ERR_STATE, "fk_score_circle: model is untrained");
  *cnorm = score_circle(m->chain, m->summand, m->gamma, m->ns);
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
  CK(launch_label(c->cf, c->cd, bx, q, n, y, (cudaStream_t)stream));
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

// ------------------------------------------------ premises of the band ---
static int run_check(const char *name, double *out, cudaError_t (*launch)(unsigned long long *, const void *),
                     const void *arg) {
  unsigned long long *d = nullptr;
  CK(cudaMalloc(&d, sizeof *d));
  cudaError_t e = cudaMemset(d, 0, sizeof *d);
  if (e == cudaSuccess) e = launch(d, arg);
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(FK_ERR_CUDA, "%s: %s", name, cudaGetErrorString(e));
  memcpy(out, &h, sizeof *out);
  return FK_OK;
}

extern "C" int fk_check_rcp(int e_lo, int e_hi, double *max_rel) {
  if (!max_rel) return fail(FK_ERR_ARG, "fk_check_rcp: NULL pointer");
  if (e_lo < -126 || e_hi > 127 || e_lo > e_hi) return fail(FK_ERR_ARG, "fk_check_rcp: binades outside [-126, 127]");
  struct A { int lo, hi; } a{e_lo, e_hi};
  return run_check("fk_check_rcp", max_rel, [](unsigned long long *d, const void *p) {
    const A *x = static_cast<const A *>(p);
    return launch_check_rcp(x->lo, x->hi, d, 0);
  }, &a);
}

extern "C" int fk_check_sincos(float hi, double theta0, double *max_abs) {
  if (!max_abs) return fail(FK_ERR_ARG, "fk_check_sincos: NULL pointer");
  if (!(hi >= 0.f) || !(fabs(theta0) + hi < 65536.0)) return fail(FK_ERR_ARG, "fk_check_sincos: need 0 <= hi, |theta| < 2^16");
  struct A { float hi; double th0; } a{hi, theta0};
  return run_check("fk_check_sincos", max_abs, [](unsigned long long *d, const void *p) {
    const A *x = static_cast<const A *>(p);
    return launch_check_sincos(x->hi, x->th0, d, 0);
  }, &a);
}

extern "C" int fk_forward_dd(const fk_chain_t *c, const float *q, int64_t n, double scale, float *cp, void *stream) {
  if (!c) return fail(FK_ERR_ARG, "fk_forward_dd: chain is NULL");
  if (n < 0) return fail(FK_ERR_ARG, "fk_forward_dd: n < 0");
  if (n == 0) return FK_OK;
  if (!q || !cp) return fail(FK_ERR_ARG, "fk_forward_dd: NULL pointer");
  if (!(scale > 0.0) || !std::isfinite(scale)) return fail(FK_ERR_ARG, "fk_forward_dd: scale must be finite and > 0");
  CK(launch_forward_dd(c->cf, q, n, scale, cp, (cudaStream_t)stream));
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
// memory, so kernels get the address found here.  The cache assumes that the
// device's primary context lives as long as the process: after a
// cudaDeviceReset the cached address is stale and the call must not be used.
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
  const bool gauss = m->summand == FK_SUMMAND_GAUSS;
  ChainF cf = c->cf;
  ChainD cd = c->cd;
  cf.summand = cd.summand = m->summand;
  float eps0 = 0.f, eps1 = 0.f;
  score_band(c->cf, m->summand, m->gamma, m->ns, false, rescore_eps, &eps0, &eps1);
  ScoreArgs sa{q, n, m->rec.as<float4>(), 2 * rec_pairs(m->ns), sqrt(gauss ? 0.5 * m->gamma * M_LOG2E : 0.5 * m->gamma),
               eps0, eps1, f, label, band, cnt, err, g_wait_limit, gauss ? g_gauss_poly : 0, m->npos.as<int32_t>(),
               score_circle(c, m->summand, m->gamma, m->ns)};
  CK(launch_score_f32(cf, sa, s));
  RescoreArgs ra{q, band, cnt, n, m->cp64.as<double>(), m->alpha_s.as<double>(), m->ns, m->gamma, f, label};
  CK(launch_rescore_f64(cd, ra, s));
  // the error word is read back on every call (one synchronisation): a tile
  // wait that gave up leaves labels undefined, and the next call's memset
  // would erase the only record of it
  int32_t h[2];
  CK(cudaMemcpyAsync(h, scratch, sizeof h, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h[1] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score_noalloc: a shared-memory tile wait timed out");
  if (n_rescored) *n_rescored = h[0];
  return FK_OK;
}

// ------------------------------------------------------------ surrogate ---
// Learned surrogate of the model value (not part of the paper).  Flat FP32
// parameter vector: W1 [256][64], b1, W2 [256][256], b2, W3 [256][256], b3,
// w4 [256], b4.
namespace fk {
cudaError_t launch_surr_features(const ChainF &c, const float *q, int64_t n, int64_t n_pad, bf16 *X, cudaStream_t s);

cudaError_t launch_gemm(int nt, const GemmArgs &g, int splits, cudaStream_t s);
cudaError_t launch_adam(float *p, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                        float eps, int64_t t, cudaStream_t s);
cudaError_t launch_weights_bf16(const float *W, int rows, int cols, bf16 *Wb, cudaStream_t s);
cudaError_t launch_surr_decide(const float *out, float scale, int64_t n, float tau, float *pred, int8_t *label,
                               int32_t *fb_idx, int32_t *fb_cnt, cudaStream_t s);
cudaError_t launch_gather_rows(const float *q, int D, const int32_t *idx, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_scatter_labels(const int8_t *src, const float *fsrc, const int32_t *idx, int64_t n, int8_t *label,
                                  float *pred, cudaStream_t s);
cudaError_t launch_sumsq(const float *x, int64_t n, double *acc, cudaStream_t s);
cudaError_t launch_scale(float *x, int64_t n, float v, cudaStream_t s);
cudaError_t launch_surr_calibrate(const float *pred, const float *f, int64_t n, unsigned *tau_bits,
                                  unsigned long long *wrong, unsigned long long *below_cnt, float tau_hint,
                                  cudaStream_t s);
cudaError_t launch_count_below(const float *pred, int64_t n, float tau, unsigned long long *cnt, cudaStream_t s);
}  // namespace fk

namespace {
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + (int64_t)kSurrW * kSurrIn;
constexpr int64_t kOffW2 = kOffB1 + kSurrW, kOffB2 = kOffW2 + (int64_t)kSurrW * kSurrW;
constexpr int64_t kOffW3 = kOffB2 + kSurrW, kOffB3 = kOffW3 + (int64_t)kSurrW * kSurrW;
constexpr int64_t kOffW4 = kOffB3 + kSurrW, kOffB4 = kOffW4 + kSurrW;
constexpr int64_t kSurrParams = kOffB4 + 1;

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// SplitMix64 for the parameter initialisation (library-private stream).
struct Mix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};
}  // namespace

struct surrogate {
  const fk_chain *chain = nullptr;
  uint64_t seed = 0;
  DevBuf p, m, v, g;
  DevBuf w1b, w2b, w3b, wc;
  float scale = 1.f;   // target scale: the network predicts f / scale
  float tau = -1.f;    // calibrated threshold in units of f (< 0: not calibrated)
  int64_t t = 0;       // Adam steps taken
  // training step (surr_train.cu): batch B's transposed activations and
  // deltas (chunk-blocked), per-tile sums, split-K partials, the device step
  // counter with its block counter and schedule, the capture stream and the
  // captured graphs
  int tB = 0;
  DevBuf tT, tstat, tpart, tstep, loss_hist;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr, exec_k = nullptr;  // one step; kSurrGraphSteps steps
  DevBuf X, Y, Yh, lab_tmp;
  DevBuf iout, iwc, fb_idx, fb_cnt, fb_q, fb_lab, fb_f, ipred;
  DevBuf err, scal;
};

static int surr_init_params(surrogate *s, cudaStream_t st) {
  std::vector<float> h((size_t)kSurrParams, 0.f);
  Mix64 r{s->seed ^ 0xA5A5A5A55A5A5A5Aull};
  auto he = [&](int64_t off, int out, int in) {
    const double lim = sqrt(6.0 / in);
    for (int64_t i = 0; i < (int64_t)out * in; ++i) h[(size_t)(off + i)] = (float)((2.0 * r.uniform() - 1.0) * lim);
  };
  he(kOffW1, kSurrW, kSurrIn);
  he(kOffW2, kSurrW, kSurrW);
  he(kOffW3, kSurrW, kSurrW);
  he(kOffW4, 1, kSurrW);
  CK(cudaMemcpyAsync(s->p.p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(s->m.p, 0, sizeof(float) * kSurrParams, st));
  CK(cudaMemsetAsync(s->v.p, 0, sizeof(float) * kSurrParams, st));
  CK(cudaStreamSynchronize(st));
  s->t = 0;
  return FK_OK;
}

static int surr_sync_weights(surrogate *s, cudaStream_t st) {
  const float *P = s->p.as<float>();
  CK(launch_weights_bf16(P + kOffW1, kSurrW, kSurrIn, s->w1b.as<bf16>(), st));
  CK(launch_weights_bf16(P + kOffW2, kSurrW, kSurrW, s->w2b.as<bf16>(), st));
  CK(launch_weights_bf16(P + kOffW3, kSurrW, kSurrW, s->w3b.as<bf16>(), st));
  CK(launch_surr_wc(s->w1b.as<bf16>(), s->w2b.as<bf16>(), s->w3b.as<bf16>(), s->wc.as<uint8_t>(), st));
  return FK_OK;
}

extern "C" int surrogate_create(const fk_chain_t *chain, uint64_t seed, surrogate_t **out) {
  if (!out) return fail(FK_ERR_ARG, "surrogate_create: out is NULL");
  *out = nullptr;
  if (!chain) return fail(FK_ERR_ARG, "surrogate_create: chain is NULL");
  const int nf = chain->M < chain->D + 1 ? chain->M : chain->D + 1;  // feature points
  if (7 * nf > kSurrIn)
    return fail(FK_ERR_CAPACITY, "surrogate_create: %d feature points need %d features, above %d", nf, 7 * nf,
                kSurrIn);
  surrogate *s = new surrogate;
  s->chain = chain;
  s->seed = seed;
  int rc = FK_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == FK_OK) rc = fail(FK_ERR_CUDA, "surrogate_create: %s", cudaGetErrorString(e));
  };
  ck(s->p.ensure(sizeof(float) * kSurrParams));
  ck(s->m.ensure(sizeof(float) * kSurrParams));
  ck(s->v.ensure(sizeof(float) * kSurrParams));
  ck(s->g.ensure(sizeof(float) * kSurrParams));
  ck(s->w1b.ensure(2 * kSurrW * kSurrIn));
  ck(s->w2b.ensure(2 * kSurrW * kSurrW));
  ck(s->w3b.ensure(2 * kSurrW * kSurrW));
  ck(s->wc.ensure(kSurrWcBytes));
  ck(s->err.ensure(64));
  ck(s->scal.ensure(64));
  ck(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
  if (rc == FK_OK) rc = surr_init_params(s, 0);
  if (rc == FK_OK) rc = surr_sync_weights(s, 0);
  if (rc == FK_OK && cudaStreamSynchronize(0) != cudaSuccess) rc = fail(FK_ERR_CUDA, "surrogate_create: sync failed");
  if (rc != FK_OK) {
    surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return FK_OK;
}

extern "C" void surrogate_destroy(surrogate_t *s) {
  if (!s) return;
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->exec_k) cudaGraphExecDestroy(s->exec_k);
  if (s->cap) cudaStreamDestroy(s->cap);
  DevBuf *bufs[] = {&s->p, &s->m, &s->v, &s->g, &s->w1b, &s->w2b, &s->w3b, &s->wc,
                    &s->tT, &s->tstat, &s->tpart, &s->tstep, &s->loss_hist, &s->X, &s->Y, &s->Yh, &s->lab_tmp,
                    &s->iout, &s->iwc, &s->fb_idx, &s->fb_cnt, &s->fb_q, &s->fb_lab, &s->fb_f, &s->ipred,
                    &s->err, &s->scal};
  for (DevBuf *b : bufs) b->release();
  delete s;
}

// Split factor of the weight-gradient products for batch B: six CTAs per
// split (three products, two M tiles), at most 24 splits (144 CTAs) and at
// least one 64-row chunk per split.
static int surr_splits(int B) {
  const int kc = B / kBK;
  return kc < 24 ? kc : 24;
}

constexpr int kSurrGraphSteps = 8;

static void surr_drop_graph(surrogate *s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->exec_k) cudaGraphExecDestroy(s->exec_k);
  s->exec = s->exec_k = nullptr;
}

// Scratch of the training step for batch B.
static int surr_step_buffers(surrogate *s, int B) {
  if (s->tB == B) return FK_OK;
  surr_drop_graph(s);
  CK(s->tT.ensure(2 * (size_t)B * (kSurrIn + 5 * kSurrW)));
  CK(s->tstat.ensure(sizeof(float) * (size_t)(B / kBM) * kTileStats));
  CK(s->tpart.ensure(sizeof(float) * (size_t)surr_splits(B) * kSurrDwPart));
  CK(s->tstep.ensure(32));  // int64 step, uint32 block counter, float schedule[3]
  s->tB = B;
  return FK_OK;
}

// Enqueues one training step (surr_train.cu) on st: the tile kernel over the
// batch (rows (step mod steps_per_epoch) B .. + B of X and Y), the three
// weight-gradient products, then the reduction into the flat gradient g and
// the loss into loss_hist[step] (if not null); with sch also Adam at that
// schedule, the BF16 weights and the step counter.
static int surr_step_enqueue(surrogate *s, const bf16 *X, const float *Y, int B, int64_t steps_per_epoch,
                             const SurrSched *sch, float *loss_hist, cudaStream_t st) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const float *P = s->p.as<float>();
  bf16 *xT = s->tT.as<bf16>();
  bf16 *h1T = xT + (int64_t)kSurrIn * B, *h2T = h1T + (int64_t)kSurrW * B;
  bf16 *d3T = h2T + (int64_t)kSurrW * B, *d2T = d3T + (int64_t)kSurrW * B, *d1T = d2T + (int64_t)kSurrW * B;
  int64_t *step = s->tstep.as<int64_t>();
  float *tstat = s->tstat.as<float>();
  SurrStepArgs a{X, Y, B, steps_per_epoch, step, s->wc.as<uint8_t>(), P + kOffB1, P + kOffB2, P + kOffB3,
                 P + kOffW4, P + kOffB4, xT, h1T, h2T, d3T, d2T, d1T, tstat, s->err.as<int32_t>(), g_wait_limit};
  CK(launch_surr_tile(a, sms, st));
  const int splits = surr_splits(B);
  float *p1 = s->tpart.as<float>(), *p2 = p1 + (int64_t)splits * kSurrW * kSurrIn;
  float *p3 = p2 + (int64_t)splits * kSurrW * kSurrW;
  float *sched = reinterpret_cast<float *>(s->tstep.as<char>() + 16);
  SurrDwArgs d{xT, h1T, h2T, d1T, d2T, d3T, B, splits, p1, p2, p3, step, sch ? *sch : SurrSched{},
               sch ? sched : nullptr, s->err.as<int32_t>(), g_wait_limit};
  CK(launch_surr_dw(d, st));
  SurrAdamArgs u{};
  u.p = s->p.as<float>();
  u.m = s->m.as<float>();
  u.v = s->v.as<float>();
  u.G = s->g.as<float>();
  u.p1 = p1;
  u.p2 = p2;
  u.p3 = p3;
  u.splits = splits;
  u.tstat = tstat;
  u.ntiles = B / kBM;
  u.B = B;
  u.loss_hist = loss_hist;
  u.step = step;
  u.done = reinterpret_cast<uint32_t *>(s->tstep.as<char>() + 8);
  u.update = sch ? 1 : 0;
  u.sched = sched;
  u.w1 = s->w1b.as<bf16>();
  u.w2 = s->w2b.as<bf16>();
  u.w3 = s->w3b.as<bf16>();
  u.wc = s->wc.as<uint8_t>();
  CK(launch_surr_adam(u, st));
  return FK_OK;
}

static int surr_check_err(surrogate *s, cudaStream_t st, const char *who) {
  int32_t h = 0;
  CK(cudaMemcpyAsync(&h, s->err.p, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h & kErrTimeout) return fail(FK_ERR_TIMEOUT, "%s: a tensor-core completion wait timed out", who);
  return FK_OK;
}

// Features of n queries into buffer X ([n_pad][64], rows n.. zero).
static int surr_features(surrogate *s, const float *q, int64_t n, int64_t n_pad, DevBuf &X, cudaStream_t st) {
  CK(X.ensure(2 * (size_t)n_pad * kSurrIn));
  CK(launch_surr_features(s->chain->cf, q, n, n_pad, X.as<bf16>(), st));
  return FK_OK;
}

// Network outputs (f / scale) of n queries q into out, with the fused
// inference kernel (features and all layers in one launch); with decide != 0
// also labels, pred and the fallback list (fb_cnt zeroed by the caller).
static int surr_forward_fused(surrogate *s, const float *q, int64_t n, float *out, int decide, float tau, float *pred,
                              int8_t *label, int32_t *fb_idx, int32_t *fb_cnt, cudaStream_t st) {
  const float *P = s->p.as<float>();
  MlpArgs a{};
  a.q = q;
  a.n = n;
  a.w1 = s->w1b.as<bf16>();
  a.w2 = s->w2b.as<bf16>();
  a.w3 = s->w3b.as<bf16>();
  a.b1 = P + kOffB1;
  a.b2 = P + kOffB2;
  a.b3 = P + kOffB3;
  a.w4 = P + kOffW4;
  a.b4 = P + kOffB4;
  a.out = out;
  a.decide = decide;
  a.scale = s->scale;
  a.tau = tau;
  a.pred = pred;
  a.label = label;
  a.fb_idx = fb_idx;
  a.fb_cnt = fb_cnt;
  a.err = s->err.as<int32_t>();
  a.wait_limit = g_wait_limit;
  CK(s->iwc.ensure(mlp_wc_bytes()));
  CK(launch_mlp_fused(s->chain->cf, a, s->iwc.as<uint8_t>(), st));
  return FK_OK;
}

extern "C" int surrogate_set_params(surrogate_t *s, const float *params, int64_t count) {
  if (!s || !params) return fail(FK_ERR_ARG, "surrogate_set_params: NULL pointer");
  if (count != kSurrParams) return fail(FK_ERR_ARG, "surrogate_set_params: expected %lld values", (long long)kSurrParams);
  CK(cudaMemcpy(s->p.p, params, sizeof(float) * kSurrParams, cudaMemcpyHostToDevice));
  int rc = surr_sync_weights(s, 0);
  if (rc != FK_OK) return rc;
  CK(cudaStreamSynchronize(0));
  return FK_OK;
}

extern "C" int surrogate_get_params(const surrogate_t *s, float *params, int64_t count, float *scale, float *tau) {
  if (!s) return fail(FK_ERR_ARG, "surrogate_get_params: NULL pointer");
  if (params) {
    if (count != kSurrParams)
      return fail(FK_ERR_ARG, "surrogate_get_params: expected %lld values", (long long)kSurrParams);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(params, s->p.p, sizeof(float) * kSurrParams, cudaMemcpyDeviceToHost));
  }
  if (scale) *scale = s->scale;
  if (tau) *tau = s->tau;
  return FK_OK;
}

extern "C" int surrogate_gradients(surrogate_t *s, const float *q, int64_t n, const float *target, float *grad,
                                   float *loss) {
  if (!s || !q || !target || !grad) return fail(FK_ERR_ARG, "surrogate_gradients: NULL pointer");
  if (n < kBM || n % kBM || n > (1 << 20)) return fail(FK_ERR_ARG, "surrogate_gradients: n must be a multiple of 128");
  cudaStream_t st = 0;
  CK(cudaMemsetAsync(s->err.p, 0, 64, st));
  int rc = surr_step_buffers(s, (int)n);
  if (rc != FK_OK) return rc;
  if ((rc = surr_features(s, q, n, n, s->X, st)) != FK_OK) return rc;
  CK(cudaMemsetAsync(s->tstep.p, 0, 16, st));  // step and block counter
  float *dl = s->scal.as<float>();  // loss_hist[0]
  if ((rc = surr_step_enqueue(s, s->X.as<bf16>(), target, (int)n, 1, nullptr, dl, st)) != FK_OK) return rc;
  if ((rc = surr_check_err(s, st, "surrogate_gradients")) != FK_OK) return rc;
  CK(cudaMemcpy(grad, s->g.p, sizeof(float) * kSurrParams, cudaMemcpyDeviceToHost));
  if (loss) CK(cudaMemcpy(loss, dl, sizeof(float), cudaMemcpyDeviceToHost));
  return FK_OK;
}

extern "C" int surrogate_adam_step(surrogate_t *s, const float *grad, float lr) {
  if (!s || !grad) return fail(FK_ERR_ARG, "surrogate_adam_step: NULL pointer");
  CK(cudaMemcpy(s->g.p, grad, sizeof(float) * kSurrParams, cudaMemcpyHostToDevice));
  ++s->t;
  CK(launch_adam(s->p.as<float>(), s->m.as<float>(), s->v.as<float>(), s->g.as<float>(), kSurrParams, lr, 0.9f,
                 0.999f, 1e-8f, s->t, 0));
  int rc = surr_sync_weights(s, 0);
  if (rc != FK_OK) return rc;
  CK(cudaStreamSynchronize(0));
  return FK_OK;
}

extern "C" int surrogate_forward(surrogate_t *s, const float *q, int64_t n, float *out, void *stream) {
  if (!s || !q || !out) return fail(FK_ERR_ARG, "surrogate_forward: NULL pointer");
  if (n <= 0) return n == 0 ? FK_OK : fail(FK_ERR_ARG, "surrogate_forward: n < 0");
  if (n > INT32_MAX - kBM) return fail(FK_ERR_CAPACITY, "surrogate_forward: n too large");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(s->err.p, 0, 64, st));
  int rc = surr_forward_fused(s, q, n, out, 0, 0.f, nullptr, nullptr, nullptr, nullptr, st);
  if (rc != FK_OK) return rc;
  return surr_check_err(s, st, "surrogate_forward");
}

extern "C" int surrogate_train(surrogate_t *s, fastron_model_t *model, const float *q, int64_t n,
                               const surrogate_train_params *prm, surrogate_stats *stats, void *stream) {
  if (!s || !model || !q || !prm) return fail(FK_ERR_ARG, "surrogate_train: NULL pointer");
  if (model->chain != s->chain) return fail(FK_ERR_ARG, "surrogate_train: model and surrogate use different chains");
  if (model->ns < 0) return fail(FK_ERR_STATE, "surrogate_train: model is untrained");
  const int B = prm->batch;
  if (B < kBM || B % kBM || B > (1 << 16)) return fail(FK_ERR_ARG, "surrogate_train: batch must be a multiple of 128 up to 65536");
  if (prm->epochs < 0 || !(prm->lr > 0.f) || !(prm->holdout >= 0.f && prm->holdout < 1.f))
    return fail(FK_ERR_ARG, "surrogate_train: bad epochs, lr or holdout");
  if (prm->schedule != FK_LR_STEP && prm->schedule != FK_LR_COSINE)
    return fail(FK_ERR_ARG, "surrogate_train: unknown learning-rate schedule %d", prm->schedule);
  const int64_t n_hold = round_up((int64_t)(prm->holdout * (double)n), kBM) <= n ? round_up((int64_t)(prm->holdout * (double)n), kBM) : 0;
  const int64_t n_tr = (n - n_hold) / B * B;
  if (n_tr < B) return fail(FK_ERR_ARG, "surrogate_train: fewer training rows than one batch");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(s->err.p, 0, 64, st));
  // exact targets: the FP32 score of every query (training and held-out rows)
  CK(s->Y.ensure(sizeof(float) * (size_t)n));
  CK(s->lab_tmp.ensure((size_t)n));
  int rc = fk_score(model, q, n, FK_F32, 0, 0.0, s->Y.as<float>(), s->lab_tmp.as<int8_t>(), nullptr, stream);
  if (rc != FK_OK) return rc;
  double *acc = reinterpret_cast<double *>(s->scal.as<char>() + 16);
  CK(cudaMemsetAsync(acc, 0, sizeof(double), st));
  CK(launch_sumsq(s->Y.as<float>(), n_tr, acc, st));
  double ss = 0.0;
  CK(cudaMemcpyAsync(&ss, acc, sizeof ss, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  s->scale = ss > 0.0 ? (float)sqrt(ss / (double)n_tr) : 1.f;
  CK(s->Yh.ensure(sizeof(float) * (size_t)(n_hold > 0 ? n_hold : 1)));
  if (n_hold > 0)
    CK(cudaMemcpyAsync(s->Yh.p, s->Y.as<float>() + (n - n_hold), sizeof(float) * (size_t)n_hold,
                       cudaMemcpyDeviceToDevice, st));
  CK(launch_scale(s->Y.as<float>(), n_tr, 1.f / s->scale, st));
  // features of the training rows
  if ((rc = surr_features(s, q, n_tr, n_tr, s->X, st)) != FK_OK) return rc;
  if ((rc = surr_step_buffers(s, B)) != FK_OK) return rc;
  if (prm->reinit) {
    if ((rc = surr_init_params(s, st)) != FK_OK) return rc;
    if ((rc = surr_sync_weights(s, st)) != FK_OK) return rc;
  }
  const int64_t steps_per_epoch = n_tr / B;
  const int64_t total = steps_per_epoch * prm->epochs;
  CK(s->loss_hist.ensure(sizeof(float) * (size_t)(total > 0 ? total : 1)));
  CK(cudaMemsetAsync(s->tstep.p, 0, 16, st));  // step and block counter
  if (total > 0) {
    // one step captured into a graph (on a library stream), replayed `total`
    // times on st: the batch, learning rate and Adam step come from the
    // device step counter
    SurrSched sch{total, steps_per_epoch, prm->epochs, s->t, prm->lr, prm->schedule == FK_LR_COSINE ? 1 : 0};
    surr_drop_graph(s);
    // graphs of one and of kSurrGraphSteps steps (within a graph each kernel
    // may start while its predecessor drains)
    for (int g = 0; g < 2; ++g) {
      const int nsteps = g == 0 ? 1 : kSurrGraphSteps;
      if (g == 1 && total < nsteps) break;
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < nsteps && rc == FK_OK; ++k)
        rc = surr_step_enqueue(s, s->X.as<bf16>(), s->Y.as<float>(), B, steps_per_epoch, &sch,
                               s->loss_hist.as<float>(), s->cap);
      cudaError_t ec = cudaStreamEndCapture(s->cap, &graph);
      if (rc != FK_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ec != cudaSuccess) return fail(FK_ERR_CUDA, "surrogate_train: capture failed: %s", cudaGetErrorString(ec));
      cudaGraphExec_t *ex = g == 0 ? &s->exec : &s->exec_k;
      ec = cudaGraphInstantiate(ex, graph, 0);
      cudaGraphDestroy(graph);
      if (ec != cudaSuccess) {
        *ex = nullptr;
        return fail(FK_ERR_CUDA, "surrogate_train: instantiate failed: %s", cudaGetErrorString(ec));
      }
    }
    int64_t k = 0;
    if (s->exec_k)
      for (; k + kSurrGraphSteps <= total; k += kSurrGraphSteps) CK(cudaGraphLaunch(s->exec_k, st));
    for (; k < total; ++k) CK(cudaGraphLaunch(s->exec, st));
    s->t += total;
  }
  if ((rc = surr_check_err(s, st, "surrogate_train")) != FK_OK) return rc;
  // calibrate tau on the held-out rows: the largest |pred| with a wrong sign
  float tau = 0.f, fb = 0.f, wrong_rate = 0.f;
  if (n_hold > 0) {
    CK(s->iout.ensure(sizeof(float) * (size_t)n_hold));
    if ((rc = surr_forward_fused(s, q + (n - n_hold) * s->chain->D, n_hold, s->iout.as<float>(), 0, 0.f, nullptr,
                                 nullptr, nullptr, nullptr, st)) != FK_OK)
      return rc;
    CK(launch_scale(s->iout.as<float>(), n_hold, s->scale, st));
    unsigned *tb = reinterpret_cast<unsigned *>(s->scal.as<char>() + 32);
    unsigned long long *wr = reinterpret_cast<unsigned long long *>(s->scal.as<char>() + 40);
    unsigned long long *below = reinterpret_cast<unsigned long long *>(s->scal.as<char>() + 48);
    CK(cudaMemsetAsync(tb, 0, 24, st));
    CK(launch_surr_calibrate(s->iout.as<float>(), s->Yh.as<float>(), n_hold, tb, wr, below, 0.f, st));
    unsigned htb = 0;
    unsigned long long hwr = 0;
    CK(cudaMemcpyAsync(&htb, tb, sizeof htb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hwr, wr, sizeof hwr, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memcpy(&tau, &htb, sizeof tau);
    CK(launch_count_below(s->iout.as<float>(), n_hold, tau, below, st));
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, below, sizeof hb, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    fb = (float)((double)hb / (double)n_hold);
    wrong_rate = (float)((double)hwr / (double)n_hold);
    if ((rc = surr_check_err(s, st, "surrogate_train")) != FK_OK) return rc;
  }
  s->tau = tau;
  if (stats) {
    std::vector<float> lh((size_t)(total > 0 ? total : 0));
    if (total > 0) CK(cudaMemcpy(lh.data(), s->loss_hist.p, sizeof(float) * lh.size(), cudaMemcpyDeviceToHost));
    stats->steps = total;
    stats->loss_first = total > 0 ? lh.front() : 0.f;
    float tail = 0.f;
    const int64_t k = total < steps_per_epoch ? total : steps_per_epoch;
    for (int64_t i = total - k; i < total; ++i) tail += lh[(size_t)i];
    stats->loss_last = k > 0 ? tail / (float)k : 0.f;
    stats->scale = s->scale;
    stats->tau = tau;
    stats->holdout_sign_error = wrong_rate;
    stats->holdout_fallback = fb;
    stats->n_train = n_tr;
    stats->n_holdout = n_hold;
  }
  return FK_OK;
}

extern "C" int surrogate_infer(surrogate_t *s, fastron_model_t *model, const float *q, int64_t n, double tau,
                               int8_t *label, float *pred, int64_t *n_fallback, void *stream) {
  if (!s || !model || !label) return fail(FK_ERR_ARG, "surrogate_infer: NULL pointer");
  if (model->chain != s->chain) return fail(FK_ERR_ARG, "surrogate_infer: model and surrogate use different chains");
  if (model->ns < 0) return fail(FK_ERR_STATE, "surrogate_infer: model is untrained");
  if (n < 0) return fail(FK_ERR_ARG, "surrogate_infer: n < 0");
  if (n_fallback) *n_fallback = 0;
  if (n == 0) return FK_OK;
  if (!q) return fail(FK_ERR_ARG, "surrogate_infer: q is NULL");
  if (n > INT32_MAX - kBM) return fail(FK_ERR_CAPACITY, "surrogate_infer: n too large");
  const float t = tau > 0.0 ? (float)tau : s->tau;
  if (!(t >= 0.f)) return fail(FK_ERR_STATE, "surrogate_infer: no threshold (train with a holdout or pass tau > 0)");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(s->err.p, 0, 64, st));
  CK(s->fb_idx.ensure(sizeof(int32_t) * (size_t)n));
  CK(s->fb_cnt.ensure(sizeof(int32_t) * 2));
  CK(cudaMemsetAsync(s->fb_cnt.p, 0, sizeof(int32_t), st));
  // features, network and decision in one launch
  int rc = surr_forward_fused(s, q, n, nullptr, 1, t, pred, label, s->fb_idx.as<int32_t>(), s->fb_cnt.as<int32_t>(),
                              st);
  if (rc != FK_OK) return rc;
  int32_t nfb = 0;
  CK(cudaMemcpyAsync(&nfb, s->fb_cnt.p, sizeof nfb, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if ((rc = surr_check_err(s, st, "surrogate_infer")) != FK_OK) return rc;
  if (nfb > 0) {
    const int D = s->chain->D;
    CK(s->fb_q.ensure(sizeof(float) * (size_t)nfb * D));
    CK(s->fb_lab.ensure((size_t)nfb));
    CK(s->fb_f.ensure(sizeof(float) * (size_t)nfb));
    CK(launch_gather_rows(q, D, s->fb_idx.as<int32_t>(), nfb, s->fb_q.as<float>(), st));
    rc = fk_score(model, s->fb_q.as<float>(), nfb, FK_F32, 1, 0.0, s->fb_f.as<float>(), s->fb_lab.as<int8_t>(),
                  nullptr, stream);
    if (rc != FK_OK) return rc;
    CK(launch_scatter_labels(s->fb_lab.as<int8_t>(), s->fb_f.as<float>(), s->fb_idx.as<int32_t>(), nfb, label, pred,
                             st));
  }
  if (n_fallback) *n_fallback = nfb;
  return FK_OK;
}

// ------------------------------------------------------ batched scenes ---
namespace fk {
int batched_num_variants();
int batched_block_queries(int v);
bool batched_supported(int mv);
size_t scene_dev_size();
size_t work_item_size();
void fill_scene_dev(void *dst, const ChainF &cf, const ChainD &cd, const void *rec, const float *sdf,
                    const double *cp64, const double *alpha, int64_t ns, const int32_t *npair_pos, double gamma,
                    float eps0, float eps1, float cnorm, int64_t q_off, int64_t n);
void fill_work_item(void *dst, int32_t scene, int32_t block);
cudaError_t launch_batched_score_args(int mv, int variant, const void *scenes, const void *items, int32_t n_items,
                                      int32_t *counter, const float *q, float *f, int8_t *label,
                                      int32_t *band_idx, int32_t *band_scene, int32_t *band_cnt, int32_t *err,
                                      uint32_t wait_limit, int circ, cudaStream_t s, bool prepare_only);
cudaError_t launch_batched_rescore_args(const void *scenes, const float *q, const int32_t *band_idx,
                                        const int32_t *band_scene, const int32_t *band_cnt, float *f, int8_t *label,
                                        cudaStream_t s);
cudaError_t launch_batched_rescore_df_args(const void *scenes, const float *q, const int32_t *band_idx,
                                           const int32_t *band_scene, const int32_t *band_cnt, double eps2, float *f,
                                           int8_t *label, int32_t *band2_idx, int32_t *band2_scene,
                                           int32_t *band2_cnt, cudaStream_t s);
}  // namespace fk

struct fk_batch {
  int n_scenes = 0, mv = 0, D = 0;
  std::vector<fastron_model *> models;
  DevBuf scenes, items, flags, band_idx, band_scene, band2_idx, band2_scene;
  std::vector<char> scenes_h, items_h;
  int32_t n_items = 0;
  std::vector<int64_t> off;  // query offsets of the current work list
  int variant = 0;
  int circ = 0;  // the plan's scenes are scored in the circle form (set by batch_plan)
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const float *g_q = nullptr;
  float *g_f = nullptr;
  int8_t *g_label = nullptr;
  int g_rescore = -1, g_variant = -1;
};

static void batch_drop_graph(fk_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

extern "C" int fk_batch_create(fastron_model_t *const *models, int n_scenes, fk_batch_t **out) {
  if (!out) return fail(FK_ERR_ARG, "fk_batch_create: out is NULL");
  *out = nullptr;
  if (!models || n_scenes < 1) return fail(FK_ERR_ARG, "fk_batch_create: need at least one model");
  const fastron_model *m0 = models[0];
  if (!m0) return fail(FK_ERR_ARG, "fk_batch_create: model 0 is NULL");
  for (int i = 0; i < n_scenes; ++i) {
    const fastron_model *m = models[i];
    if (!m) return fail(FK_ERR_ARG, "fk_batch_create: model %d is NULL", i);
    if (m->ns < 0) return fail(FK_ERR_STATE, "fk_batch_create: model %d is untrained", i);
    if (m->chain->D != m0->chain->D || m->chain->cf.Mv != m0->chain->cf.Mv)
      return fail(FK_ERR_ARG, "fk_batch_create: model %d has another DOF or control-point count", i);
    if (m->gamma > 1e7) return fail(FK_ERR_ARG, "fk_batch_create: model %d gamma out of range", i);
    if (m->summand != FK_SUMMAND_RQ)
      return fail(FK_ERR_ARG, "fk_batch_create: model %d uses the Gaussian summand (batches take the RQ kernel only)", i);
  }
  if (!batched_supported(m0->chain->cf.Mv))
    return fail(FK_ERR_ARG, "fk_batch_create: %d configuration-dependent control points is not a compiled shape",
                m0->chain->cf.Mv);
  fk_batch *b = new fk_batch;
  b->n_scenes = n_scenes;
  b->mv = m0->chain->cf.Mv;
  b->D = m0->chain->D;
  b->models.assign(models, models + n_scenes);
  b->scenes_h.resize(scene_dev_size() * (size_t)n_scenes);
  cudaError_t e = b->scenes.ensure(b->scenes_h.size());
  if (e == cudaSuccess) e = b->flags.ensure(sizeof(int32_t) * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fk_batch_destroy(b);
    return fail(FK_ERR_CUDA, "fk_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return FK_OK;
}

extern "C" void fk_batch_destroy(fk_batch_t *b) {
  if (!b) return;
  batch_drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  b->scenes.release();
  b->items.release();
  b->flags.release();
  b->band_idx.release();
  b->band_scene.release();
  b->band2_idx.release();
  b->band2_scene.release();
  delete b;
}

// Rebuilds the scene records and the cost-sorted work list for new offsets.
static int batch_plan(fk_batch *b, const int64_t *q_off) {
  const int bq = batched_block_queries(b->variant);
  std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>> it;
  // the circle form when every scene qualifies (score_circle), else none
  b->circ = b->n_scenes > 0 && (b->mv == 7 || b->mv == 11);
  for (int i = 0; i < b->n_scenes; ++i)
    b->circ = b->circ && score_circle(b->models[i]->chain, b->models[i]->summand, b->models[i]->gamma,
                                      b->models[i]->ns) > 0.f;
  for (int i = 0; i < b->n_scenes; ++i) {
    const fastron_model *m = b->models[i];
    const int64_t n = q_off[i + 1] - q_off[i];
    float eps0 = 0.f, eps1 = 0.f;
    score_band(m->chain->cf, m->summand, m->gamma, m->ns, false, 0.0, &eps0, &eps1);
    const float cnorm = b->circ ? score_circle(m->chain, m->summand, m->gamma, m->ns) : 0.f;
    fill_scene_dev(b->scenes_h.data() + scene_dev_size() * i, m->chain->cf, m->chain->cd, m->rec.p, m->sdf.as<float>(),
                   m->cp64.as<double>(), m->alpha_s.as<double>(), m->ns, m->npos.as<int32_t>(), m->gamma, eps0, eps1,
                   cnorm, q_off[i], n);
    for (int64_t blk = 0; blk * bq < n; ++blk) {
      const int64_t qn = n - blk * bq < bq ? n - blk * bq : bq;
      it.push_back({(m->ns + 1) * qn, {i, (int32_t)blk}});
    }
  }
  std::stable_sort(it.begin(), it.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
  b->n_items = (int32_t)it.size();
  b->items_h.resize(work_item_size() * (it.size() > 0 ? it.size() : 1));
  for (size_t k = 0; k < it.size(); ++k) fill_work_item(b->items_h.data() + work_item_size() * k, it[k].second.first, it[k].second.second);
  CK(cudaDeviceSynchronize());  // earlier launches may still read the old plan
  CK(b->items.ensure(b->items_h.size()));
  CK(cudaMemcpy(b->scenes.p, b->scenes_h.data(), b->scenes_h.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->items.p, b->items_h.data(), b->items_h.size(), cudaMemcpyHostToDevice));
  b->off.assign(q_off, q_off + b->n_scenes + 1);
  batch_drop_graph(b);
  return FK_OK;
}

// Enqueues the batched work on stream s (flags cleared, score, re-score).
static int batch_enqueue(fk_batch *b, const float *q, float *f, int8_t *label, int rescore, cudaStream_t s) {
  int32_t *fl = b->flags.as<int32_t>();
  CK(cudaMemsetAsync(fl, 0, sizeof(int32_t) * 4, s));
  CK(launch_batched_score_args(b->mv, b->variant, b->scenes.p, b->items.p, b->n_items, fl, q, f, label,
                               rescore ? b->band_idx.as<int32_t>() : nullptr,
                               rescore ? b->band_scene.as<int32_t>() : nullptr, fl + 1, fl + 2, g_wait_limit, b->circ,
                               s, false));
  if (rescore) {
    // double-float first; what it cannot decide goes to FP64 (count in fl[3])
    CK(launch_batched_rescore_df_args(b->scenes.p, q, b->band_idx.as<int32_t>(), b->band_scene.as<int32_t>(), fl + 1,
                                      kDefaultEpsDf, f, label, b->band2_idx.as<int32_t>(),
                                      b->band2_scene.as<int32_t>(), fl + 3, s));
    CK(launch_batched_rescore_args(b->scenes.p, q, b->band2_idx.as<int32_t>(), b->band2_scene.as<int32_t>(), fl + 3,
                                   f, label, s));
  }
  return FK_OK;
}

extern "C" int fk_score_batched(fk_batch_t *b, const float *q, const int64_t *q_off, int rescore, float *f,
                                int8_t *label, int64_t *n_rescored, void *stream) {
  if (!b || !q_off) return fail(FK_ERR_ARG, "fk_score_batched: NULL pointer");
  if (q_off[0] != 0) return fail(FK_ERR_ARG, "fk_score_batched: q_off[0] must be 0");
  for (int i = 0; i < b->n_scenes; ++i)
    if (q_off[i + 1] < q_off[i]) return fail(FK_ERR_ARG, "fk_score_batched: q_off must not decrease");
  const int64_t total = q_off[b->n_scenes];
  if (total > (int64_t)INT32_MAX) return fail(FK_ERR_CAPACITY, "fk_score_batched: more than 2^31 - 1 queries");
  if (n_rescored) *n_rescored = 0;
  if (total == 0) return FK_OK;
  if (!q || !label) return fail(FK_ERR_ARG, "fk_score_batched: q and label must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->off.size() != (size_t)b->n_scenes + 1 || !std::equal(b->off.begin(), b->off.end(), q_off)) {
    int rc = batch_plan(b, q_off);
    if (rc != FK_OK) return rc;
  }
  if (rescore) {
    const void *before[4] = {b->band_idx.p, b->band_scene.p, b->band2_idx.p, b->band2_scene.p};
    CK(b->band_idx.ensure(sizeof(int32_t) * (size_t)total));
    CK(b->band_scene.ensure(sizeof(int32_t) * (size_t)total));
    CK(b->band2_idx.ensure(sizeof(int32_t) * (size_t)total));
    CK(b->band2_scene.ensure(sizeof(int32_t) * (size_t)total));
    const void *after[4] = {b->band_idx.p, b->band_scene.p, b->band2_idx.p, b->band2_scene.p};
    if (!std::equal(before, before + 4, after)) batch_drop_graph(b);  // the captured graph holds the old pointers
  }
  // replay the captured graph when nothing it depends on has changed
  if (!b->exec || b->g_q != q || b->g_f != f || b->g_label != label || b->g_rescore != (rescore != 0) ||
      b->g_variant != b->variant) {
    batch_drop_graph(b);
    CK(launch_batched_score_args(b->mv, b->variant, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, nullptr, 0, b->circ, s, true));
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue(b, q, f, label, rescore, b->cap);
    cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
    if (rc != FK_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(FK_ERR_CUDA, "fk_score_batched: capture failed: %s", cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) {
      b->exec = nullptr;
      return fail(FK_ERR_CUDA, "fk_score_batched: instantiate failed: %s", cudaGetErrorString(ec));
    }
    b->g_q = q;
    b->g_f = f;
    b->g_label = label;
    b->g_rescore = rescore != 0;
    b->g_variant = b->variant;
  }
  CK(cudaGraphLaunch(b->exec, s));
  if (n_rescored) {
    int32_t h[4];
    CK(cudaMemcpyAsync(h, b->flags.p, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[2] & kErrTimeout) return fail(FK_ERR_TIMEOUT, "fk_score_batched: a shared-memory tile wait timed out");
    *n_rescored = rescore ? h[1] : 0;
  }
  return FK_OK;
}

extern "C" int fk_batch_tune(fk_batch_t *b, const float *q, const int64_t *q_off, int8_t *label, float *ms,
                             int cap, int *best) {
  if (!b || !q || !q_off || !label) return fail(FK_ERR_ARG, "fk_batch_tune: NULL pointer");
  const int nv = batched_num_variants();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_ms = 0.f;
  int best_v = 0;
  for (int v = 0; v < nv; ++v) {
    b->variant = v;
    b->off.clear();  // block size depends on the variant: rebuild the plan
    int rc = fk_score_batched(b, q, q_off, 1, nullptr, label, nullptr, b->cap);
    if (rc != FK_OK) return rc;
    float t = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0, b->cap));
      rc = fk_score_batched(b, q, q_off, 1, nullptr, label, nullptr, b->cap);
      if (rc != FK_OK) return rc;
      CK(cudaEventRecord(e1, b->cap));
      CK(cudaEventSynchronize(e1));
      float x = 0.f;
      CK(cudaEventElapsedTime(&x, e0, e1));
      t = x < t ? x : t;
    }
    if (ms && v < cap) ms[v] = t;
    if (v == 0 || t < best_ms) {
      best_ms = t;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = best_v;
  b->off.clear();
  batch_drop_graph(b);
  if (best) *best = best_v;
  return FK_OK;
}
