/*
 * fkfast: forward-kinematics (FK) kernel proxy collision checking on one
 * GB300 GPU.  C ABI of libfkfast.so.
 *
 * Method: Das and Yip, "Forward Kinematics Kernel for Improved Proxy
 * Collision Checking", arXiv 1910.06451.  Sections and equations below refer
 * to that paper.
 *
 * Conventions for every call:
 *   - Pointers marked "device" are CUDA device pointers owned by the caller;
 *     pointers marked "host" are ordinary host memory owned by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it in call order; a call returns
 *     once its work is enqueued, except where an output is host memory, in
 *     which case the call synchronises `stream` before returning.
 *   - Arrays are dense and row-major unless stated otherwise.
 *   - Return value 0 (FK_OK) on success, a negative FK_ERR_* code otherwise;
 *     fk_last_error() then describes the failure (thread-local string).  No
 *     call falls back to the CPU.
 *   - Handles (fk_chain_t, fastron_model_t) own their device workspaces.  A
 *     handle may be used from one stream at a time; calls on one handle from
 *     different streams must be ordered by the caller.
 *   - Labels are int8: +1 = in collision (C_obs), -1 = free (C_free)
 *     (Sec. II-B).  A score f = 0 is labelled +1.
 */
#ifndef FKFAST_H
#define FKFAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FK_OK 0
#define FK_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, unsupported shape) */
#define FK_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define FK_ERR_CAPACITY (-3)  /* a size exceeds the handle's or the library's limit */
#define FK_ERR_TIMEOUT (-4)   /* a bounded wait inside a kernel gave up */
#define FK_ERR_STATE (-5)     /* handle not ready for this call (e.g. untrained model) */

#define FK_REVOLUTE 0
#define FK_PRISMATIC 1

#define FK_F32 0  /* FP32 arithmetic */
#define FK_F64 1  /* FP64 arithmetic */
#define FK_F16 2  /* packed FP16 distances, FP32 reciprocals and sums (fk_score only) */
#define FK_DF64 3 /* FP64 inputs and outputs, double-float arithmetic on the FP32 pipes (fk_gram, training) */
#define FK_DF32 4 /* as FK_DF64, each result rounded to FP32 once: the kernel matrix stored in
                     single precision (fk_gram: float K; training: half the memory) */

#define FK_LR_STEP 0   /* surrogate_train_params.schedule */
#define FK_LR_COSINE 1

#define FK_SUMMAND_RQ 0     /* the paper's summand: the RQ kernel of Eq. 3 (default) */
#define FK_SUMMAND_GAUSS 1  /* not in the paper: exp(-gamma/2 |x - x'|^2) (fk_chain_set_summand) */

#define FK_MAX_DOF 16
#define FK_MAX_CP 32

/* One standard Denavit-Hartenberg link (Eq. 1).  For a revolute joint the
 * joint value adds to theta0; for a prismatic joint it adds to d. */
typedef struct {
    double a, alpha, d, theta0;
    int32_t type; /* FK_REVOLUTE or FK_PRISMATIC */
    int32_t reserved;
} fk_dh;

/* One control point (Eq. 2): position of frame `joint` (0 = base frame,
 * i = frame of joint i) offset by the static translation t (in that frame). */
typedef struct {
    int32_t joint;
    int32_t reserved;
    double t[3];
} fk_cp;

typedef struct fk_chain fk_chain_t;
typedef struct fastron_model fastron_model_t;

/* Text of the last error on this thread ("" if none). */
const char *fk_last_error(void);

/* ---- kinematic chain ---------------------------------------------------
 * Builds a chain from D links (host array, 1 <= D <= FK_MAX_DOF), the
 * world-from-frame-0 transform base4x4 (host, 16 doubles, row-major; NULL =
 * identity) and M control points (host array, 1 <= M <= FK_MAX_CP, joint in
 * [0, D]).  The paper places control points at joint-frame origins (T_m = I,
 * Sec. III-A); any offsets are accepted.  *out receives the handle. */
int fk_chain_create(const fk_dh *dh, int D, const double *base4x4, const fk_cp *cps, int M, fk_chain_t **out);
void fk_chain_destroy(fk_chain_t *chain);

/* Summand of the FK kernel (Eq. 4) for every later call on this chain:
 * FK_SUMMAND_RQ (the default) is the paper's RQ kernel of Eq. 3;
 * FK_SUMMAND_GAUSS replaces it by exp(-gamma/2 |x - x'|^2), keeping the mean
 * over control points.  The Gaussian summand is NOT the paper's kernel; it is
 * offered as an alternative (it is the kernel family whose exponential the
 * MUFU ex2 unit and its packed-half form evaluate directly).  With it:
 *   - fk_gram accepts FK_F64 and FK_F32 only (no double-float form), and
 *     fastron_train builds its matrix in FP64 (gram 0 selects FK_F64;
 *     FK_DF64/FK_DF32 are rejected);
 *   - fk_score (FK_F32 and FK_F16) evaluates 2^(-|d'|^2) with d' the control
 *     points scaled by sqrt(gamma/2 log2 e), on MUFU ex2 (FK_F16: ex2.f16x2);
 *     the band is re-scored in double-float (a pair-arithmetic 2^(-t)),
 *     then in FP64;
 *   - fk_batch_create rejects its models (FK_ERR_ARG).
 * A model keeps the summand it was trained or set with.  Returns FK_ERR_ARG
 * for an unknown summand or a chain whose shape has no Gaussian score kernel
 * (compiled for 3, 7 and 11 configuration-dependent control points). */
int fk_chain_set_summand(fk_chain_t *chain, int summand);

/* ---- forward kinematics (Sec. II-A, Eqs. 1-2) --------------------------
 * q: device, n x D joint values.  cp: device, control-point positions in
 * structure-of-arrays layout [M][3][n] (coordinate c of point m of
 * configuration k at cp[(m*3 + c)*n + k]).  n = 0 is a no-op. */
int fk_forward(const fk_chain_t *chain, const float *q, int64_t n, float *cp, void *stream);
int fk_forward_f64(const fk_chain_t *chain, const double *q, int64_t n, double *cp, void *stream);

/* ---- kernel matrix (Sec. II-B with the FK kernel of Eq. 4) -------------
 * K[i][j] = K_FK(Xa_i, Xb_j) = (1/M) sum_m (1 + gamma/2 |FK_m(Xa_i) - FK_m(Xb_j)|^2)^-2.
 * precision FK_F64: Xa, Xb are device double arrays (na x D, nb x D) and K a
 * device double array na x nb.  FK_DF64: the same FP64 inputs and output,
 * computed in double-float arithmetic (pairs of FP32 values, error-free
 * transformations; entries within about 1e-13 of the FP64 ones, some ten
 * times faster on this part, whose FP64 rate is 1/64 of its FP32 rate).
 * FK_DF32: FP64 inputs, a device float K holding each FK_DF64 entry rounded to
 * FP32 once.  FK_F32: float inputs and a float K.  gamma > 0.
 * Control points are computed into the chain's workspace first. */
int fk_gram(const fk_chain_t *chain, const void *Xa, int64_t na, const void *Xb, int64_t nb, double gamma,
            int precision, void *K, void *stream);

/* ---- Fastron model (Sec. III-B) ---------------------------------------- */
typedef struct {
    double gamma;      /* FK kernel width, > 0 (Eq. 3) */
    double beta;       /* conditional bias, >= 1 (Eq. 5): b_i = beta for y_i = +1, 1 otherwise */
    int64_t iter_max;  /* iteration limit of Algorithm 1, >= 0 */
    int64_t s_max;     /* support-set size limit S_max of Algorithm 1, >= 1 */
    int32_t warm_start;/* loadPreviousModel: 1: start from this model's alpha and F of the
                          previous call on the same training set; 2: the training set has
                          changed and its first |S| rows are this model's support points in
                          the model's order (as fk_active_samples writes them): they keep
                          their weights, the other rows start at 0, and F = K alpha is
                          computed on the device; 0: alpha = F = 0 */
    int32_t trace;     /* 1: record every pass (kind, index, change of alpha) for
                          fastron_model_trace; 0: do not */
    int32_t gram;      /* arithmetic and storage of the training kernel matrix: FK_DF64
                          (0 selects it) or FK_F64, both stored in FP64 (N^2 doubles), or
                          FK_DF32, stored in FP32 (N^2 floats; 17.2 GB at N = 65,536) */
    int32_t reuse_gram;/* 1: X is the training set of this model's previous call, with the same
                          N and gram: its stored kernel matrix is used again instead of being
                          rebuilt (a changing environment relabels a fixed training set).  X
                          must be the same device buffer as in the call that built the matrix
                          (else FK_ERR_STATE), with unchanged contents (not checked);
                          0: build it */
} fastron_params;

typedef struct {
    int64_t iterations; /* passes of Algorithm 1 that changed alpha */
    int64_t adds;       /* add/adjust steps (Eqs. 6-8) */
    int64_t removes;    /* redundant-support removals */
    int64_t n_support;  /* |S| after removeNonsupportPoints */
    int32_t converged;  /* 1 if every training margin y_i F_i > 0 and no removal applied */
    int32_t reserved;
} fastron_stats;

/* Creates an empty (untrained) model bound to `chain`; the chain must outlive it. */
int fastron_model_create(const fk_chain_t *chain, fastron_model_t **out);
void fastron_model_destroy(fastron_model_t *model);

/* Algorithm 1.  X: device double, N x D training configurations; y: device
 * int8 labels (+1/-1), N >= 1.  The FP64 kernel matrix of X is built on the
 * device, then the greedy coordinate descent runs in one persistent kernel:
 * argmin of the margins y_i F_i (lowest index wins ties; a margin <= 0 is a
 * misclassification), add/adjust alpha_i by b_i y_i - F_i and F by that times
 * column i, subject to S_max; otherwise remove the support point with the
 * largest y_i (F_i - alpha_i) > 0 (lowest index wins ties); stop when neither
 * applies or after iter_max passes.  alpha and F are FP64.  The support set
 * (ascending training indices with alpha != 0) and its weights become the
 * model.  stats: host, may be NULL; filling it synchronises `stream`.
 * The kernel matrix is stored (N^2 entries of 8 or 4 bytes, see gram) and
 * kept with the model.  Requires N <= 65,536, else FK_ERR_CAPACITY; the
 * matrix must fit in device memory, else FK_ERR_CUDA.  Sizes above 32,768
 * need a 16-CTA thread-block cluster.  The CTAs of the cluster exchange
 * their candidates through shared-memory barriers polled at most
 * fk_set_wait_limit times per pass; if one runs out the call returns
 * FK_ERR_TIMEOUT, the model keeps its previous support set, and the
 * incomplete weights and margins are discarded (no warm start or matrix
 * reuse follows from them). */
int fastron_train(fastron_model_t *model, const double *X, const int8_t *y, int64_t N, const fastron_params *p,
                  fastron_stats *stats, void *stream);

/* Two-stage active learning (Sec. III-B, after Algorithm 1): the next
 * training set from this model's support set S (|S| = ns rows).  X: device
 * double [rows][D], rows = ns (1 + k_near) + n_uniform, laid out as
 *   rows [0, ns)                    the support configurations, in the
 *                                   model's order (for warm_start = 2);
 *   rows ns + c ns + s, c < k_near  support point s with every joint moved by
 *                                   a draw uniform in [-sigma, sigma] and
 *                                   clipped to [-qlim, qlim] (stage 1: small
 *                                   changes of the C-space obstacles);
 *   the last n_uniform rows         configurations uniform in [-qlim, qlim]
 *                                   (stage 2: obstacles entering the workspace).
 * Draws: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based
 * generator; draw k of stream `seed` is the finaliser of
 * seed + (k + 1) * 0x9E3779B97F4A7C15, top 53 bits scaled to [0, 1), mapped to
 * [lo, hi) as lo + (hi - lo) u in FP64.  Draw (c ns + s) D + d moves joint d
 * of support point s in copy c; draw k_near ns D + i D + d is joint d of
 * uniform sample i.  New values are rounded to FP32 once (so the FP32 copy
 * X32, device float [rows][D] or NULL, holds the same configurations).
 * cap: rows X can hold; *n_out (host) receives rows; rows > cap is
 * FK_ERR_CAPACITY.  The model must be trained or set (FK_ERR_STATE). */
int fk_active_samples(const fastron_model_t *model, int32_t k_near, double sigma, int64_t n_uniform, double qlim,
                      uint64_t seed, double *X, float *X32, int64_t cap, int64_t *n_out, void *stream);

/* Copies the per-pass record of the last fastron_train call made with
 * p->trace = 1: kind (host int8: 1 add/adjust, 2 removal), idx (host int64,
 * training index) and delta (host double, change of alpha_i) for up to cap
 * passes; *n receives the number of passes.  Any output may be NULL except n.
 * Synchronous. */
int fastron_model_trace(const fastron_model_t *model, int8_t *kind, int64_t *idx, double *delta, int64_t cap,
                        int64_t *n);

/* Replaces the model by the given support set: q host double ns x D
 * configurations, alpha host double ns weights, kernel width gamma.  Used to
 * score a model trained elsewhere.  Synchronous. */
int fastron_model_set(fastron_model_t *model, const double *q, const double *alpha, int64_t ns, double gamma);

/* Copies src's support set, as packed for scoring (configurations, weights,
 * gamma, training indices), into dst, which must use the same chain: dst can
 * then be scored while src trains again (for example on another stream), the
 * double buffer of a pipelined update/query loop.  dst's own training state
 * (kernel matrix, margins) is dropped; it cannot be warm-started.  The device
 * copies are enqueued on `stream` after whatever is queued there (src's
 * training, if it ran on that stream); dst must not be in use by another
 * stream meanwhile.  Returns FK_ERR_STATE if src is untrained.  Not part of
 * the paper: a device-side form of its model handover between updates. */
int fastron_model_copy(fastron_model_t *dst, const fastron_model_t *src, void *stream);

/* Copies the support set out: idx (host int64, training indices; NULL
 * allowed) and alpha (host double) for up to cap entries; *ns receives |S|.
 * Synchronous. */
int fastron_model_get(const fastron_model_t *model, int64_t *idx, double *alpha, int64_t cap, int64_t *ns);

/* ---- proxy collision check (Sec. III-B) --------------------------------
 * f(q) = sum_{s in S} alpha_s K_FK(S_s, q); label = +1 if f >= 0 else -1.
 * q: device float, n x D.  label: device int8 [n].  f: device float [n] or NULL.
 * precision FK_F32: FK of each query and the kernel sums run in FP32; a bound
 * B(q) = sum_s |alpha_s| K_FK(S_s, q) is accumulated beside f.
 * rescore != 0: every query with |f| <= eps(q) B(q) (the FP32 band, see
 * fk_score_band) is evaluated again, and its f and label are replaced, so
 * that labels equal an FP64 evaluation: first in double-float arithmetic
 * (FP64 kinematics, summands and sums as FP32 pairs, ~1e-13 relative), then,
 * for the queries it leaves within 1e-9 B(q) of zero, in FP64 (FK and
 * kernel).  The call reads the band size back, so it synchronises `stream`
 * once.  rescore_eps <= 0 selects the derived bound of fk_score_band (the
 * labels are then exact); rescore_eps > 0 replaces it by the constant
 * eps(q) = rescore_eps (no guarantee below the bound).  n_rescored (host, may
 * be NULL) receives the size of the FP32 band; filling it synchronises
 * `stream`.
 * With rescore = 0 and n_rescored NULL the call does not synchronise and
 * does not read the error word: a shared-memory tile wait that gave up
 * (FK_ERR_TIMEOUT on the other paths) then goes unreported and the labels
 * are undefined; pass n_rescored to have it checked.
 * precision FK_F16: the differences and t = 1 + gamma/2 |p - s|^2 are
 * computed in packed half precision, the rest in FP32; with rescore != 0 every
 * query with |f| <= eps(q) B(q) (the half band of fk_score_band) goes through the FP32
 * path above (and its FP64 re-score), so the labels are again those of an
 * FP64 evaluation; n_rescored then counts the queries of the half pass's
 * band.  The call synchronises `stream` once when rescore != 0. */
int fk_score(fastron_model_t *model, const float *q, int64_t n, int precision, int rescore, double rescore_eps,
             float *f, int8_t *label, int64_t *n_rescored, void *stream);

/* The default FP32 band of fk_score (Sec. III-B label rule made exact): the
 * kernel sends a query to the re-score when |f| <= eps(q) B(q) with
 * eps(q) = eps0 + eps1 (|p(q)| + |s|max), |p(q)| the largest norm of the
 * query's configuration-dependent control points and |s|max that of the
 * support set's, both in coordinates scaled by sqrt(gamma/2).  eps(q)
 * bounds the kernel's whole error |f~ - f| / B(q) (kinematics, summands,
 * reciprocals, accumulation), so every label it decides without the
 * re-score is the sign of the exact f.  precision FK_F32 or FK_F16; for the
 * non-paper Gaussian summand the bands are measured, not derived (eps1 = 0).
 * eps0, eps1: host out. */
int fk_score_band(const fastron_model_t *model, int precision, double *eps0, double *eps1);

/* The circle term of the FP32 band (Sec. II-A, Eqs. 1-2 for link 1; the RQ
 * summand of Eq. 3).  When the first configuration-dependent control point
 * sits on frame 1 and joint 1 is revolute, the point moves on a circle of
 * radius rho about that joint's axis, and |p - s| = 2 rho |sin((theta -
 * theta_s) / 2)|.  fk_score with precision FK_F32 then computes that point's
 * summand in this form, which takes three FP32 operations in place of six,
 * and uses eps(q) = eps0 + eps1 max(|p(q)| + |s|max, cnorm) with
 * cnorm = 6 rho sqrt(gamma/2).  The derivation is in the source beside
 * score_circle.  *cnorm = 0 means every point is in the direct form.
 * The circle form is used when the chain qualifies, the summand is RQ,
 * 0 < rho sqrt(gamma/2) <= 4, the support set has at least 128 points (below
 * that the per-query sine and cosine cost more than the form saves), and
 * fk_set_circle_form has not switched it off.  cnorm: host out.  Errors: FK_ERR_ARG for NULL pointers,
 * FK_ERR_STATE for an untrained model. */
int fk_score_circle(const fastron_model_t *model, double *cnorm);

/* Switches the circle form of fk_score_circle on (on != 0, the default) or
 * off for all later FP32 score calls in this process.  With it off, every
 * point takes the direct form and eps(q) = eps0 + eps1 (|p(q)| + |s|max).
 * The labels are exact either way.  Always returns FK_OK. */
int fk_set_circle_form(int on);

/* fk_score with rescore = 1 for callers that must not allocate device memory
 * while they score (a real-time planner loop, a process whose device memory
 * is handed to a fixed pool, code under a budget fixed at start-up).  The
 * paper has no counterpart: this is a deployment variant of the same two
 * kernels.  fk_score may grow the model's band buffer with cudaMalloc; this
 * call allocates nothing.  Its scratch (band counter, error word, band list)
 * is one static device array of 1,048,576 + 64 int32 (about 4 MiB) that every
 * GPU loading the library holds until the process exits.  Limits and rules:
 *   - n <= 1,048,576 queries per call, else FK_ERR_CAPACITY (split larger
 *     batches into several calls);
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress): make that first call before any stream capture;
 *   - every call on a device shares the one array: calls whose GPU work
 *     overlaps (e.g. on two streams without ordering) race and corrupt each
 *     other's band lists; order them on one stream;
 *   - the model must have been trained or set beforehand (its own buffers are
 *     allocated by fastron_train / fastron_model_set, not here);
 *   - every call reads its error word back, so it synchronises `stream` once
 *     and returns FK_ERR_TIMEOUT if a tile wait gave up;
 *   - the array's address is cached per device for the life of the process:
 *     do not call this after a cudaDeviceReset of that device.
 * Arguments and results are those of fk_score with precision FK_F32 and
 * rescore = 1. */
int fk_score_noalloc(fastron_model_t *model, const float *q, int64_t n, double rescore_eps, float *f, int8_t *label,
                     int64_t *n_rescored, void *stream);

/* ---- premises of the band of fk_score_band -----------------------------
 * The derivation of the band takes three facts about the arithmetic of the
 * score kernel; these calls let a test check them on the device that scores.
 * They are not part of the paper's method.
 *
 * fk_check_rcp: max |rcp(x) x - 1| of the kernel's MUFU reciprocal
 * (rcp.approx.ftz.f32) over every FP32 mantissa of the binades
 * [2^e_lo, 2^(e_hi + 1)), -126 <= e_lo <= e_hi <= 127.  The bound assumes
 * 2^-23.  Synchronous; max_rel host out.
 * fk_check_sincos: max absolute error of the kernels' pair-arithmetic sine
 * and cosine of x + theta0 against FP64, over every FP32 x in [-hi, hi]
 * (|theta0| + hi < 2^16).  Synchronous; max_abs host out.
 * fk_forward_dd: the configuration-dependent control points (Eq. 2) of n
 * configurations q (device float, n x D) as the score kernels form them:
 * pair-arithmetic kinematics times `scale`, rounded once to FP32; cp device
 * float SoA [Mv][3][n] (Mv = points not fixed to the base, in chain order).
 * Stream-ordered. */
int fk_check_rcp(int e_lo, int e_hi, double *max_rel);
int fk_check_sincos(float hi, double theta0, double *max_abs);
int fk_forward_dd(const fk_chain_t *chain, const float *q, int64_t n, double scale, float *cp, void *stream);

/* ---- ground-truth labels (geometric checker) ---------------------------
 * Link i (1..D) is the segment between the origins of frames i-1 and i,
 * swept by a sphere of radius `radius`; a configuration collides (+1) if any
 * link comes within `radius` of any axis-aligned box, else -1.  Stands in for
 * the geometric checker used to label training data (Sec. III-B active
 * learning, Sec. IV).  boxes: host double nb x 6 (lo xyz, hi xyz), nb <= 64.
 * q: device float n x D.  y: device int8 [n].  The labels are those of an
 * FP64 evaluation: pairs are first decided in FP32 when their distance is
 * more than 1e-5 m from the radius, and a configuration with a pair closer
 * than that to the radius (and no clear hit) is evaluated again in FP64. */
int fk_label(const fk_chain_t *chain, const double *boxes, int64_t nb, double radius, const float *q, int64_t n,
             int8_t *y, void *stream);

/* Sets how many times a kernel polls a shared-memory barrier (a tile, a
 * tensor-core completion, a cluster exchange) before it gives up, raises
 * FK_ERR_TIMEOUT and exits cleanly (default 4194304 polls,
 * about a quarter of a second).  0 makes every such wait give up at once,
 * which exercises the timeout path without a hang.  Process-wide; not
 * synchronised with calls in flight on other threads. */
void fk_set_wait_limit(uint32_t polls);

/* Gaussian summand (FK_SUMMAND_GAUSS, not the paper's kernel) on chains with
 * 7 configuration-dependent control points: how many of the 7 summands of
 * each support point fk_score's FP32 kernel evaluates with an FMA polynomial
 * for 2^(-t) instead of the MUFU ex2 unit (0, the default, 1 or 2), to move
 * work from the MUFU pipe to the FP32 pipe.  Other shapes ignore it.  The
 * polynomial's relative error is about 2.3e-7, inside the band of the FP64
 * re-score, so labels do not depend on it.  Process-wide.  FK_ERR_ARG outside
 * 0..2. */
int fk_set_gauss_poly(int points);

/* ---- many scenes in one launch -----------------------------------------
 * A batch groups trained models (one per scene, each with its own chain,
 * support set and kernel width; all with the same DOF and number of
 * configuration-dependent control points).  fk_score_batched scores every
 * scene's queries in one persistent launch: work items (scene, block of
 * queries) sorted by cost |S| x queries, longest first, handed out by an
 * atomic counter; then the band queries of all scenes are evaluated again
 * in double-float (one warp per query) and those still within 1e-9 B(q) of
 * zero in FP64, band sizes kept on the device.  The launches are captured
 * once in a CUDA graph and replayed while q, f, label,
 * rescore, q_off and the tuned variant stay the same.  When every scene
 * qualifies for the circle form of fk_score_circle (7 or 11 points), each
 * scene is scored in it with its own cnorm; otherwise every scene takes the
 * direct form.  That choice follows fk_set_circle_form when the work list is
 * built (a change of q_off rebuilds it).  The models must stay
 * alive and unchanged while the batch exists (recreate it after retraining).
 * The paper's evaluation scores one scene at a time; this is the multi-scene
 * form of Sec. III-B's check. */
typedef struct fk_batch fk_batch_t;
int fk_batch_create(fastron_model_t *const *models, int n_scenes, fk_batch_t **out);
void fk_batch_destroy(fk_batch_t *batch);

/* q: device float, all scenes' queries concatenated, scene i at rows
 * q_off[i] .. q_off[i+1]-1 (q_off: host int64 [n_scenes + 1], q_off[0] = 0).
 * label (device int8 [total]) and f (device float [total] or NULL) in the same
 * order; rescore and n_rescored as in fk_score.  A change of q_off rebuilds
 * the work list (the device is synchronised, then the list is uploaded). */
int fk_score_batched(fk_batch_t *batch, const float *q, const int64_t *q_off, int rescore, float *f, int8_t *label,
                     int64_t *n_rescored, void *stream);

/* Autotuner: times every compiled tile variant (queries per thread, support
 * pairs per shared-memory tile, threads per CTA) on this batch and keeps the
 * fastest for later calls.  ms (host, may be NULL) receives up to cap times;
 * best (host, may be NULL) the chosen variant.  Synchronous. */
int fk_batch_tune(fk_batch_t *batch, const float *q, const int64_t *q_off, int8_t *label, float *ms, int cap,
                  int *best);

/* ---- learned surrogate (not part of the paper) -------------------------
 * A 64-256-256-256-1 ReLU MLP that predicts the model value f(q) from
 * features of the control points (position of each control point, sin/cos of
 * the joint values on either side of its frame: 7 per point, at most 9
 * points, zero-padded to 64).  Its layers run on tcgen05 tensor cores with
 * BF16 operands and FP32 accumulation; training is mean-squared error on
 * f / scale with Adam on FP32 master weights.  Inference answers a query with
 * sign(pred) when |pred| > tau and sends every other query to fk_score
 * (FP32 score + FP64 re-score), so those labels are exact. */
typedef struct surrogate surrogate_t;

typedef struct {
    int32_t epochs;   /* passes over the training rows */
    int32_t batch;    /* rows per step, a multiple of 128, <= 65536 */
    float lr;         /* Adam step size (schedule below) */
    float holdout;    /* fraction of the queries held out to calibrate tau, in [0, 1) */
    int32_t reinit;   /* 1: reinitialise the weights first; 0: continue (fine-tune) */
    int32_t schedule; /* FK_LR_STEP: lr, divided by 3 for the last third of the epochs;
                         FK_LR_COSINE: lr * (1 + cos(pi k / K)) / 2 at step k of K */
} surrogate_train_params;

typedef struct {
    int64_t steps, n_train, n_holdout;
    float loss_first, loss_last;  /* mean squared error of the first step / last epoch (units of f / scale) */
    float scale;                  /* root mean square of f over the training rows */
    float tau;                    /* calibrated threshold in units of f: no held-out row with |pred| > tau had a wrong sign */
    float holdout_sign_error;     /* fraction of held-out rows whose sign(pred) differs from the exact score's */
    float holdout_fallback;       /* fraction of held-out rows with |pred| <= tau */
} surrogate_stats;

/* Creates a surrogate for `chain` with He-uniform weights drawn from `seed`. */
int surrogate_create(const fk_chain_t *chain, uint64_t seed, surrogate_t **out);
void surrogate_destroy(surrogate_t *s);

/* Trains on n query configurations q (device float n x D): the targets are
 * the model's FP32 scores of the same queries, computed here; the last
 * `holdout` fraction (rounded to 128 rows) is held out to calibrate tau.
 * The steps run on tcgen05 tensor cores as CUDA graphs of three launches per
 * step (a two-CTA-cluster tile kernel: forward, output unit and both delta
 * products; the weight-gradient products; the reduction and Adam), replayed
 * with the batch, learning rate and Adam count taken from a device counter.
 * stats: host, may be NULL.  Synchronous. */
int surrogate_train(surrogate_t *s, fastron_model_t *model, const float *q, int64_t n,
                    const surrogate_train_params *p, surrogate_stats *stats, void *stream);

/* Labels n queries (device float n x D) into label (device int8 [n]).  pred
 * (device float [n] or NULL) receives the surrogate's prediction of f, or the
 * exact f for fallback queries.  tau <= 0 uses the calibrated threshold.
 * n_fallback (host, may be NULL) receives the number of fallback queries.
 * Synchronises `stream` once (to size the fallback pass). */
int surrogate_infer(surrogate_t *s, fastron_model_t *model, const float *q, int64_t n, double tau, int8_t *label,
                    float *pred, int64_t *n_fallback, void *stream);

/* Raw network outputs (units of f / scale) for n queries: out device float [n]. */
int surrogate_forward(surrogate_t *s, const float *q, int64_t n, float *out, void *stream);

/* Parameters as one FP32 vector of 148,481 values: W1 [256][64], b1 [256],
 * W2 [256][256], b2, W3 [256][256], b3, w4 [256], b4.  get also returns the
 * target scale and tau (each may be NULL).  Synchronous. */
int surrogate_set_params(surrogate_t *s, const float *params, int64_t count);
int surrogate_get_params(const surrogate_t *s, float *params, int64_t count, float *scale, float *tau);

/* One forward and backward pass on n queries (device float n x D, n a
 * multiple of 128) against targets (device float [n], units of f / scale):
 * the gradient of the mean squared error (host float [148481]) and the loss
 * (host, may be NULL).  Synchronous. */
int surrogate_gradients(surrogate_t *s, const float *q, int64_t n, const float *target, float *grad, float *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the given gradient
 * (host float [148481]).  Synchronous. */
int surrogate_adam_step(surrogate_t *s, const float *grad, float lr);

/* ---- tensor-core GEMM ---------------------------------------------------
 * C_z = A B^T over the z-th of `splits` equal K ranges, on tcgen05 tensor
 * cores: A device bf16 M x K (row stride lda elements), B device bf16 N x K
 * (row stride ldb), C device float splits x M x N.  M % 128 == 0, N % 64 ==
 * 0, K % (64 splits) == 0, lda, ldb >= K and multiples of 8, pointers 16-byte
 * aligned.  A plain library GEMM on the tensor cores, exposed for testing
 * (the surrogate's training step and inference run fused kernels of their
 * own).  Synchronous (checks the kernel's timeout flag). */
int fk_tc_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int M, int N, int K, int splits,
                    float *C, void *stream);

/* ---- pipe throughput probes --------------------------------------------
 * Measures sustained per-SM throughput of one instruction class with a
 * register-only loop on all SMs: kind 0 FP32 FMA, 1 packed FP32x2 FMA,
 * 2 FP32 reciprocal (MUFU), 3 packed FP16x2 FMA, 4 FP64 FMA, 5 FP16x2 ex2
 * (MUFU); mixed streams with equal numbers of instructions: 6 FP32x2 FMA +
 * FP32 FMA, 7 FP32x2 FMA + FP16x2 FMA, 8 FP32 FMA + FP16x2 FMA, 9 FP32x2 FMA
 * + twice as many FP32 FMA.  *ops_per_clk_sm (host) receives lane-operations per SM clock,
 * from clock64() deltas; *seconds the kernel's wall time.  Synchronous. */
int fk_probe_pipe(int kind, double *ops_per_clk_sm, double *seconds);

#ifdef __cplusplus
}
#endif

#endif /* FKFAST_H */
