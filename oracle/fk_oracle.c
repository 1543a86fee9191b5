/*
 * FP64 CPU oracle for the forward-kinematics (FK) kernel and the Fastron
 * proxy collision checker (Das and Yip, "Forward Kinematics Kernel for
 * Improved Proxy Collision Checking", arXiv 1910.06451).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the CUDA library computes.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Everything is FP64.  Inputs are the canonical FP32 values widened to FP64.
 * Compiled with -ffp-contract=off so that x86 and Arm builds round alike.
 *
 * Layouts (all row-major, caller-owned):
 *   dh      D rows of (a, alpha, d, theta0, type), type 0 revolute, 1 prismatic
 *   base    4x4 world-from-frame-0 transform
 *   q       n rows of D joint values
 *   cp      n x M x 3 control-point positions
 *   boxes   nb rows of (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z)
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- FK ---- */

/* C = A * B for row-major 4x4 matrices. */
static void mat4_mul(const double *A, const double *B, double *C)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k)
                s += A[4 * r + k] * B[4 * k + c];
            C[4 * r + c] = s;
        }
}

/* The standard DH link transform of Eq. 1 for one joint with joint value q.
 * A revolute joint adds q to theta, a prismatic joint adds q to d. */
static void dh_link(const double *row, double q, double *A)
{
    double a = row[0], alpha = row[1], d = row[2], theta = row[3];
    if ((int)row[4] == 0)
        theta += q;
    else
        d += q;
    double ct = cos(theta), st = sin(theta), ca = cos(alpha), sa = sin(alpha);
    double M[16] = {
        ct, -ca * st,  sa * st, a * ct,
        st,  ca * ct, -sa * ct, a * st,
        0.0,      sa,       ca,      d,
        0.0,     0.0,      0.0,    1.0,
    };
    memcpy(A, M, sizeof M);
}

/* Frame poses of one configuration (Sec. II-A): T[0] = wA0 (the base) and
 * T[i] = wA0 0A1 ... (i-1)Ai for i = 1..D.  T holds (D+1) 4x4 matrices. */
void orc_frames(int D, const double *dh, const double *base, const double *q, double *T)
{
    memcpy(T, base, 16 * sizeof(double));
    for (int i = 1; i <= D; ++i) {
        double A[16];
        dh_link(dh + 5 * (i - 1), q[i - 1], A);
        mat4_mul(T + 16 * (i - 1), A, T + 16 * i);
    }
}

/* Control-point positions, Eq. 2: FK_m(x) = pos(wA_{j_m} T_m) with T_m the
 * translation by cp_off[m].  Returns 0, or -1 if a joint index is invalid. */
int orc_fk_points(int D, const double *dh, const double *base, int M, const int32_t *cp_joint,
                  const double *cp_off, int64_t n, const double *q, double *cp)
{
    for (int m = 0; m < M; ++m)
        if (cp_joint[m] < 0 || cp_joint[m] > D)
            return -1;
    double *T = (double *)malloc(sizeof(double) * 16 * (size_t)(D + 1));
    if (!T)
        return -2;
    for (int64_t k = 0; k < n; ++k) {
        orc_frames(D, dh, base, q + k * D, T);
        for (int m = 0; m < M; ++m) {
            const double *W = T + 16 * cp_joint[m];
            const double *t = cp_off + 3 * m;
            for (int c = 0; c < 3; ++c)
                cp[(k * M + m) * 3 + c] = W[4 * c + 0] * t[0] + W[4 * c + 1] * t[1] + W[4 * c + 2] * t[2] + W[4 * c + 3];
        }
    }
    free(T);
    return 0;
}

/* ------------------------------------------------------------ kernels --- */

/* Second-order rational quadratic kernel, Eq. 3, between two dim-vectors:
 * (1 + gamma/2 * |x - x'|^2)^-2, evaluated as 1 / (t * t). */
double orc_k_rq(int dim, const double *x, const double *xp, double gamma)
{
    double d2 = 0.0;
    for (int c = 0; c < dim; ++c) {
        double dc = x[c] - xp[c];
        d2 += dc * dc;
    }
    double t = 1.0 + 0.5 * gamma * d2;
    return 1.0 / (t * t);
}

/* Gaussian summand exp(-gamma/2 * |x - x'|^2) between two dim-vectors.  NOT
 * the paper's kernel: the paper builds the FK kernel from the RQ kernel of
 * Eq. 3 only.  It is the library's optional alternative summand (the same
 * mean over control points as Eq. 4, exp in place of the RQ term). */
double orc_k_gauss(int dim, const double *x, const double *xp, double gamma)
{
    double d2 = 0.0;
    for (int c = 0; c < dim; ++c) {
        double dc = x[c] - xp[c];
        d2 += dc * dc;
    }
    return exp(-0.5 * gamma * d2);
}

/* The summand of kind `kind`: 0 the RQ kernel of Eq. 3 (the paper's), 1 the
 * Gaussian above. */
static double summand(int kind, const double *x, const double *xp, double gamma)
{
    return kind == 1 ? orc_k_gauss(3, x, xp, gamma) : orc_k_rq(3, x, xp, gamma);
}

/* FK kernel, Eq. 4, with summand `kind`: the mean over the M corresponding
 * control points, summed in ascending m.  cpa, cpb: M x 3 each. */
double orc_k_fk_s(int M, const double *cpa, const double *cpb, double gamma, int kind)
{
    double s = 0.0;
    for (int m = 0; m < M; ++m)
        s += summand(kind, cpa + 3 * m, cpb + 3 * m, gamma);
    return s / M;
}

/* FK kernel, Eq. 4, with the paper's RQ summand. */
double orc_k_fk(int M, const double *cpa, const double *cpb, double gamma)
{
    return orc_k_fk_s(M, cpa, cpb, gamma, 0);
}

/* Kernel matrix K[i][j] = K_FK(a_i, b_j) (Sec. II-B), na x nb, summand kind. */
void orc_gram_s(int M, double gamma, int64_t na, const double *cpa, int64_t nb, const double *cpb, double *K,
                int kind)
{
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j)
            K[i * nb + j] = orc_k_fk_s(M, cpa + i * M * 3, cpb + j * M * 3, gamma, kind);
}

void orc_gram(int M, double gamma, int64_t na, const double *cpa, int64_t nb, const double *cpb, double *K)
{
    orc_gram_s(M, gamma, na, cpa, nb, cpb, K, 0);
}

/* ------------------------------------------------------------- score ---- */

typedef struct {
    int M, kind;
    double gamma;
    int64_t ns;
    const double *cps, *alpha;
    const double *cpq;
    double *f;
    int64_t lo, hi;
} score_job;

static void *score_range(void *arg)
{
    score_job *j = (score_job *)arg;
    for (int64_t k = j->lo; k < j->hi; ++k) {
        double f = 0.0;
        for (int64_t s = 0; s < j->ns; ++s)
            f += j->alpha[s] * orc_k_fk_s(j->M, j->cps + s * j->M * 3, j->cpq + k * j->M * 3, j->gamma, j->kind);
        j->f[k] = f;
    }
    return NULL;
}

/* Fastron model value (Sec. III-B): f(x) = sum_s alpha_s K_FK(S_s, x), the
 * support points taken in ascending order.  Queries are split into nthreads
 * contiguous blocks; each query is summed by one thread, so the result does
 * not depend on nthreads. */
int orc_score_s(int M, double gamma, int64_t ns, const double *cps, const double *alpha, int64_t nq,
                const double *cpq, double *f, int nthreads, int kind)
{
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    pthread_t th[256];
    score_job jobs[256];
    int64_t per = (nq + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        score_job j = {M, kind, gamma, ns, cps, alpha, cpq, f, t * per, (t + 1) * per};
        if (j.hi > nq)
            j.hi = nq;
        if (j.lo >= j.hi)
            break;
        jobs[t] = j;
        if (t == 0)
            continue;
        if (pthread_create(&th[t], NULL, score_range, &jobs[t]) != 0) {
            for (int u = 1; u <= started; ++u)
                pthread_join(th[u], NULL);
            return -1;
        }
        started = t;
    }
    if (nq > 0)
        score_range(&jobs[0]);
    for (int t = 1; t <= started; ++t)
        pthread_join(th[t], NULL);
    return 0;
}

int orc_score(int M, double gamma, int64_t ns, const double *cps, const double *alpha, int64_t nq,
              const double *cpq, double *f, int nthreads)
{
    return orc_score_s(M, gamma, ns, cps, alpha, nq, cpq, f, nthreads, 0);
}

/* ----------------------------------------------------------- Fastron ---- */

/* Column i of the kernel matrix over the training set (computeKernelMatrixColumn).
 * store32 != 0: every entry is rounded to the nearest FP32 value, the kernel
 * matrix as it is held when it is stored in single precision (65,536
 * training points take 17.2 GB in FP32); the margins and weights stay FP64.
 *
 * The entries of a column are independent, so a column may be split over
 * threads: each entry is the same orc_k_fk_s call whichever thread makes it,
 * and the column, hence Algorithm 1, does not depend on the thread count.
 * The workers of one training call wait on a condition variable for each
 * column (a generation counter) and report back on another. */
typedef struct {
    int M, store32, kind, nthreads, stop;
    double gamma;
    int64_t N, i;
    const double *cpX;
    double *col;
    pthread_mutex_t mu;
    pthread_cond_t go, fin;
    int64_t gen;   /* column generation: a worker computes its range once per value */
    int pending;   /* workers still computing the current column */
} col_pool;

typedef struct {
    col_pool *p;
    int rank;
} col_worker_arg;

static void column_range(const col_pool *p, int rank)
{
    int64_t per = (p->N + p->nthreads - 1) / p->nthreads;
    int64_t lo = rank * per, hi = lo + per < p->N ? lo + per : p->N;
    for (int64_t j = lo; j < hi; ++j) {
        double k = orc_k_fk_s(p->M, p->cpX + j * p->M * 3, p->cpX + p->i * p->M * 3, p->gamma, p->kind);
        p->col[j] = p->store32 ? (double)(float)k : k;
    }
}

static void *column_worker(void *arg)
{
    col_worker_arg *a = (col_worker_arg *)arg;
    col_pool *p = a->p;
    int64_t seen = 0;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        while (!p->stop && p->gen == seen)
            pthread_cond_wait(&p->go, &p->mu);
        if (p->stop) {
            pthread_mutex_unlock(&p->mu);
            break;
        }
        seen = p->gen;
        pthread_mutex_unlock(&p->mu);
        column_range(p, a->rank);
        pthread_mutex_lock(&p->mu);
        if (--p->pending == 0)
            pthread_cond_signal(&p->fin);
        pthread_mutex_unlock(&p->mu);
    }
    return NULL;
}

static void kernel_column(col_pool *p, int64_t i)
{
    if (p->nthreads > 1) {
        pthread_mutex_lock(&p->mu);
        p->i = i;
        p->pending = p->nthreads - 1;
        ++p->gen;
        pthread_cond_broadcast(&p->go);
        pthread_mutex_unlock(&p->mu);
    } else {
        p->i = i;
    }
    column_range(p, 0);
    if (p->nthreads > 1) {
        pthread_mutex_lock(&p->mu);
        while (p->pending > 0)
            pthread_cond_wait(&p->fin, &p->mu);
        pthread_mutex_unlock(&p->mu);
    }
}

/* Stops and joins the first n - 1 workers. */
static void pool_stop(col_pool *p, pthread_t *th, int n)
{
    pthread_mutex_lock(&p->mu);
    p->stop = 1;
    pthread_cond_broadcast(&p->go);
    pthread_mutex_unlock(&p->mu);
    for (int t = 1; t < n; ++t)
        pthread_join(th[t], NULL);
}

/*
 * Fastron model update, Algorithm 1 (Sec. III-B), taken step by step:
 *
 *   for iter = 1..iter_max:
 *     if min_j y_j F_j <= 0:                               (misclassified point)
 *       i = argmin_j y_j F_j
 *       if count(alpha != 0) < s_max or alpha_i != 0:      (add / adjust, Eqs. 6-8)
 *         delta = b_i y_i - F_i,  b_i = beta^(0.5 (y_i + 1))
 *         alpha_i += delta;  F += delta K e_i;  continue
 *     if max_{alpha_j != 0} y_j (F_j - alpha_j) > 0:       (redundant support point)
 *       i = that argmax;  F -= alpha_i K e_i;  alpha_i = 0;  continue
 *     break
 *
 * Readings where the paper is silent: argmin/argmax ties go to the lowest
 * index; "continue" after an add means a removal is tried only when no add
 * was made in that pass; each pass is one iteration; the margin update
 * F_j + delta K_ji (Eq. 8) is one fused multiply-add, rounded once (C99 fma).
 *
 * alpha and F are in/out (zeros for a cold start, a previous model's values
 * for a warm start, loadPreviousModel).  stats = {iterations, adds, removals,
 * converged (1 if the loop ended by break), support size}.  If trace_kind is
 * not NULL, pass k records kind (1 add, 2 removal), index and delta (the
 * change of alpha_i) in trace_kind/trace_idx/trace_delta[k].  store32: see
 * kernel_column.  kind: the summand of the FK kernel, 0 the paper's RQ
 * kernel (Eq. 3), 1 the Gaussian alternative (orc_k_gauss).  nthreads: the
 * threads that share each column's entries (the passes themselves stay
 * sequential); the result is the same for every nthreads.
 */
int orc_fastron_train_mt(int M, double gamma, int64_t N, const double *cpX, const int8_t *y, double beta,
                         int64_t iter_max, int64_t s_max, double *alpha, double *F, int64_t *stats,
                         int8_t *trace_kind, int64_t *trace_idx, double *trace_delta, int store32, int kind,
                         int nthreads)
{
    double *col = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!col)
        return -2;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    col_pool pool;
    memset(&pool, 0, sizeof pool);
    pool.M = M;
    pool.store32 = store32;
    pool.kind = kind;
    pool.gamma = gamma;
    pool.N = N;
    pool.cpX = cpX;
    pool.col = col;
    pool.nthreads = 1;
    pthread_mutex_init(&pool.mu, NULL);
    pthread_cond_init(&pool.go, NULL);
    pthread_cond_init(&pool.fin, NULL);
    pthread_t th[256];
    col_worker_arg wa[256];
    int started = 1;
    for (int t = 1; t < nthreads; ++t) {
        wa[t].p = &pool;
        wa[t].rank = t;
        if (pthread_create(&th[t], NULL, column_worker, &wa[t]) != 0)
            break;
        started = t + 1;
    }
    /* workers read nthreads only once a column is posted, under the mutex */
    pthread_mutex_lock(&pool.mu);
    pool.nthreads = started;
    pthread_mutex_unlock(&pool.mu);
    int64_t nnz = 0, adds = 0, removes = 0, iters = 0;
    int converged = 0;
    for (int64_t j = 0; j < N; ++j)
        nnz += alpha[j] != 0.0;

    for (int64_t iter = 1; iter <= iter_max; ++iter) {
        /* check for misclassifications */
        int64_t i = -1;
        double mmin = INFINITY;
        for (int64_t j = 0; j < N; ++j) {
            double m = y[j] * F[j];
            if (m < mmin) {
                mmin = m;
                i = j;
            }
        }
        if (i >= 0 && mmin <= 0.0) {
            kernel_column(&pool, i);
            if (nnz < s_max || alpha[i] != 0.0) {
                double b = y[i] > 0 ? beta : 1.0;
                double delta = b * y[i] - F[i];
                int was_zero = alpha[i] == 0.0;
                alpha[i] += delta;
                for (int64_t j = 0; j < N; ++j)
                    F[j] = fma(delta, col[j], F[j]);
                nnz += (alpha[i] != 0.0) - !was_zero;
                ++adds;
                ++iters;
                if (trace_kind) {
                    trace_kind[iter - 1] = 1;
                    trace_idx[iter - 1] = i;
                    trace_delta[iter - 1] = delta;
                }
                continue;
            }
        }
        /* remove redundant support points */
        int64_t r = -1;
        double mmax = -INFINITY;
        for (int64_t j = 0; j < N; ++j) {
            if (alpha[j] == 0.0)
                continue;
            double m = y[j] * (F[j] - alpha[j]);
            if (m > mmax) {
                mmax = m;
                r = j;
            }
        }
        if (r >= 0 && mmax > 0.0) {
            kernel_column(&pool, r);
            double a = alpha[r];
            for (int64_t j = 0; j < N; ++j)
                F[j] = fma(-a, col[j], F[j]);
            alpha[r] = 0.0;
            --nnz;
            ++removes;
            ++iters;
            if (trace_kind) {
                trace_kind[iter - 1] = 2;
                trace_idx[iter - 1] = r;
                trace_delta[iter - 1] = -a;
            }
            continue;
        }
        converged = 1;
        break;
    }
    pool_stop(&pool, th, started);
    pthread_mutex_destroy(&pool.mu);
    pthread_cond_destroy(&pool.go);
    pthread_cond_destroy(&pool.fin);
    free(col);
    stats[0] = iters;
    stats[1] = adds;
    stats[2] = removes;
    stats[3] = converged;
    stats[4] = nnz;
    return 0;
}

int orc_fastron_train_kind(int M, double gamma, int64_t N, const double *cpX, const int8_t *y, double beta,
                           int64_t iter_max, int64_t s_max, double *alpha, double *F, int64_t *stats,
                           int8_t *trace_kind, int64_t *trace_idx, double *trace_delta, int store32, int kind)
{
    return orc_fastron_train_mt(M, gamma, N, cpX, y, beta, iter_max, s_max, alpha, F, stats, trace_kind, trace_idx,
                                trace_delta, store32, kind, 1);
}

int orc_fastron_train_store(int M, double gamma, int64_t N, const double *cpX, const int8_t *y, double beta,
                            int64_t iter_max, int64_t s_max, double *alpha, double *F, int64_t *stats,
                            int8_t *trace_kind, int64_t *trace_idx, double *trace_delta, int store32)
{
    return orc_fastron_train_kind(M, gamma, N, cpX, y, beta, iter_max, s_max, alpha, F, stats, trace_kind,
                                  trace_idx, trace_delta, store32, 0);
}

int orc_fastron_train(int M, double gamma, int64_t N, const double *cpX, const int8_t *y, double beta,
                      int64_t iter_max, int64_t s_max, double *alpha, double *F, int64_t *stats,
                      int8_t *trace_kind, int64_t *trace_idx, double *trace_delta)
{
    return orc_fastron_train_store(M, gamma, N, cpX, y, beta, iter_max, s_max, alpha, F, stats, trace_kind,
                                   trace_idx, trace_delta, 0);
}

/*
 * Margins of a carried-over model on a new training set (loadPreviousModel
 * when the training set has changed, Sec. III-B): the first ns training
 * points are the previous support set with weights alpha[0..ns); the rest
 * start at 0, so F_j = sum_{s < ns} alpha_s K(X_s, X_j), summed in ascending
 * s, each step a fused multiply-add as in the update of Eq. 8.  store32: kernel entries
 * rounded to FP32 as in kernel_column.
 */
void orc_margins(int M, double gamma, int64_t N, const double *cpX, int64_t ns, const double *alpha, int store32,
                 double *F)
{
    for (int64_t j = 0; j < N; ++j) {
        double f = 0.0;
        for (int64_t s = 0; s < ns; ++s) {
            double k = orc_k_fk(M, cpX + s * M * 3, cpX + j * M * 3, gamma);
            if (store32)
                k = (double)(float)k;
            f = fma(alpha[s], k, f);
        }
        F[j] = f;
    }
}

/* --------------------------------------------------- geometric checker -- */

/* Squared distance from point p to the box [lo, hi]. */
static double point_box_dist2(const double *p, const double *lo, const double *hi)
{
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
        double e = 0.0;
        if (p[c] < lo[c])
            e = lo[c] - p[c];
        else if (p[c] > hi[c])
            e = p[c] - hi[c];
        s += e * e;
    }
    return s;
}

/* Squared distance from the segment p0 -> p1 to the box [lo, hi].
 * g(t) = dist2(p0 + t (p1 - p0), box) is convex and quadratic between the
 * parameters where a coordinate crosses a slab face.  On each piece the
 * quadratic's minimiser is found in closed form, clamped to the piece, and g
 * is evaluated there; the smallest value over the pieces is the distance. */
double orc_seg_box_dist2(const double *p0, const double *p1, const double *lo, const double *hi)
{
    double dp[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double ts[8];
    int nt = 0;
    ts[nt++] = 0.0;
    ts[nt++] = 1.0;
    for (int c = 0; c < 3; ++c) {
        if (dp[c] == 0.0)
            continue;
        double bnd[2] = {lo[c], hi[c]};
        for (int b = 0; b < 2; ++b) {
            double t = (bnd[b] - p0[c]) / dp[c];
            if (t > 0.0 && t < 1.0)
                ts[nt++] = t;
        }
    }
    for (int a = 1; a < nt; ++a)            /* insertion sort */
        for (int b = a; b > 0 && ts[b - 1] > ts[b]; --b) {
            double tmp = ts[b];
            ts[b] = ts[b - 1];
            ts[b - 1] = tmp;
        }
    double best = INFINITY;
    for (int k = 0; k + 1 < nt; ++k) {
        double ta = ts[k], tb = ts[k + 1];
        double tm = 0.5 * (ta + tb);
        double sab = 0.0, sbb = 0.0;
        for (int c = 0; c < 3; ++c) {
            double x = p0[c] + tm * dp[c];
            double bound;
            if (x < lo[c])
                bound = lo[c];
            else if (x > hi[c])
                bound = hi[c];
            else
                continue;
            double A = p0[c] - bound, B = dp[c];
            sab += A * B;
            sbb += B * B;
        }
        double t = ta;
        if (sbb > 0.0) {
            t = -sab / sbb;
            if (t < ta)
                t = ta;
            if (t > tb)
                t = tb;
        }
        double p[3] = {p0[0] + t * dp[0], p0[1] + t * dp[1], p0[2] + t * dp[2]};
        double g = point_box_dist2(p, lo, hi);
        if (g < best)
            best = g;
    }
    double ge0 = point_box_dist2(p0, lo, hi), ge1 = point_box_dist2(p1, lo, hi);
    if (ge0 < best)
        best = ge0;
    if (ge1 < best)
        best = ge1;
    return best;
}

/* Ground-truth labels: link i (i = 1..D) is the segment between the origins of
 * frames i-1 and i, swept by a sphere of the given radius.  A configuration
 * collides (+1) if any link comes within radius of any box (touching counts),
 * else it is free (-1).  Labels follow Sec. II-B: +1 = C_obs, -1 = C_free. */
int orc_check(int D, const double *dh, const double *base, int64_t nb, const double *boxes, double radius,
              int64_t n, const double *q, int8_t *y)
{
    double *T = (double *)malloc(sizeof(double) * 16 * (size_t)(D + 1));
    if (!T)
        return -2;
    double r2 = radius * radius;
    for (int64_t k = 0; k < n; ++k) {
        orc_frames(D, dh, base, q + k * D, T);
        int hit = 0;
        for (int i = 1; i <= D && !hit; ++i) {
            double o0[3] = {T[16 * (i - 1) + 3], T[16 * (i - 1) + 7], T[16 * (i - 1) + 11]};
            double o1[3] = {T[16 * i + 3], T[16 * i + 7], T[16 * i + 11]};
            for (int64_t b = 0; b < nb && !hit; ++b)
                if (orc_seg_box_dist2(o0, o1, boxes + 6 * b, boxes + 6 * b + 3) <= r2)
                    hit = 1;
        }
        y[k] = hit ? 1 : -1;
    }
    free(T);
    return 0;
}
