/*
 * nss_oracle.c -- plain, slow, FP64 CPU oracle of Nested Slice Sampling
 * (Yallup, Kroupa & Handley, "Nested Slice Sampling: Vectorized Nested
 * Sampling for GPU-Accelerated Inference", arxiv 2601.23252).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table
 * or constant generator with the CUDA path.  Every step follows the paper's
 * order and notation, in double precision, with no blocking, fusion or
 * reordering beyond what the paper states.
 *
 * Conventions.  The paper works with an energy E = -log L; this file works
 * in log-likelihood, so "the k highest energies" are "the k lowest logL" and
 * the constraint E(x) < E_batch reads logL(x) > logL*.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), written here from that
 * description.  Counter layout (the method's reading of its random draws):
 *   key     = (seed_lo32, seed_hi32 ^ run_id)
 *   HRSS    : counter (iteration, chain, step, word/4), word layout per step
 *             [0, 2*ceil(d/2))  Box-Muller pairs of the direction z
 *             nz = 2*ceil(d/2)  bracket position U
 *             nz + 1            slice height (non-flat prior only)
 *             nz + 2            reserved
 *             nz + 3 + r        shrinkage proposal r, r = 0..99
 *   parents : counter (iteration, chain, TAG_PARENT, 0), word 0
 *   init    : counter (0, slot, TAG_INIT, word/4)
 *   volumes : counter (trajectory, dead/2, TAG_VOLSIM, 0), words 2*(dead&1)+{0,1}
 *   u24(w)  = (2*(w>>9) + 1) * 2^-24                (exact in FP32 and FP64)
 *   u53(a,b)= (2*(((a>>6)<<26) | (b>>6)) + 1) * 2^-53 (exact in FP64)
 *
 * Parity unpinned: none of the functions below is unpinned; the logistic and
 * GP likelihood values are pinned against library routines, the NS evidence
 * against closed forms and quadrature (see tests/test_oracle_*.py).
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_TAG_PARENT 0xFFFFFFF0u
#define ORC_TAG_INIT   0xFFFFFFF1u
#define ORC_TAG_VOLSIM 0xFFFFFFF2u

#define ORC_STEP_OUT_CAP 10   /* Sec. B.4 "Stepping-out": at most 10 expansions per side */
#define ORC_SHRINK_CAP  100   /* Sec. B.4 "Shrinkage": at most 100 proposals, then null move */

enum { ORC_PRIOR_BOX = 0, ORC_PRIOR_GAUSS = 1 };
enum {
    ORC_LIK_GAUSS = 0,      /* isotropic Gaussian, normalised            */
    ORC_LIK_GMM = 1,        /* equal-weight isotropic mixture, normalised */
    ORC_LIK_LOGREG = 2,     /* Bayesian logistic regression              */
    ORC_LIK_GP = 3,         /* GP marginal likelihood, RBF + white kernel */
    ORC_LIK_FLAT = 4,       /* logL = 0 (plateau / pure prior)          */
    ORC_LIK_RASTRIGIN = 5   /* Gaussian + Rastrigin mixture, App. F.3     */
};

typedef struct {
    int prior_kind;
    int d;
    const double *a;     /* box: lower bounds; Gaussian prior: means       */
    const double *b;     /* box: upper bounds; Gaussian prior: std devs    */
    int lik_kind;
    int n_comp;          /* mixture components                               */
    int n_data;          /* logistic rows N or GP points n                   */
    double sigma;        /* Gaussian / mixture scale                          */
    double alpha;        /* Rastrigin mixture weight                          */
    const double *mu;    /* [n_comp][d]                                       */
    const double *X;     /* logistic design [N][d]                            */
    const double *y;     /* logistic labels in {0,1} [N]; GP targets [n]     */
    const double *t;     /* GP inputs [n]                                     */
} orc_problem;

typedef struct {
    int n_live, k, p;
    double w;            /* slice width in the whitened metric                 */
    int dir_norm;        /* 0: v = Lz/|z| (Mahalanobis unit), 1: v = Lz/|Lz|  */
    double cov_eps;      /* relative diagonal regularisation of the metric     */
    double tol;          /* live-evidence fraction at which the run stops      */
    int max_iter;
    uint64_t seed;
    uint32_t run_id;
    int kernel;          /* 0: HRSS (Sec. 3.2); 1: constrained random walk     */
    double rw_scale;     /* random-walk proposal x + s L z; 0 = 2.38 / sqrt(d) */
} orc_opts;

typedef struct {
    int *dead_idx;       /* [k] slots removed, worst first                      */
    int *parent;         /* [k]                                                  */
    double *L;           /* [d*d] Cholesky factor, row major, lower             */
    double *new_x;       /* [k*d]                                               */
    double *new_logL;    /* [k]                                                 */
    int *evals, *accepts, *nulls, *expansions, *shrinks, *cap_out; /* [k]     */
    double *margin;      /* [k] min |logL(y) - logL*| over likelihood tests     */
    double *pmargin;     /* [k] min |log Pi(y) - height| over prior-height tests */
    double *bmargin;     /* [k] min distance of a proposal to the box boundary  */
    double logLstar;
    double logZ, logX;   /* deterministic running estimates after the step      */
    int done;            /* termination test after the step                     */
} orc_trace;

typedef struct {
    long long n_dead;
    int iters;
    long long evals;
    long long nulls;
    long long cap_out;   /* stepping-out expansions stopped by the cap          */
    double logZ_det;     /* running Delta-X quadrature incl. the final live set */
    double logX;
    int status;          /* 0 ok, 1 max_iter reached, -4 capacity             */
} orc_summary;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 description: 10 rounds of two 32x32->64     */
/* multiplications with the published multipliers, key bumped by the        */
/* published Weyl constants between rounds.                                  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void orc_key(uint64_t seed, uint32_t run_id, uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32) ^ run_id;
}

static uint32_t orc_word(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t w)
{
    uint32_t ctr[4] = {c0, c1, c2, w >> 2}, out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w & 3u];
}

double orc_u24(uint32_t w) { return (2.0 * (double)(w >> 9) + 1.0) * 0x1p-24; }

double orc_u53(uint32_t a, uint32_t b)
{
    uint64_t x = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return (2.0 * (double)x + 1.0) * 0x1p-53;
}

/* d standard normals from words [0, 2*ceil(d/2)) of one counter stream,
   Box-Muller (Box & Muller 1958): r = sqrt(-2 ln u1), angle 2 pi u2. */
static void orc_normals(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2, int d, double *z)
{
    for (int q = 0; 2 * q < d; ++q) {
        double u1 = orc_u24(orc_word(key, c0, c1, c2, 2u * q));
        double u2 = orc_u24(orc_word(key, c0, c1, c2, 2u * q + 1u));
        double r = sqrt(-2.0 * log(u1));
        z[2 * q] = r * cos(2.0 * M_PI * u2);
        if (2 * q + 1 < d) z[2 * q + 1] = r * sin(2.0 * M_PI * u2);
    }
}

/* ------------------------------------------------------------------------ */
/* Prior and likelihood (Eq. eq:target / eq:integral_Z: pi(x) L(x), L=e^-E)  */
/* ------------------------------------------------------------------------ */
static double orc_logaddexp(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}

int orc_in_support(const orc_problem *pb, const double *x)
{
    if (pb->prior_kind != ORC_PRIOR_BOX) return 1;
    for (int i = 0; i < pb->d; ++i)
        if (!(x[i] >= pb->a[i] && x[i] <= pb->b[i])) return 0;
    return 1;
}

/* distance of x to the boundary of the box (negative when outside) */
static double orc_box_margin(const orc_problem *pb, const double *x)
{
    double m = INFINITY;
    if (pb->prior_kind != ORC_PRIOR_BOX) return m;
    for (int i = 0; i < pb->d; ++i) {
        double lo = x[i] - pb->a[i], hi = pb->b[i] - x[i];
        double v = lo < hi ? lo : hi;
        if (fabs(v) < m) m = fabs(v);
    }
    return m;
}

double orc_log_prior(const orc_problem *pb, const double *x)
{
    double s = 0.0;
    if (pb->prior_kind == ORC_PRIOR_BOX) {
        for (int i = 0; i < pb->d; ++i) {
            if (!(x[i] >= pb->a[i] && x[i] <= pb->b[i])) return -INFINITY;
            s -= log(pb->b[i] - pb->a[i]);
        }
        return s;
    }
    for (int i = 0; i < pb->d; ++i) {
        double u = (x[i] - pb->a[i]) / pb->b[i];
        s += -0.5 * u * u - log(pb->b[i]) - 0.5 * log(2.0 * M_PI);
    }
    return s;
}

/* Cholesky A = L L^T in place (lower, row major); returns 0 on success. */
static int orc_cholesky_inplace(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int q = 0; q < j; ++q) s -= A[j * n + q] * A[j * n + q];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int q = 0; q < j; ++q) t -= A[i * n + q] * A[j * n + q];
            A[i * n + j] = t / ljj;
        }
        for (int q = j + 1; q < n; ++q) A[j * n + q] = 0.0;
    }
    return 0;
}

/* GP marginal likelihood with theta = (ln lengthscale, ln amplitude, ln noise):
   K_ij = a^2 exp(-(t_i - t_j)^2 / (2 l^2)) + s^2 delta_ij,
   log p(y) = -1/2 y^T K^-1 y - sum_i ln L_ii - n/2 ln 2 pi   (Sec. 4.4, GP). */
static double orc_gp_loglik(const orc_problem *pb, const double *th)
{
    int n = pb->n_data;
    double ell = exp(th[0]), amp = exp(th[1]), sn = exp(th[2]);
    double *K = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *alpha = (double *)malloc(sizeof(double) * n);
    if (!K || !alpha) { free(K); free(alpha); return NAN; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double dt = pb->t[i] - pb->t[j];
            K[i * n + j] = amp * amp * exp(-dt * dt / (2.0 * ell * ell)) + (i == j ? sn * sn : 0.0);
        }
    double out;
    if (orc_cholesky_inplace(n, K) != 0) {
        out = -INFINITY;
    } else {
        /* forward solve L alpha = y; then y^T K^-1 y = |alpha|^2 */
        double q = 0.0, ld = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = pb->y[i];
            for (int j = 0; j < i; ++j) s -= K[i * n + j] * alpha[j];
            alpha[i] = s / K[i * n + i];
            q += alpha[i] * alpha[i];
            ld += log(K[i * n + i]);
        }
        out = -0.5 * q - ld - 0.5 * n * log(2.0 * M_PI);
    }
    free(K); free(alpha);
    return out;
}

/* log L(x); NaN is read as -inf (a point with undefined likelihood is
   outside every constraint set). */
double orc_loglik(const orc_problem *pb, const double *x)
{
    int d = pb->d;
    double v;
    switch (pb->lik_kind) {
    case ORC_LIK_GAUSS: {
        double q = 0.0;
        for (int i = 0; i < d; ++i) { double e = x[i] - pb->mu[i]; q += e * e; }
        v = -q / (2.0 * pb->sigma * pb->sigma) - 0.5 * d * log(2.0 * M_PI * pb->sigma * pb->sigma);
        break;
    }
    case ORC_LIK_GMM: {
        double acc = -INFINITY;
        for (int c = 0; c < pb->n_comp; ++c) {
            double q = 0.0;
            for (int i = 0; i < d; ++i) { double e = x[i] - pb->mu[c * d + i]; q += e * e; }
            acc = orc_logaddexp(acc, -q / (2.0 * pb->sigma * pb->sigma));
        }
        v = acc - log((double)pb->n_comp) - 0.5 * d * log(2.0 * M_PI * pb->sigma * pb->sigma);
        break;
    }
    case ORC_LIK_LOGREG: {
        /* sum_n [y_n z_n - softplus(z_n)], z = X x  (Bernoulli-logit likelihood) */
        double s = 0.0;
        for (int r = 0; r < pb->n_data; ++r) {
            double z = 0.0;
            for (int i = 0; i < d; ++i) z += pb->X[(size_t)r * d + i] * x[i];
            double sp = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
            s += pb->y[r] * z - sp;
        }
        v = s;
        break;
    }
    case ORC_LIK_GP:
        v = orc_gp_loglik(pb, x);
        break;
    case ORC_LIK_FLAT:
        v = 0.0;
        break;
    case ORC_LIK_RASTRIGIN: {
        /* L = alpha f + (1-alpha) g, f = exp(-|x|^2/2),
           g = exp(-A d + A sum cos(2 pi x_i)), A = 10  (App. F.3) */
        double q = 0.0, c = 0.0;
        for (int i = 0; i < d; ++i) { q += x[i] * x[i]; c += cos(2.0 * M_PI * x[i]); }
        double lf = -0.5 * q, lg = -10.0 * d + 10.0 * c;
        double a = pb->alpha;
        double t1 = a > 0.0 ? log(a) + lf : -INFINITY;
        double t2 = a < 1.0 ? log1p(-a) + lg : -INFINITY;
        v = orc_logaddexp(t1, t2);
        break;
    }
    default:
        v = NAN;
    }
    if (isnan(v)) v = -INFINITY;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Initial live set: m independent prior draws (Sec. 2.1).                   */
/* ------------------------------------------------------------------------ */
void orc_prior_draw(const orc_problem *pb, uint64_t seed, uint32_t run_id, uint32_t slot, double *x)
{
    uint32_t key[2];
    orc_key(seed, run_id, key);
    int d = pb->d;
    if (pb->prior_kind == ORC_PRIOR_BOX) {
        for (int i = 0; i < d; ++i)
            x[i] = pb->a[i] + (pb->b[i] - pb->a[i]) * orc_u24(orc_word(key, 0u, slot, ORC_TAG_INIT, (uint32_t)i));
    } else {
        orc_normals(key, 0u, slot, ORC_TAG_INIT, d, x);
        for (int i = 0; i < d; ++i) x[i] = pb->a[i] + pb->b[i] * x[i];
    }
}

/* ------------------------------------------------------------------------ */
/* (i) Reweight/delete: order live points by (logL, slot) ascending; the     */
/* first k are dead, logL* is the k-th (Sec. 3.1 (i); Algorithm 1).  The     */
/* survivors are listed in ascending slot order.                             */
/* ------------------------------------------------------------------------ */
static const double *g_sort_logL;
static int orc_cmp_slot(const void *pa, const void *pb)
{
    int i = *(const int *)pa, j = *(const int *)pb;
    double a = g_sort_logL[i], b = g_sort_logL[j];
    if (a < b) return -1;
    if (a > b) return 1;
    return (i > j) - (i < j);
}

void orc_select(int m, int k, const double *logL, int *dead, int *surv, double *logLstar)
{
    int *order = (int *)malloc(sizeof(int) * m);
    char *is_dead = (char *)calloc(m, 1);
    for (int i = 0; i < m; ++i) order[i] = i;
    g_sort_logL = logL;
    qsort(order, m, sizeof(int), orc_cmp_slot);
    for (int j = 0; j < k; ++j) { dead[j] = order[j]; is_dead[order[j]] = 1; }
    *logLstar = logL[order[k - 1]];
    int s = 0;
    for (int i = 0; i < m; ++i) if (!is_dead[i]) surv[s++] = i;
    free(order); free(is_dead);
}

/* ------------------------------------------------------------------------ */
/* Evidence bookkeeping, one unrolled death with n live points:               */
/* X_j = X_{j-1} e^{-1/n} (E[log t] = -1/n, Eq. eq:dlnX; App. D.1),          */
/* Z += L_j (X_{j-1} - X_j)  (Eq. eq:marginal).                              */
/* ------------------------------------------------------------------------ */
void orc_evidence_death(double logL, int n, double *logZ, double *logX)
{
    double logX_prev = *logX;
    *logX = logX_prev - 1.0 / n;
    double log_dX = logX_prev + log(-expm1(-1.0 / n));
    *logZ = orc_logaddexp(*logZ, logL + log_dX);
}

/* Remaining live contribution Z_live = X mean(L_live); the run stops when
   Z_live / (Z + Z_live) < tol (Sec. B.3 termination, reading: live fraction). */
int orc_should_stop(int m, const double *logL, double logZ, double logX, double tol)
{
    double mx = -INFINITY;
    for (int i = 0; i < m; ++i) if (logL[i] > mx) mx = logL[i];
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += exp(logL[i] - mx);
    double logZ_live = logX + mx + log(s) - log((double)m);
    if (mx == -INFINITY) logZ_live = -INFINITY;
    double tot = orc_logaddexp(logZ, logZ_live);
    return (logZ_live - tot) < log(tol);
}

/* ------------------------------------------------------------------------ */
/* Direction metric (Sec. 3.2 "Direction metric"): M^-1 = empirical          */
/* covariance of the current live set (divisor m-1) plus a relative          */
/* diagonal regularisation eps * tr(Sigma)/d; L = chol(M^-1).  A failed      */
/* factorisation retries with 10x the jitter (up to 6 times); a degenerate   */
/* live set (zero or non-finite trace) falls back to the identity.           */
/* ------------------------------------------------------------------------ */
int orc_covariance(int m, int d, const double *X, double *Sigma)
{
    double *mu = (double *)calloc(d, sizeof(double));
    for (int i = 0; i < m; ++i)
        for (int a = 0; a < d; ++a) mu[a] += X[(size_t)i * d + a];
    for (int a = 0; a < d; ++a) mu[a] /= m;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int i = 0; i < m; ++i)
                s += (X[(size_t)i * d + a] - mu[a]) * (X[(size_t)i * d + b] - mu[b]);
            Sigma[a * d + b] = s / (m - 1);
        }
    free(mu);
    return 0;
}

int orc_metric(int m, int d, const double *X, double eps, double *L)
{
    double *S = (double *)malloc(sizeof(double) * d * d);
    orc_covariance(m, d, X, S);
    double tr = 0.0;
    for (int a = 0; a < d; ++a) tr += S[a * d + a];
    int status = 0;
    if (!(tr > 0.0) || !isfinite(tr)) {
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) L[a * d + b] = (a == b) ? 1.0 : 0.0;
        free(S);
        return 1;
    }
    double reg = eps * tr / d;
    for (int attempt = 0; attempt <= 6; ++attempt) {
        memcpy(L, S, sizeof(double) * d * d);
        for (int a = 0; a < d; ++a) L[a * d + a] += reg;
        if (orc_cholesky_inplace(d, L) == 0) { free(S); return status; }
        reg *= 10.0;
        status = 2;
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) L[a * d + b] = (a == b) ? 1.0 : 0.0;
    free(S);
    return 3;
}

/* ------------------------------------------------------------------------ */
/* (ii) Resample: k parents uniformly with replacement from the m-k          */
/* survivors (multinomial with binary weights, Sec. 3.1 (ii)).               */
/* ------------------------------------------------------------------------ */
void orc_parents(uint64_t seed, uint32_t run_id, uint32_t iter, int m, int k, const int *surv, int *parent)
{
    uint32_t key[2];
    orc_key(seed, run_id, key);
    for (int j = 0; j < k; ++j) {
        uint32_t w = orc_word(key, iter, (uint32_t)j, ORC_TAG_PARENT, 0u);
        uint64_t idx = ((uint64_t)w * (uint64_t)(m - k)) >> 32;
        parent[j] = surv[idx];
    }
}

/* ------------------------------------------------------------------------ */
/* (iii) Mutate: one Hit-and-Run Slice Sampling step (Sec. 3.2; App. B.4).   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int evals, accepts, nulls, expansions, shrinks, cap_out;
    double margin, pmargin, bmargin;
} orc_counts;

typedef struct {
    const orc_problem *pb;
    double logLstar;
    int nonflat;
    double height;       /* log Pi threshold for a non-flat prior */
    orc_counts *cnt;
    double *y;           /* scratch [d] */
} orc_slice;

/* y is in the slice when it is in the prior support, above the prior
   slice height (non-flat prior, App. B.4 "given a slice height") and
   strictly above the likelihood threshold (Sec. 3.1: E < E_batch).  Every
   call is one logical likelihood evaluation. */
static int orc_in_slice(orc_slice *sl, const double *y, double *logLy)
{
    const orc_problem *pb = sl->pb;
    sl->cnt->evals++;
    double bm = orc_box_margin(pb, y);
    if (bm < sl->cnt->bmargin) sl->cnt->bmargin = bm;
    if (!orc_in_support(pb, y)) return 0;
    if (sl->nonflat) {
        double lp = orc_log_prior(pb, y);
        double pm = fabs(lp - sl->height);
        if (pm < sl->cnt->pmargin) sl->cnt->pmargin = pm;
        if (!(lp > sl->height)) return 0;
    }
    double ll = orc_loglik(pb, y);
    double mg = fabs(ll - sl->logLstar);
    if (mg < sl->cnt->margin) sl->cnt->margin = mg;
    *logLy = ll;
    return ll > sl->logLstar;
}

static void orc_line(int d, const double *x, double t, const double *v, double *y)
{
    for (int i = 0; i < d; ++i) y[i] = x[i] + t * v[i];
}

void orc_hrss_step(const orc_problem *pb, const double *L, double w, int dir_norm, double logLstar,
                   uint64_t seed, uint32_t run_id, uint32_t iter, uint32_t chain, uint32_t step,
                   double *x, double *logLx, orc_counts *cnt)
{
    int d = pb->d;
    uint32_t key[2];
    orc_key(seed, run_id, key);
    uint32_t nz = 2u * (uint32_t)((d + 1) / 2);
    double *z = (double *)malloc(sizeof(double) * d);
    double *v = (double *)malloc(sizeof(double) * d);
    double *y = (double *)malloc(sizeof(double) * d);

    /* random direction d~ = L z, z ~ N(0, I)  (Sec. 3.2 "Direction metric") */
    orc_normals(key, iter, chain, step, d, z);
    double zz = 0.0, dd = 0.0;
    for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int b = 0; b <= a; ++b) s += L[a * d + b] * z[b];
        v[a] = s;
        zz += z[a] * z[a];
        dd += s * s;
    }
    double nrm = dir_norm == 0 ? sqrt(zz) : sqrt(dd);
    for (int a = 0; a < d; ++a) v[a] /= nrm;

    orc_slice sl;
    sl.pb = pb; sl.logLstar = logLstar; sl.cnt = cnt; sl.y = y;
    sl.nonflat = pb->prior_kind != ORC_PRIOR_BOX;
    sl.height = 0.0;
    if (sl.nonflat) {
        /* slice height under the prior: log Pi(x) - e, e ~ Exp(1) */
        double uh = orc_u24(orc_word(key, iter, chain, step, nz + 1u));
        sl.height = orc_log_prior(pb, x) + log(uh);
    }

    /* randomised initial bracket of width w around t = 0 (App. B.4) */
    double U = orc_u24(orc_word(key, iter, chain, step, nz));
    double tl = -w * U;
    double tr = tl + w;
    double ll_dummy;
    int n = 0;
    for (;;) {
        if (n >= ORC_STEP_OUT_CAP) { cnt->cap_out++; break; }
        orc_line(d, x, tl, v, y);
        if (!orc_in_slice(&sl, y, &ll_dummy)) break;
        tl -= w; n++; cnt->expansions++;
    }
    n = 0;
    for (;;) {
        if (n >= ORC_STEP_OUT_CAP) { cnt->cap_out++; break; }
        orc_line(d, x, tr, v, y);
        if (!orc_in_slice(&sl, y, &ll_dummy)) break;
        tr += w; n++; cnt->expansions++;
    }

    /* shrinkage: uniform proposal in [tl, tr]; accept if in the slice, else
       the bracket end on the proposal's side moves to it; cap -> null move */
    int accepted = 0;
    for (int r = 0; r < ORC_SHRINK_CAP; ++r) {
        double u = orc_u24(orc_word(key, iter, chain, step, nz + 3u + (uint32_t)r));
        double t = tl + u * (tr - tl);
        orc_line(d, x, t, v, y);
        double lly;
        cnt->shrinks++;
        if (orc_in_slice(&sl, y, &lly)) {
            memcpy(x, y, sizeof(double) * d);
            *logLx = lly;
            accepted = 1;
            break;
        }
        if (t < 0.0) tl = t; else tr = t;
    }
    if (accepted) cnt->accepts++; else cnt->nulls++;
    free(z); free(v); free(y);
}

/* Constrained Gaussian random walk (the baseline replacement kernel of
   Sec. 3.1 and App. "Slice sampling vs random walk"): one proposal
   y = x + s L z per step, z ~ N(0, I) from the step's normal words, L the
   live-set Cholesky factor (proposal covariance s^2 L L^T, matched to the
   live set).  y replaces x when it is in the prior support, above logL*,
   and, for a Gaussian prior, passes the Metropolis test
   ln u < log Pi(y) - log Pi(x) with u the step's word 2 ceil(d/2);
   otherwise the chain stays (a null move). */
void orc_rw_step(const orc_problem *pb, const double *L, double scale, double logLstar,
                 uint64_t seed, uint32_t run_id, uint32_t iter, uint32_t chain, uint32_t step,
                 double *x, double *logLx, orc_counts *cnt)
{
    int d = pb->d;
    uint32_t key[2];
    orc_key(seed, run_id, key);
    uint32_t nz = 2u * (uint32_t)((d + 1) / 2);
    double *z = (double *)malloc(sizeof(double) * d);
    double *y = (double *)malloc(sizeof(double) * d);
    orc_normals(key, iter, chain, step, d, z);
    for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int b = 0; b <= a; ++b) s += L[a * d + b] * z[b];
        y[a] = x[a] + scale * s;
    }
    orc_slice sl;
    sl.pb = pb; sl.logLstar = logLstar; sl.cnt = cnt; sl.y = y;
    sl.nonflat = pb->prior_kind != ORC_PRIOR_BOX;
    sl.height = 0.0;
    if (sl.nonflat) sl.height = orc_log_prior(pb, x) + log(orc_u24(orc_word(key, iter, chain, step, nz)));
    double lly;
    if (orc_in_slice(&sl, y, &lly)) {
        memcpy(x, y, sizeof(double) * d);
        *logLx = lly;
        cnt->accepts++;
    } else {
        cnt->nulls++;
    }
    free(z); free(y);
}

/* ------------------------------------------------------------------------ */
/* One outer iteration (Sec. 3.1 (i)-(iv); Algorithm 1).  The live set is    */
/* x [m][d], logL [m], birth [m]; the dead points of this iteration are      */
/* appended to the store when one is given (cap > n_dead).                   */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_problem *pb, const orc_opts *op, uint32_t iter,
             double *x, double *logL, double *birth, double *logZ, double *logX,
             double *dead_x, double *dead_logL, double *dead_birth, int *dead_n,
             long long *n_dead, long long cap, orc_trace *tr, long long *evals_total)
{
    int m = op->n_live, k = op->k, d = pb->d;
    int *dead = (int *)malloc(sizeof(int) * k);
    int *surv = (int *)malloc(sizeof(int) * (m - k));
    int *parent = (int *)malloc(sizeof(int) * k);
    double *L = (double *)malloc(sizeof(double) * d * d);
    double *nx = (double *)malloc(sizeof(double) * (size_t)k * d);
    double *nl = (double *)malloc(sizeof(double) * k);
    double logLstar;

    /* (i) delete the k worst, threshold logL* = k-th worst */
    orc_select(m, k, logL, dead, surv, &logLstar);

    /* record the dead points, unrolled with n = m, m-1, ..., m-k+1 (App. D.1) */
    for (int j = 0; j < k; ++j) {
        int s = dead[j];
        orc_evidence_death(logL[s], m - j, logZ, logX);
        if (dead_x && n_dead && *n_dead < cap) {
            memcpy(dead_x + (size_t)(*n_dead) * d, x + (size_t)s * d, sizeof(double) * d);
            dead_logL[*n_dead] = logL[s];
            dead_birth[*n_dead] = birth[s];
            dead_n[*n_dead] = m - j;
            (*n_dead)++;
        } else if (dead_x && n_dead) {
            free(dead); free(surv); free(parent); free(L); free(nx); free(nl);
            return -4;
        }
    }

    /* adaptive metric from the live set at the start of the iteration */
    orc_metric(m, d, x, op->cov_eps, L);

    /* (ii) resample parents from the survivors */
    orc_parents(op->seed, op->run_id, iter, m, k, surv, parent);

    /* (iii) mutate: p HRSS steps from each parent */
    for (int j = 0; j < k; ++j) {
        orc_counts cnt;
        memset(&cnt, 0, sizeof(cnt));
        cnt.margin = INFINITY; cnt.pmargin = INFINITY; cnt.bmargin = INFINITY;
        double *xj = nx + (size_t)j * d;
        memcpy(xj, x + (size_t)parent[j] * d, sizeof(double) * d);
        double lj = logL[parent[j]];
        double rws = op->rw_scale > 0.0 ? op->rw_scale : 2.38 / sqrt((double)d);
        for (int s = 0; s < op->p; ++s) {
            if (op->kernel == 1)
                orc_rw_step(pb, L, rws, logLstar, op->seed, op->run_id, iter, (uint32_t)j, (uint32_t)s,
                            xj, &lj, &cnt);
            else
                orc_hrss_step(pb, L, op->w, op->dir_norm, logLstar, op->seed, op->run_id,
                              iter, (uint32_t)j, (uint32_t)s, xj, &lj, &cnt);
        }
        nl[j] = lj;
        if (evals_total) *evals_total += cnt.evals;
        if (tr) {
            tr->evals[j] = cnt.evals; tr->accepts[j] = cnt.accepts; tr->nulls[j] = cnt.nulls;
            tr->expansions[j] = cnt.expansions; tr->shrinks[j] = cnt.shrinks;
            tr->cap_out[j] = cnt.cap_out;
            tr->margin[j] = cnt.margin; tr->pmargin[j] = cnt.pmargin; tr->bmargin[j] = cnt.bmargin;
        }
    }

    /* (iv) replace the dead slots with the new points, born at logL* */
    for (int j = 0; j < k; ++j) {
        int s = dead[j];
        memcpy(x + (size_t)s * d, nx + (size_t)j * d, sizeof(double) * d);
        logL[s] = nl[j];
        birth[s] = logLstar;
    }

    int stop = orc_should_stop(m, logL, *logZ, *logX, op->tol);
    if (tr) {
        memcpy(tr->dead_idx, dead, sizeof(int) * k);
        memcpy(tr->parent, parent, sizeof(int) * k);
        memcpy(tr->L, L, sizeof(double) * d * d);
        memcpy(tr->new_x, nx, sizeof(double) * (size_t)k * d);
        memcpy(tr->new_logL, nl, sizeof(double) * k);
        tr->logLstar = logLstar;
        tr->logZ = *logZ; tr->logX = *logX;
        tr->done = stop;
    }
    free(dead); free(surv); free(parent); free(L); free(nx); free(nl);
    return stop;
}

/* Kill the final live set in (logL, slot) order with n = m, m-1, ..., 1
   (X_{N+1} := 0 in App. D.2). */
int orc_kill_live(const orc_problem *pb, int m, const double *x, const double *logL, const double *birth,
                  double *logZ, double *logX, double *dead_x, double *dead_logL, double *dead_birth,
                  int *dead_n, long long *n_dead, long long cap)
{
    int d = pb->d;
    int *order = (int *)malloc(sizeof(int) * m);
    for (int i = 0; i < m; ++i) order[i] = i;
    g_sort_logL = logL;
    qsort(order, m, sizeof(int), orc_cmp_slot);
    for (int j = 0; j < m; ++j) {
        int s = order[j];
        orc_evidence_death(logL[s], m - j, logZ, logX);
        if (*n_dead >= cap) { free(order); return -4; }
        memcpy(dead_x + (size_t)(*n_dead) * d, x + (size_t)s * d, sizeof(double) * d);
        dead_logL[*n_dead] = logL[s];
        dead_birth[*n_dead] = birth[s];
        dead_n[*n_dead] = m - j;
        (*n_dead)++;
    }
    free(order);
    return 0;
}

/* Draw the initial live set; logL of each prior draw, birth level -inf. */
void orc_init_live(const orc_problem *pb, const orc_opts *op, double *x, double *logL, double *birth)
{
    int d = pb->d;
    for (int i = 0; i < op->n_live; ++i) {
        orc_prior_draw(pb, op->seed, op->run_id, (uint32_t)i, x + (size_t)i * d);
        logL[i] = orc_loglik(pb, x + (size_t)i * d);
        birth[i] = -INFINITY;
    }
}

/* Whole run: initial draws, iterations until the termination test holds,
   then the final live set.  Dead points go to caller buffers of size cap. */
int orc_run(const orc_problem *pb, const orc_opts *op,
            double *dead_x, double *dead_logL, double *dead_birth, int *dead_n, long long cap,
            orc_summary *sum)
{
    int m = op->n_live, d = pb->d;
    double *x = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *logL = (double *)malloc(sizeof(double) * m);
    double *birth = (double *)malloc(sizeof(double) * m);
    orc_init_live(pb, op, x, logL, birth);
    double logZ = -INFINITY, logX = 0.0;
    long long n_dead = 0, evals = 0;
    int it = 0, status = 0;
    for (;;) {
        if (it >= op->max_iter) { status = 1; break; }
        int st = orc_step(pb, op, (uint32_t)it, x, logL, birth, &logZ, &logX,
                          dead_x, dead_logL, dead_birth, dead_n, &n_dead, cap, NULL, &evals);
        it++;
        if (st < 0) { status = st; break; }
        if (st == 1) break;
    }
    if (status >= 0) {
        int ks = orc_kill_live(pb, m, x, logL, birth, &logZ, &logX, dead_x, dead_logL, dead_birth,
                               dead_n, &n_dead, cap);
        if (ks < 0) status = ks;
    }
    sum->n_dead = n_dead; sum->iters = it; sum->evals = evals;
    sum->logZ_det = logZ; sum->logX = logX; sum->status = status;
    sum->nulls = 0; sum->cap_out = 0;
    free(x); free(logL); free(birth);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Post-hoc volume simulation (App. D.2): R trajectories, each death with    */
/* n live points shrinks log X by log(u)/n, u ~ U(0,1); trapezoid elements    */
/* dX_i = (X_{i-1} - X_{i+1})/2 with X_0 = 1, X_{N+1} = 0; per trajectory    */
/* log Z^(r) = logsumexp_i (log L_i + log dX_i); the estimate is the mean     */
/* over r, its error the standard deviation (ddof 1); posterior weights are  */
/* the geometric mean over r of w_i^(r), normalised.                          */
/* ------------------------------------------------------------------------ */
int orc_finalise(long long n, const double *logL, const int *nlive, int R,
                 uint64_t seed, uint32_t run_id,
                 double *logZ_mean, double *logZ_std, double *log_w, double *logZ_r)
{
    uint32_t key[2];
    orc_key(seed, run_id, key);
    double *lx = (double *)malloc(sizeof(double) * (size_t)(n + 2));
    double *lwsum = (double *)calloc((size_t)n, sizeof(double));
    double *lz = (double *)malloc(sizeof(double) * R);
    for (int r = 0; r < R; ++r) {
        lx[0] = 0.0;
        for (long long i = 1; i <= n; ++i) {
            long long di = i - 1;
            uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(di >> 1), ORC_TAG_VOLSIM, 0u}, out[4];
            orc_philox4x32_10(ctr, key, out);
            int o = (int)(di & 1) * 2;
            double u = orc_u53(out[o], out[o + 1]);
            lx[i] = lx[i - 1] + log(u) / nlive[di];
        }
        double acc = -INFINITY;
        for (long long i = 1; i <= n; ++i) {
            double ldx;
            if (i < n) ldx = lx[i - 1] + log1p(-exp(lx[i + 1] - lx[i - 1])) - log(2.0);
            else ldx = lx[i - 1] - log(2.0);
            double lw = logL[i - 1] + ldx;
            lwsum[i - 1] += lw;
            acc = orc_logaddexp(acc, lw);
        }
        lz[r] = acc;
    }
    double mean = 0.0;
    for (int r = 0; r < R; ++r) mean += lz[r];
    mean /= R;
    double var = 0.0;
    for (int r = 0; r < R; ++r) var += (lz[r] - mean) * (lz[r] - mean);
    var = R > 1 ? var / (R - 1) : 0.0;
    *logZ_mean = mean;
    *logZ_std = sqrt(var);
    if (logZ_r) memcpy(logZ_r, lz, sizeof(double) * R);
    if (log_w) {
        double acc = -INFINITY;
        for (long long i = 0; i < n; ++i) { log_w[i] = lwsum[i] / R; acc = orc_logaddexp(acc, log_w[i]); }
        for (long long i = 0; i < n; ++i) log_w[i] -= acc;
    }
    free(lx); free(lwsum); free(lz);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Slice-width theory helpers (App. E).                                      */
/* ------------------------------------------------------------------------ */

/* u* solves u - ln(1+u) = 1/2 (Theorem "optimal slice width in a fixed
   slice"); bisection on the strictly increasing g(u) = u - ln(1+u). */
double orc_u_star(void)
{
    double lo = 0.0, hi = 10.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid - log1p(mid) < 0.5) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Expected HRSS cost on a slice of length ell (Theorem "computational cost"):
   E[N_out] = ell/w, E[N_shrink] = 1 + 2 phi(w/ell),
   phi(u) = ((1+u) ln(1+u) - u)/u. */
double orc_phi(double u) { return ((1.0 + u) * log1p(u) - u) / u; }

/* kappa_inf solves kappa = 1/2 + E[R ln(1 + kappa/R)], R = sqrt(S)/E[sqrt(S)],
   S ~ Gamma(3/2, scale 2) (Theorem "optimal slice width in an ellipsoid"),
   by fixed-point iteration; the expectation by composite Simpson in
   s = q^2 over q in [0, 40]. */
double orc_kappa_inf(void)
{
    const double c = 2.0 * sqrt(2.0 / M_PI);          /* E[sqrt(S)] */
    const double g32 = 0.5 * sqrt(M_PI);              /* Gamma(3/2) */
    const int N = 200000;
    const double qmax = 40.0;
    double kappa = 1.0;
    for (int it = 0; it < 200; ++it) {
        double h = qmax / N, acc = 0.0;
        for (int i = 0; i <= N; ++i) {
            double q = i * h;
            double f = 0.0;
            if (q > 0.0) {
                double s = q * q;
                /* density of S at s times ds/dq = 2q */
                double fs = sqrt(s) * exp(-0.5 * s) / (g32 * pow(2.0, 1.5));
                double Rv = q / c;
                f = Rv * log1p(kappa / Rv) * fs * 2.0 * q;
            }
            double wgt = (i == 0 || i == N) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            acc += wgt * f;
        }
        double nk = 0.5 + acc * h / 3.0;
        if (fabs(nk - kappa) < 1e-13) { kappa = nk; break; }
        kappa = nk;
    }
    return kappa;
}

/* Mean chord E[l_d] through a uniform point of a d-ball of radius R along a
   uniform direction: l = 2 sqrt(R^2 - r^2 sin^2 th), r with density
   d r^(d-1)/R^d, th with density ∝ sin^(d-2) th on [0, pi]; 2-D composite
   Simpson.  Used by the slice-width rule w = kappa_inf E[l_d] with
   R = sqrt(d+2) (the whitened uniform ball, Sec. 3.3 "Isotropic level sets"). */
double orc_mean_chord_ball(int d, double R)
{
    if (d == 1) return 2.0 * R;
    const int NR = 2000, NT = 2000;
    double hr = R / NR, ht = M_PI / NT;
    double num = 0.0, den = 0.0;
    for (int j = 0; j <= NT; ++j) {
        double th = j * ht;
        double wt = (j == 0 || j == NT) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
        double st = sin(th);
        double pth = d == 2 ? 1.0 : pow(st, d - 2);
        den += wt * pth;
        double inner = 0.0;
        for (int i = 0; i <= NR; ++i) {
            double r = i * hr;
            double wr = (i == 0 || i == NR) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            double pr = d * pow(r, d - 1) / pow(R, d);
            double v = R * R - r * r * st * st;
            inner += wr * pr * 2.0 * sqrt(v > 0.0 ? v : 0.0);
        }
        num += wt * pth * inner * hr / 3.0;
    }
    return num / den;
}

/* One volume trajectory r of the post-hoc simulation (App. D.2):
   log X_i = log X_{i-1} + log(u_{r,i}) / n_i, log X_0 = 0. */
void orc_volume_trajectory(long long n, const int *nlive, int r, uint64_t seed, uint32_t run_id,
                           double *logX)
{
    uint32_t key[2];
    orc_key(seed, run_id, key);
    double acc = 0.0;
    for (long long i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(i >> 1), ORC_TAG_VOLSIM, 0u}, out[4];
        orc_philox4x32_10(ctr, key, out);
        int o = (int)(i & 1) * 2;
        acc += log(orc_u53(out[o], out[o + 1])) / nlive[i];
        logX[i] = acc;
    }
}

/* Posterior expectations over weighted dead points, with the normalised
   weights w_i = exp(log_w_i) of App. D.2, and the Fisher identity: for
   Z(theta) = int L(x; theta) Pi(x; theta) dx,
     d log Z / d theta = E_post[d/dtheta log L(x; theta) + d/dtheta log Pi(x; theta)].
   kind 0: likelihood width sigma (Gaussian / equal-weight mixture)
           d/dsigma log L = sum_c r_c |x - mu_c|^2 / sigma^3 - d / sigma;
   kind 1: the means, n_comp * d values: r_c (x - mu_c) / sigma^2;
   kind 2: a common log-precision lambda of a Gaussian prior (sd b_i e^{-lambda/2})
           at lambda = 0: d/2 - sum_i ((x_i - a_i) / b_i)^2 / 2;
   kind 3: a noise multiplier s of the GP (K = a^2 k + (s sigma_n)^2 I) at s = 1:
           sigma_n^2 (|K^-1 y|^2 - tr K^-1);
   kind 4: the posterior mean of x, d values.
   r_c = N(x; mu_c) / sum_c' N(x; mu_c').  Returns the number of values written,
   or -1 if the kind does not apply. */
static double orc_gp_noise_term(const orc_problem *pb, const double *th)
{
    int n = pb->n_data;
    double ell = exp(th[0]), amp = exp(th[1]), sn = exp(th[2]);
    double *K = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *beta = (double *)malloc(sizeof(double) * n);
    if (!K || !z || !beta) { free(K); free(z); free(beta); return NAN; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double dt = pb->t[i] - pb->t[j];
            K[i * n + j] = amp * amp * exp(-dt * dt / (2.0 * ell * ell)) + (i == j ? sn * sn : 0.0);
        }
    double out = NAN;
    if (orc_cholesky_inplace(n, K) == 0) {
        /* beta = K^-1 y: L z = y, then L^T beta = z */
        for (int i = 0; i < n; ++i) {
            double s = pb->y[i];
            for (int j = 0; j < i; ++j) s -= K[i * n + j] * z[j];
            z[i] = s / K[i * n + i];
        }
        double bb = 0.0;
        for (int i = n - 1; i >= 0; --i) {
            double s = z[i];
            for (int j = i + 1; j < n; ++j) s -= K[j * n + i] * beta[j];
            beta[i] = s / K[i * n + i];
            bb += beta[i] * beta[i];
        }
        /* tr K^-1 = sum_j |L^-1 e_j|^2 */
        double tr = 0.0;
        for (int c = 0; c < n; ++c) {
            for (int i = c; i < n; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int j = c; j < i; ++j) s -= K[i * n + j] * z[j];
                z[i] = s / K[i * n + i];
                tr += z[i] * z[i];
            }
        }
        out = sn * sn * (bb - tr);
    }
    free(K); free(z); free(beta);
    return out;
}

int orc_posterior_expectation(const orc_problem *pb, int kind, long long n, const double *x,
                              const double *log_w, double *out)
{
    int d = pb->d;
    int gauss = pb->lik_kind == ORC_LIK_GAUSS || pb->lik_kind == ORC_LIK_GMM;
    int K = pb->lik_kind == ORC_LIK_GMM ? pb->n_comp : 1;
    int count;
    switch (kind) {
    case 0: count = gauss ? 1 : -1; break;
    case 1: count = gauss ? K * d : -1; break;
    case 2: count = pb->prior_kind == ORC_PRIOR_GAUSS ? 1 : -1; break;
    case 3: count = pb->lik_kind == ORC_LIK_GP ? 1 : -1; break;
    case 4: count = d; break;
    default: count = -1;
    }
    if (count < 0) return -1;
    for (int q = 0; q < count; ++q) out[q] = 0.0;
    double s2 = pb->sigma * pb->sigma;
    double *qd = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
    double *r = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
    for (long long i = 0; i < n; ++i) {
        const double *xi = x + i * d;
        double w = exp(log_w[i]);
        if (kind == 4) {
            for (int a = 0; a < d; ++a) out[a] += w * xi[a];
        } else if (kind == 2) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) { double u = (xi[a] - pb->a[a]) / pb->b[a]; s += u * u; }
            out[0] += w * (0.5 * d - 0.5 * s);
        } else if (kind == 3) {
            if (w > 0.0) out[0] += w * orc_gp_noise_term(pb, xi);
        } else {
            double qmin = INFINITY;
            for (int c = 0; c < K; ++c) {
                double s = 0.0;
                for (int a = 0; a < d; ++a) { double e = xi[a] - pb->mu[c * d + a]; s += e * e; }
                qd[c] = s;
                if (s < qmin) qmin = s;
            }
            double rs = 0.0;
            for (int c = 0; c < K; ++c) { r[c] = exp(-(qd[c] - qmin) / (2.0 * s2)); rs += r[c]; }
            if (kind == 0) {
                double e = 0.0;
                for (int c = 0; c < K; ++c) e += r[c] * qd[c];
                out[0] += w * (e / rs / (s2 * pb->sigma) - d / pb->sigma);
            } else {
                for (int c = 0; c < K; ++c)
                    for (int a = 0; a < d; ++a) out[c * d + a] += w * (r[c] / rs) * (xi[a] - pb->mu[c * d + a]) / s2;
            }
        }
    }
    free(qd); free(r);
    return count;
}
