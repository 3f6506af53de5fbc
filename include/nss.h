/*
 * nss.h -- C ABI of the GB300 (sm_103a) Nested Slice Sampling library
 * (libnss_gb300.so).
 *
 * The library implements the batched constrained-update sweep of Nested
 * Slice Sampling (Yallup, Kroupa & Handley, arxiv 2601.23252):
 *   (i)   delete the k lowest-likelihood live points, threshold logL* = the
 *         largest of them                              (Sec. 3.1 (i); Alg. 1)
 *   (ii)  resample k parents uniformly from the m-k survivors (Sec. 3.1 (ii))
 *   (iii) whiten directions with the Cholesky factor of the regularised
 *         live-set covariance                          (Sec. 3.2 "Direction metric")
 *         and run k Hit-and-Run Slice Sampling chains of p steps each, with
 *         stepping-out (<= 10 per side) and shrinkage (<= 100, then a null
 *         move), the likelihood evaluated inside the sweep (Sec. 3.2; App. B.4)
 *   (iv)  replace the dead slots                       (Sec. 3.1 (iv))
 * plus the unrolled evidence bookkeeping (Eq. eq:marginal, Eq. eq:dlnX,
 * App. D.1) and the post-hoc volume-shrinkage simulation, posterior weights
 * and evidence error (App. D.2).
 *
 * Conventions
 *   - log-likelihood throughout (the paper's energy is E = -log L); the
 *     constraint E < E_batch reads logL > logL* (strict).
 *   - Positions, likelihoods and slice arithmetic are FP32; the evidence,
 *     log prior volume and volume simulation accumulate in FP64.
 *   - Random numbers: Philox4x32-10 keyed by (seed_lo32, seed_hi32 ^ run_id);
 *     counter (iteration, chain, step, word/4) for the HRSS draws, with the
 *     word layout of each step: [0, 2*ceil(d/2)) Box-Muller pairs, then the
 *     bracket position U, the prior slice height, one reserved word, and the
 *     shrinkage proposals r = 0..99.  Uniforms u = (2*(w>>9)+1) * 2^-24.
 *
 * Ownership: the library allocates and owns all device state of a context.
 * Input arrays (prior bounds, likelihood parameters and data) are read from
 * host memory and copied during nss_create*; the caller may free them after
 * the call returns.  Output arrays are caller-owned and may be host or
 * device pointers (unified addressing decides the copy direction).
 *
 * Errors: every entry point returns an nss_status; nothing aborts, throws or
 * resets device state.  A CUDA error is reported as NSS_ERR_CUDA and leaves
 * the context unusable except for nss_destroy; nss_last_error() gives text.
 * No device code waits on another block, so no kernel can hang.
 *
 * Threading and streams: a context is used by one host thread at a time.
 * All device work of a context is enqueued on the stream given in
 * nss_options.cuda_stream (NULL = the legacy default stream).
 */
#ifndef NSS_GB300_H
#define NSS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NSS_ABI_VERSION 7

typedef struct nss_ctx nss_ctx;

typedef enum {
    NSS_OK = 0,
    NSS_DONE = 1,            /* the termination test holds for every run     */
    NSS_ERR_ARG = -1,        /* invalid argument; nothing was done           */
    NSS_ERR_CUDA = -2,       /* CUDA runtime error (text in nss_last_error)  */
    NSS_ERR_OOM = -3,        /* device allocation failed                      */
    NSS_ERR_CAPACITY = -4,   /* the dead-point store of a run is full         */
    NSS_ERR_TIMEOUT = -5,    /* max_iter reached before termination           */
    NSS_ERR_NUMERIC = -6,    /* non-finite evidence                            */
    NSS_ERR_STATE = -7       /* call out of order (e.g. trace before a step)  */
} nss_status;

/* Prior Pi (Eq. eq:target).  Box: uniform on [a_i, b_i]; Gaussian: independent
   N(a_i, b_i^2).  a and b are host arrays of length d. */
enum { NSS_PRIOR_UNIFORM_BOX = 0, NSS_PRIOR_GAUSS_DIAG = 1 };
typedef struct {
    int kind;
    int d;
    const double *a;
    const double *b;
} nss_prior;

/* Likelihood L = exp(-E) (Eq. eq:target).  Kinds and their fields:
 *   GAUSS_ISO       normalised N(x; mu, sigma^2 I); mu [d]
 *   GMM_ISO_EQUAL   (1/n_comp) sum_c N(x; mu_c, sigma^2 I); mu [n_comp][d]
 *   LOGREG          sum_n [y_n z_n - softplus(z_n)], z = X x; X [n_data][d]
 *                   row-major FP32 (values are used as given, rounded to
 *                   bfloat16 on the device: pass bf16-exact data), y [n_data]
 *   GP_RBF_WHITE    theta = (ln lengthscale, ln amplitude, ln noise); GP
 *                   marginal likelihood of gp_y [n_data] at gp_t [n_data]
 *   FLAT            logL = 0 (pure prior / plateau tests)
 *   TEST_FAULT      isotropic Gaussian whose value is replaced by NaN
 *                   (fault_mode 1) or +inf (fault_mode 2) where x_0 <
 *                   fault_param; NaN is read as -inf and counted.
 *   RASTRIGIN       the Gaussian-Rastrigin mixture of App. F.3 (unnormalised):
 *                   L = alpha exp(-|x|^2/2)
 *                       + (1 - alpha) exp(-A d + A sum_i cos(2 pi x_i)), A = 10;
 *                   0 <= alpha <= 1 in `alpha`.  Its slice tests evaluate the
 *                   cosine sum per test (it is not affine along a line).
 * All pointers are host pointers, copied at create. */
enum {
    NSS_LOGLIK_GAUSS_ISO = 0,
    NSS_LOGLIK_GMM_ISO_EQUAL = 1,
    NSS_LOGLIK_LOGREG = 2,
    NSS_LOGLIK_GP_RBF_WHITE = 3,
    NSS_LOGLIK_FLAT = 4,
    NSS_LOGLIK_TEST_FAULT = 5,
    NSS_LOGLIK_RASTRIGIN = 6
};
typedef struct {
    int kind;
    int n_comp;
    int n_data;
    double sigma;
    const double *mu;
    const float *X;
    const float *y;
    const double *gp_t;
    const double *gp_y;
    int fault_mode;
    double fault_param;
    double alpha;              /* RASTRIGIN mixture weight                      */
} nss_loglik;

/* Direction normalisation: MAHAL v = L z / |z| (unit Mahalanobis length, the
   slice width then acts in whitened units, App. B.3); EUCLID v = L z / |L z|
   (the literal form of Sec. 3.2). */
enum { NSS_DIR_MAHAL = 0, NSS_DIR_EUCLID = 1 };
/* Slice-width rule: FIXED uses w as given (the paper's experiments use
   w = 1.0, App. B.3); THEORY uses w = kappa_inf * E[l_d] for the uniform
   whitened ball of radius sqrt(d+2) (Theorem "optimal slice width in an
   ellipsoid"; Sec. 3.3 "Isotropic level sets"). */
enum { NSS_W_FIXED = 0, NSS_W_THEORY = 1 };

typedef struct {
    uint64_t seed;
    uint32_t run_id;
    double w;                  /* slice width (NSS_W_FIXED)                      */
    int w_rule;                /* NSS_W_FIXED or NSS_W_THEORY                    */
    int dir_norm;              /* NSS_DIR_MAHAL or NSS_DIR_EUCLID                */
    double tol;                /* stop when Z_live/(Z+Z_live) < tol (App. B.3)   */
    int max_iter;              /* iteration cap; reaching it ends the run        */
    long long dead_capacity;   /* dead points per run; 0 = 2000*k + m           */
    int n_sim;                 /* volume-simulation trajectories R (App. D.2)    */
    double cov_eps;            /* metric regularisation eps * tr(Sigma)/d        */
    void *cuda_stream;         /* cudaStream_t; NULL = default stream            */
    int sweep_cfg;             /* sweep configuration id, -1 = default           */
    int kernel;                /* NSS_KERNEL_HRSS (the paper's NSS) or
                                  NSS_KERNEL_RW (constrained random walk)       */
    double rw_scale;           /* RW proposal x + rw_scale * L z; 0 = 2.38/sqrt(d) */
    int path;                  /* NSS_PATH_BATCHED (default) or NSS_PATH_PLAIN   */
    int run_groups;            /* batched path: 0 = automatic (two streams when
                                  every run uses the generic sweep), 1 = one    */
    int dir_fp32;              /* 0: the whitening L z of the step directions on
                                  the tensor cores (tcgen05 kind::tf32, 3xTF32
                                  split, FP32 accumulation) for 16 < d <= 64;
                                  1: FP32 CUDA cores for every d (same for
                                  every run of a context)                       */
} nss_options;

/* Execution paths.  BATCHED: the device-resident batched sweep (persistent
   chain-group kernels, directions drawn ahead, outer iterations replayed
   from CUDA graphs, many runs per launch).  PLAIN: the plain single-run FP32
   GPU path that the batched sweep is measured against -- one kernel per
   phase of an outer iteration (selection; dead append and evidence; metric;
   parents; directions; one HRSS kernel launch per step; termination), the
   run's k chains as one thread each advancing in lockstep evaluation rounds
   (every chain evaluates one candidate per round, as one batched likelihood
   call over the k chains does, Sec. 3.1 "Vectorised execution"), every
   candidate's likelihood evaluated from scratch over all d coordinates, and
   a host loop that waits for each iteration.  Its FP32 expressions follow
   the batched sweep's in the run's sweep configuration, so both paths give
   bit-identical dead points for the same configuration.  For a logistic
   likelihood each round's candidate points take their logits from one
   tensor-core GEMM over all k chains (the batched path forms them
   line-affinely, one GEMM per HRSS step), and the host reads after every
   round whether a chain is still testing.  PLAIN requires a single run
   (nss_create or n_runs = 1), the HRSS kernel, a Gaussian, mixture, flat or
   logistic likelihood, k <= 1024 and a grouped sweep configuration
   (sweep_cfg < 22; -1 picks the default one); otherwise NSS_ERR_ARG. */
enum { NSS_PATH_BATCHED = 0, NSS_PATH_PLAIN = 1 };

/* Replacement kernels.  HRSS: hit-and-run slice sampling (Sec. 3.2).  RW:
   the constrained Gaussian random-walk baseline (Sec. 3.1 "Vectorised
   execution"; App. "Slice sampling vs random walk"): each of the p steps
   proposes y = x + s L z with L the live-set Cholesky factor (the proposal
   covariance matched to the live set) and z ~ N(0, I) from the step's normal
   words; y replaces x when it lies in the prior support, logL(y) > logL* and,
   for a Gaussian prior, ln u < ln Pi(y) - ln Pi(x) (Metropolis, u the step's
   word 2 ceil(d/2)); otherwise the chain stays (a rejected step counts as a
   null move).  Gaussian, mixture and flat likelihoods only. */
enum { NSS_KERNEL_HRSS = 0, NSS_KERNEL_RW = 1 };

/* Fills the paper's defaults: w = 1, MAHAL, tol = 1e-3, max_iter = 100000,
   n_sim = 100, cov_eps = 1e-6, seed 0, run_id 0, default stream,
   default sweep configuration, the batched path, automatic run groups. */
void nss_options_default(nss_options *opt);

/* Per-run state after a step. */
typedef struct {
    int iter;                  /* iterations completed                           */
    int done;                  /* termination test held                          */
    float logLstar;            /* threshold of the last iteration                */
    double logZ;               /* running Delta-X evidence (deterministic X)     */
    double logX;               /* deterministic log prior volume, -sum 1/n       */
    long long n_dead;
    long long evals;           /* logical likelihood evaluations so far          */
    long long nulls;           /* HRSS steps that hit the shrinkage cap          */
    long long cap_out;         /* stepping-out sides stopped by the cap          */
    long long nan_evals;       /* evaluations whose likelihood was NaN           */
    long long spec_evals;      /* slice tests run beyond the logical evaluations
                                  (a chain group tests several stepping-out ends
                                  or shrinkage proposals at once)               */
    long long group_rounds;    /* slice-test rounds run by the chain groups of
                                  the grouped sweep (a warp's groups run every
                                  round until all of them are done), summed over
                                  groups                                        */
    long long active_group_rounds; /* ... of which the group was still testing:
                                  the rest are lockstep idle rounds             */
    int metric_status;         /* 0 ok, 1 identity fallback, 2 jitter retried    */
    int status;                /* nss_status of the run                          */
} nss_step_info;

/* Result of a finished run (App. D.2): logZ = mean over the R simulated
   volume trajectories, logZ_err = their standard deviation (ddof 1),
   logZ_det = the running Delta-X estimate with deterministic volumes. */
typedef struct {
    double logZ;
    double logZ_err;
    double logZ_det;
    long long n_dead;
    int iters;
    long long evals;
    long long nulls;
    long long cap_out;
    long long nan_evals;
    long long spec_evals;      /* as in nss_step_info                            */
    long long group_rounds;    /* as in nss_step_info                            */
    long long active_group_rounds;
    int status;
} nss_result;

/* State of one run for export/import (checkpoint/resume and parity tests). */
typedef struct {
    int iter;
    double logZ;
    double logX;
    long long n_dead;
} nss_state;

/* Per-chain record of the last iteration of one run; host pointers of
   length k (L: d*d, row-major lower triangle, zeros above). */
typedef struct {
    int *dead_idx;       /* slots deleted, worst first                  */
    int *parent;         /* parent slot of each chain                    */
    float *L;            /* Cholesky factor of the metric                */
    int *evals, *accepts, *nulls, *expansions, *shrinks, *cap_out;
    float *new_x;        /* [k][d] final chain positions                 */
    float *new_logL;     /* [k]                                          */
    float logLstar;
} nss_trace;

/* Per-kernel timing collected while profiling is on (CUDA events on the
   stream of every launch of that kernel, around the launch).  With two run
   groups the groups' launches overlap in time, so the per-kind sums can
   exceed the wall time; a context with run_groups = 1 serialises them. */
#define NSS_PROFILE_KINDS 12
typedef struct {
    long long launches[NSS_PROFILE_KINDS];
    double ms[NSS_PROFILE_KINDS];          /* summed event time           */
    long long total_launches;
    long long h2d_bytes;   /* host-to-device bytes copied by the library   */
    long long d2h_bytes;   /* device-to-host bytes copied by the library   */
} nss_profile;
/* INIT prior draw; PROLOGUE selection, evidence, metric, parents (one
   kernel, or the plain path's four); SWEEP the HRSS sweep (generic
   likelihoods; the plain path's per-step kernel); TERMINATE; FINAL_SORT;
   VOLSIM every volume-simulation kernel; DIRGEN the directions drawn ahead;
   LOGITS the tensor-core logistic contraction; LR_SLICE the logistic slice
   kernel; GP_SWEEP the GP sweep; OTHER the logistic helpers (centre,
   parents, directions, replacement).  Kind 6 is unused. */
enum { NSS_K_INIT = 0, NSS_K_PROLOGUE = 1, NSS_K_SWEEP = 2, NSS_K_TERMINATE = 3,
       NSS_K_FINAL_SORT = 4, NSS_K_VOLSIM = 5, NSS_K_WEIGHTS = 6, NSS_K_OTHER = 7,
       NSS_K_DIRGEN = 8, NSS_K_LOGITS = 9, NSS_K_LR_SLICE = 10, NSS_K_GP_SWEEP = 11 };

/* Create a single-run context: copies the problem to the device and draws
   the m initial live points from the prior (Sec. 2.1).  n_live = m >= 2,
   1 <= k < m, p >= 1, 1 <= d <= 128. */
nss_status nss_create(const nss_prior *prior, const nss_loglik *loglik, int n_live, int k, int p,
                      const nss_options *opt, nss_ctx **out);

/* Create a context of n_runs independent runs advanced together (one launch
   per kernel for all runs).  prior, loglik, n_live, k, p and opt are arrays of
   length n_runs; the stream of opt[0] is used for all runs. */
nss_status nss_create_batch(int n_runs, const nss_prior *prior, const nss_loglik *loglik,
                            const int *n_live, const int *k, const int *p,
                            const nss_options *opt, nss_ctx **out);

/* One outer iteration (i)-(iv) for every run that has not terminated, then
   the termination test.  info: array of n_runs entries or NULL.  Returns
   NSS_DONE when every run has terminated. */
nss_status nss_step(nss_ctx *ctx, nss_step_info *info);

/* Iterate until every run terminates (or hits max_iter), kill the final
   live points (n = m, ..., 1), run the volume simulation and weights.
   res: array of n_runs entries or NULL. */
nss_status nss_run(nss_ctx *ctx, nss_result *res);

/* Start every run of the context again from a fresh prior draw (same
   problem, same sizes, no reallocation).  seeds: n_runs new seeds, or NULL to
   keep the current ones.  Counters and the dead-point store are cleared. */
nss_status nss_reset(nss_ctx *ctx, const uint64_t *seeds);

/* Sweep configurations.  A chain is owned by G lanes of a warp, each lane
   holding DPL of its dimensions (G x DPL = the smallest power of two >= max(d,
   4)); a warp runs 32/G chains.  nss_autotune times every configuration that
   fits each run's dimension for `iters` outer iterations from a fresh prior
   draw, keeps the fastest (device time per likelihood evaluation) for each
   dimension class, and leaves the context reset to its prior draw (call it
   right after create).  cfg_out: n_runs entries or NULL.  The configuration
   changes only the order of FP32 additions inside a likelihood, not the
   method. */
nss_status nss_autotune(nss_ctx *ctx, int iters, int *cfg_out);
nss_status nss_set_cfg(nss_ctx *ctx, int run, int cfg);
/* Cost measured by the last nss_autotune for every configuration id (device
   milliseconds per 10^6 logical evaluations; 0 = not tried).  cost: array of
   NSS_NUM_CFGS entries. */
#define NSS_NUM_CFGS 25
nss_status nss_autotune_report(const nss_ctx *ctx, double *cost);
int nss_get_cfg(const nss_ctx *ctx, int run);
int nss_cfg_lanes(int cfg);
int nss_cfg_dims(int cfg);

/* Finalise runs that were stepped to termination with nss_step. */
nss_status nss_finalise(nss_ctx *ctx, nss_result *res);

/* Dead points of run `run` in death order.  Any output pointer may be NULL;
   x is [n][d], log_w are normalised log posterior weights (valid after
   nss_run/nss_finalise), nlive the live count at each death.  cap = 0 only
   reports the count in *n_out. */
nss_status nss_get_dead(nss_ctx *ctx, int run, float *x, float *logL, double *log_w, float *birth,
                        int *nlive, size_t cap, size_t *n_out);

/* Live set of a run: x [m][d], logL [m], birth [m] (any may be NULL). */
nss_status nss_export_state(nss_ctx *ctx, int run, float *x, float *logL, float *birth,
                            nss_state *st);
nss_status nss_import_state(nss_ctx *ctx, int run, const float *x, const float *logL,
                            const float *birth, const nss_state *st);

/* Per-chain record of the last nss_step of run `run`. */
nss_status nss_step_trace(nss_ctx *ctx, int run, nss_trace *tr);

nss_status nss_set_profiling(nss_ctx *ctx, int on);
nss_status nss_get_profile(nss_ctx *ctx, nss_profile *prof);

/* The batched logit contraction of the logistic-regression sweep, exposed for
   verification: Z[j][n] = sum_i X[n][i] U[j][i] for host arrays X [n][d]
   (rounded to bfloat16, as the likelihood uses it) and U [nu][d] (FP32, split
   into three bfloat16 parts), computed by the tcgen05 tensor-core kernel with
   FP32 accumulation.  Z [nu][n] is a host array.  1 <= d <= 128,
   1 <= n <= 1<<20, 1 <= nu <= 1<<16.  Allocates and frees its own device
   memory; runs on the default stream and synchronises. */
nss_status nss_logreg_logits(const float *X, int n, int d, const float *U, int nu, float *Z);

/* The GP hyperparameter log-likelihood of the GP sweep, exposed for
   verification (Sec. 4.3; RBF + white kernel as NSS_LOGLIK_GP_RBF_WHITE):
   out[i] = -1/2 y^T K^-1 y - 1/2 ln det K - n/2 ln 2 pi at theta[i] =
   (ln l, ln a, ln s), K_ij = a^2 exp(-(t_i - t_j)^2 / (2 l^2)) + s^2 [i == j],
   computed by the tensor-core factorisation (kernel matrix in tensor memory,
   3xTF32 trailing updates with FP32 accumulation, FP64 ln det and |L^-1 y|^2);
   -inf where an FP32 pivot is not positive.  Host arrays t [n], y [n]
   (rounded to FP32), theta [m][3], out [m]; 1 <= n <= 256, 1 <= m <= 1<<20.
   Allocates and frees its own device memory; runs on the default stream
   and synchronises.  NSS_ERR_TIMEOUT if a tensor-core wait ran out. */
nss_status nss_gp_loglik(const double *t, const double *y, int n, const double *theta, int m, float *out);

/* Self-test of the device-side bounded waits (the tensor-core kernels wait
   on mbarriers with a poll limit, then record an error and return): a
   one-warp kernel waits on an mbarrier that nothing completes, with at most
   max_polls polls (1 <= max_polls <= 1<<20).  *outcome = 2 when the wait gave
   up as designed, 1 if it completed.  Allocates and frees its own device
   memory; runs on the default stream and synchronises.  NSS_ERR_ARG on bad
   arguments, NSS_ERR_CUDA on a CUDA error. */
nss_status nss_wait_selftest(unsigned max_polls, int *outcome);

/* Posterior expectations over a finished run's dead points (App. D.2 weights:
   the normalised geometric-mean weights w_i = exp(log_w_i), sum 1), reduced in
   FP64 on the device in a fixed order.  The gradient kinds are the Fisher
   identity: for Z(theta) = int L(x; theta) Pi(x; theta) dx,
     d log Z / d theta = E_post[ d/dtheta log L(x; theta) + d/dtheta log Pi(x; theta) ],
   estimated by sum_i w_i (d/dtheta log L + d/dtheta log Pi)(x_i).
     NSS_GRAD_LIK_SIGMA        GAUSS_ISO / GMM_ISO_EQUAL: the likelihood width sigma;
                               1 value: sum_c r_c |x - mu_c|^2 / sigma^3 - d / sigma
                               (r_c the component responsibilities)
     NSS_GRAD_LIK_MU           GAUSS_ISO / GMM_ISO_EQUAL: the means; n_comp * d
                               values: r_c (x - mu_c) / sigma^2
     NSS_GRAD_PRIOR_LOG_PREC   GAUSS_DIAG prior: a common log-precision lambda of
                               all coordinates (sd b_i -> b_i e^{-lambda/2}) at
                               lambda = 0; 1 value: d/2 - sum_i ((x_i - a_i)/b_i)^2 / 2
     NSS_GRAD_GP_NOISE_SCALE   GP_RBF_WHITE: a fixed multiplier s of the noise sd
                               (K = a^2 k + (s sigma_n)^2 I) at s = 1; 1 value:
                               sigma_n^2 (|K^-1 y|^2 - tr K^-1), from an FP32
                               Cholesky and triangular inverse of K per dead point
                               with weight above 1e-12 of the largest
     NSS_MOMENT_MEAN           any kind: the posterior mean of x; d values
   Requires a finished run (nss_run or nss_finalise).  out: host array of n_out
   values (NSS_ERR_ARG if n_out differs from the kind's count or the kind does
   not fit the run's likelihood/prior).  Synchronises the context's stream. */
enum {
    NSS_GRAD_LIK_SIGMA = 0,
    NSS_GRAD_LIK_MU = 1,
    NSS_GRAD_PRIOR_LOG_PREC = 2,
    NSS_GRAD_GP_NOISE_SCALE = 3,
    NSS_MOMENT_MEAN = 4
};
nss_status nss_posterior_expectation(nss_ctx *ctx, int run, int kind, double *out, int n_out);

/* Reweighting a finished run to inverse temperature beta (Eq. eq:marginal,
   Z(beta) = sum_i L_i^beta dX_i, from the same dead points; App. D.2):
     out[0] = log Z(beta), the mean over the R simulated volume trajectories,
     out[1] = its standard deviation (ddof 1),
     out[2] = the Kish effective sample size (sum w)^2 / sum w^2 of the
              geometric-mean weights at beta.
   beta = 1 reproduces nss_run's logZ and logZ_err.  beta must be finite and
   > 0 (else NSS_ERR_ARG); a dead point with logL = -inf keeps weight 0.  Runs
   the context's own volume simulation (its R trajectories, any number of
   dead points) on beta * logL with per-call scratch; the run's stored
   weights and results are unchanged.  Synchronises the context's stream. */
nss_status nss_reweight(nss_ctx *ctx, int run, double beta, double *out);

/* Volume simulation without allocation.  The paper has no counterpart: this
   is a library convenience for callers that must not allocate device memory
   when they need it, e.g. a service whose framework allocator owns and caches
   the device memory, or latency-bound code that forbids cudaMalloc/cudaFree
   (which synchronise the device) after start-up.  It computes what
   nss_run/nss_finalise compute after the last iteration -- logZ mean and
   standard deviation over n_sim simulated volume trajectories and the
   normalised log posterior weights -- for a dead-point list the caller already
   holds, and allocates nothing: its partial sums live in one fixed 2 MiB
   __device__ array that every GPU loading this library keeps until the
   process exits.
     logL [n], nlive [n]      device inputs (death order, as nss_get_dead gives)
     log_w [n]                device output
     logZ_stats [2]           device output: logZ mean, logZ standard deviation
     seed, run_id             the run's Philox key, as in nss_options
     cuda_stream              stream for the work (NULL = legacy default stream)
   Limits: 1 <= n <= 524288 dead points, 2 <= n_sim <= 128; larger sizes
   return NSS_ERR_ARG.  Every call looks up the array's device address
   (cudaGetSymbolAddress) on the current device; the first call on a device
   also loads the array's module there, so make it before any stream
   capture.  Every call shares the array and leaves its contents
   behind; calls whose work overlaps on the GPU race on it, so order them.
   Returns after enqueueing (no synchronisation). */
nss_status nss_volume_sim_static(const float *logL, const int *nlive, long long n, int n_sim,
                                 uint64_t seed, uint32_t run_id, double *log_w, double *logZ_stats,
                                 void *cuda_stream);

int nss_n_runs(const nss_ctx *ctx);
/* Slice width actually used by a run (after the width rule). */
double nss_run_width(const nss_ctx *ctx, int run);
void nss_destroy(nss_ctx *ctx);
const char *nss_status_string(nss_status s);
const char *nss_last_error(const nss_ctx *ctx);
int nss_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NSS_GB300_H */
