// nss_kernels.h -- host-side launchers of the Nested Slice Sampling kernels.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nss_internal.h"

namespace nss {

struct VolLaunch {
  const int2* tiles;
  const int* vbase;
  int n_tiles, R;
  double *tsum, *toff, *tmax, *tacc;
  // reweighting: run >= 0 simulates that run alone, reading logL_in and
  // writing its log weights to lw_out and (logZ mean, std, norm) to
  // stats_out; run = -1 serves every run from and into its own store
  int run = -1;
  const float* logL_in = nullptr;
  double* lw_out = nullptr;
  double* stats_out = nullptr;
};

// Device workspace of one logistic-regression run (line-affine logits).
struct LRArgs {
  const uint32_t* ybits;   // [512] label bits, bit i of word t = y[t + 512 i]
  float* zx;               // [cols_pad][ldz] logits X x of each chain's point
  float* zv;               // [cols_pad][ldz] logits X v of each chain's direction
  long long ldz;
  float* xc;               // [cols_pad][128] chain positions
  float* vdir;             // [cols_pad][128] chain directions
  float* lc;               // [cols_pad] chain logL
  __nv_bfloat16* parts;    // [3][cols_pad][128] bf16 split of the vectors being multiplied
  long long part_stride;   // cols_pad * 128
  const __nv_bfloat16* Xb; // [rows_pad][128] design matrix
  float* center;           // [128] centre mu of the contraction (live-set mean)
  float* zref;             // [rows_pad] X mu
};

// Per-chain state of the plain path's logistic HRSS step (direct evaluation:
// every slice test's logits recomputed from the candidate point).
struct LRDirect {
  float tl, tr, t;       // bracket ends and the candidate under test
  float height;          // prior slice height (Gaussian prior)
  int phase;             // 0 stepping out left, 1 right, 2 shrinking, 3 done
  int e, r;              // expansions of the current side; shrinkage proposal index
  int evals, exps, shr, capo, nanc, acc;
};

// Device data of one GP run: inputs and targets (FP32).
struct GPArgs {
  const float* t;
  const float* y;
};
cudaError_t setup_gp_attributes();
cudaError_t setup_gp_tc_attributes();
// the GP sweep with the tensor-core factorisation (nss_gp_tc.cu): chains of
// run `run` over min(k, num_sms) blocks; *err set when a tensor-core wait ran out
cudaError_t launch_gp_sweep_tc(const Dev& D, const GPArgs& A, int run, int k, int n, int num_sms, int* err,
                               cudaStream_t s);
// logL of m points theta [m][3] by the tensor-core factorisation alone
cudaError_t launch_gp_loglik_tc(const float* t, const float* y, int n, const float* theta, int m, float* out,
                                int num_sms, int* err, cudaStream_t s);
cudaError_t launch_gp_init(const Dev& D, const GPArgs& A, int run, int m, int n, cudaStream_t s);

// Posterior expectations over a finished run's dead points (nss_post.cu).
enum { kPostLikSigma = 0, kPostLikMu = 1, kPostPriorLogPrec = 2, kPostGpNoise = 3, kPostMean = 4 };
struct PostArgs {
  const float* x;      // dead points [n][ld]
  const double* lw;    // normalised log weights [n]
  long long n;
  int d, ld, kind, K;
  const float* mu;     // [K][ld] (likelihood kinds)
  const float* pa;     // prior a (mean) [d]
  const float* pb;     // prior b (sd) [d]
  double sigma;
};
// pass 1 + 2; coef: [n] or [n][K] FP64 scratch; out: device, 1 / d / K*d values
cudaError_t launch_post(const PostArgs& A, double* coef, double* out, cudaStream_t s);
cudaError_t launch_post_sum(const double* coef, long long n, double* out, cudaStream_t s);
cudaError_t launch_scale_logL(const float* logL, float beta, long long n, float* out, cudaStream_t s);
cudaError_t launch_sq_weights(const double* lw, long long n, double* out, cudaStream_t s);
// GP noise-scale term sigma_n^2 (|K^-1 y|^2 - tr K^-1) times the weight, for
// the dead points idx[0..n_idx) of run `run`, into coef[idx[j]] (others untouched)
cudaError_t launch_gp_noise_grad(const Dev& D, const GPArgs& A, int run, const int* idx, int n_idx, int n,
                                 double* coef, cudaStream_t s);

// one-time function attributes (dynamic shared memory above 48 KB)
cudaError_t setup_kernel_attributes();
cudaError_t setup_logits_attributes();

bool make_map_bf16(CUtensorMap* map, void* base, unsigned long long rows);
cudaError_t launch_logits(const CUtensorMap& mapX, const CUtensorMap& mapU, int rows_pad, int cols_pad, float* out,
                          long long ldo, int n_rows, int n_cols, int* err, const int* skip, const float* zref,
                          cudaStream_t s);
cudaError_t launch_lr_center(const Dev& D, const LRArgs& A, int run, int n_data, cudaStream_t s);
cudaError_t launch_lr_parents(const Dev& D, const LRArgs& A, int run, int k, cudaStream_t s);
cudaError_t launch_lr_live_parts(const Dev& D, const LRArgs& A, int run, int m, cudaStream_t s);
cudaError_t launch_lr_rowll(const Dev& D, const LRArgs& A, int run, int m, int emax, cudaStream_t s);
cudaError_t launch_lr_dir(const Dev& D, const LRArgs& A, int run, int k, int step, cudaStream_t s);
cudaError_t launch_lr_slice(const Dev& D, const LRArgs& A, int run, int k, int step, int emax, cudaStream_t s);
cudaError_t launch_lr_replace(const Dev& D, const LRArgs& A, int run, int k, cudaStream_t s);
// the plain path's logistic HRSS step s in lockstep evaluation rounds: init
// (bracket, slice height), then per round the candidate points' bf16 parts,
// the logits GEMM over them (launch_logits into A.zx) and the evaluation with
// each chain's transition; *active counts the chains still testing
cudaError_t launch_lr_direct_init(const Dev& D, const LRArgs& A, LRDirect* st, int run, int k, int step,
                                  cudaStream_t s);
cudaError_t launch_lr_direct_cand(const Dev& D, const LRArgs& A, const LRDirect* st, int run, int k, cudaStream_t s);
cudaError_t launch_lr_direct_eval(const Dev& D, const LRArgs& A, LRDirect* st, int run, int k, int step, int emax,
                                  int* active, cudaStream_t s);
// bounded-wait self-test: *out = 2 when the wait gave up (the expected outcome)
cudaError_t launch_wait_selftest(int* out, uint32_t max_polls, cudaStream_t s);

cudaError_t launch_init(int cfg, const Dev& D, const WorkItem* items, int n, cudaStream_t s);
// runs [run0, run0 + n_runs)
cudaError_t launch_prologue(const Dev& D, int run0, int n_runs, size_t smem, cudaStream_t s);
// the sweep of configuration cfg for runs of mixture bound kc = sweep_kc(.)
cudaError_t launch_sweep(int cfg, int kc, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                         cudaStream_t s);
int sweep_kc(int lik_kind, int n_comp);
cudaError_t launch_terminate(const Dev& D, int run0, int n_runs, cudaStream_t s);
// the plain single-run path (nss_plain.cu and its phase kernels): phase 0
// selection, 1 dead append + evidence, 2 metric, 3 parents of run `run`
cudaError_t launch_plain_phase(int phase, const Dev& D, int run, int k, size_t smem, cudaStream_t s);
// HRSS step s of every chain of run `run`, one thread per chain (k <= 1024),
// lockstep evaluation rounds; arithmetic of sweep configuration (G, DPL)
cudaError_t launch_plain_hrss(const Dev& D, int run, int k, int s, int G, int DPL, cudaStream_t st);
cudaError_t launch_final_sort(const Dev& D, int n_runs, size_t smem, cudaStream_t s);
cudaError_t launch_volsim(const Dev& D, const VolLaunch& V, int n_runs, cudaStream_t s);
int sweep_blocks_per_sm(int cfg, int kc);
// directions V[chain][step] of every generic-sweep chain of the iteration;
// items hold up to 32 chains each, dclass = dirgen_class(d) of their runs
int dirgen_class(int d);
cudaError_t setup_dirgen_attributes();
cudaError_t launch_dirgen(int dclass, const Dev& D, const WorkItem* items, int n, int max_p, cudaStream_t s);
// the same directions with the whitening product on the tensor cores
// (nss_dirgen_tc.cu): items {run, q0, q1} are tiles of at most 128 rows
// q = chain * p + step of one run, kc = 1 for 16 < d <= 32, 2 for d <= 64;
// *err set when a tensor-core wait ran out
cudaError_t setup_dirgen_tc_attributes();
int dirgen_tc_blocks_per_sm(int kc);
cudaError_t launch_dirgen_tc(int kc, const Dev& D, const WorkItem* items, int n, int grid, int* err, cudaStream_t s);
cudaError_t launch_sweep_lane(int dmax, int kc, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                              cudaStream_t s);
int sweep_lane_blocks_per_sm(int dmax, int kc);
int sweep_lane_warps_per_block();
int sweep_warps_per_block(int cfg);
int cfg_g(int cfg);
int cfg_dpl(int cfg);

}  // namespace nss
