// nss_internal.h -- device-side layout of a Nested Slice Sampling context.
//
// A context holds R independent runs.  Their data live in three pools (FP32,
// INT32, FP64) addressed by per-run offsets, so one launch of each kernel
// serves every run.  Live points are stored point-major, x[slot][dpad] with
// dpad = d rounded up to a multiple of 4, so that a chain group loads its
// parent and stores its result with aligned float4 accesses.
#pragma once
#include <cstdint>

namespace nss {

constexpr int kMaxD = 128;          // largest dimension of the sweep kernels
constexpr int kMaxLive = 4096;      // largest m of the in-block selection sort
constexpr int kStepOutCap = 10;     // stepping-out expansions per side (App. B.4)
constexpr int kShrinkCap = 100;     // shrinkage proposals before a null move (App. B.4)
constexpr uint32_t kTagParent = 0xFFFFFFF0u;
constexpr uint32_t kTagInit = 0xFFFFFFF1u;
constexpr uint32_t kTagVolsim = 0xFFFFFFF2u;
constexpr int kPrologueThreads = 1024;  // one block per run; fixed, so every context reduces in the same order
constexpr int kNumCfgs = 25;
constexpr int kLaneCfg0 = 22;       // configurations 22..24 run one chain per lane
constexpr int kStepWords = 12;      // a step's scalar words drawn ahead: U, height, reserved, shrink 0..8
constexpr int kVolTile = 1024;      // dead points per volume-simulation tile

enum PriorKind { kPriorBox = 0, kPriorGauss = 1 };
enum KernelKind { kKernelHrss = 0, kKernelRw = 1 };
enum LikKind { kLikGauss = 0, kLikGmm = 1, kLikLogreg = 2, kLikGp = 3, kLikFlat = 4, kLikFault = 5, kLikRastrigin = 6 };

struct RunDesc {
  int d, dpad, m, k, p, m2;         // m2: power of two >= m for the sort
  int prior_kind, lik_kind, n_comp, n_data;
  int dir_norm, cfg;                // cfg: sweep configuration (G lanes x DPL dims)
  int fault_mode, max_iter;
  int kernel;                       // kKernelHrss / kKernelRw
  float ras_la, ras_l1a;            // Rastrigin mixture: ln alpha, ln(1 - alpha)
  float rw_scale;                   // RW proposal scale s (x + s L z)
  float w, cov_eps, fault_param;
  float inv2s2, lognorm;            // Gaussian / mixture constants
  float prior_const;                // Gaussian prior: sum(-log b - log(2 pi)/2)
  double tol;
  uint32_t key0, key1;
  // FP32 pool offsets
  long long o_x, o_logL, o_birth;   // live set
  long long o_dx, o_dlogL, o_dbirth;// dead store
  long long o_a, o_b, o_mu;         // prior bounds [dpad], means [n_comp][dpad]
  long long o_L;                    // metric factor [dpad][dpad]
  long long o_V;                    // directions of the iteration [k][p][dpad]
  // INT32 pool offsets
  long long o_dn;                   // dead store live counts
  long long o_dead, o_parent;       // [k] each
  long long o_stats;                // [6][k] evals, accepts, nulls, expansions, shrinks, cap_out
  long long o_wd;                   // [k][p][kStepWords] words nz .. nz+11 of each step's counter stream
  long long o_surv;                 // [m] survivors in slot order (plain single-run path)
  // FP64 pool offsets
  long long o_cum, o_lnd;           // [m+1]: sum_{j'<j} 1/(m-j'); [m]: log(-expm1(-1/(m-j)))
  long long o_lw;                   // [dead_cap] log posterior weights
  long long dead_cap;
};

struct RunState {
  double logZ, logX;
  long long n_dead, evals, nulls, cap_out, nan_evals;
  long long spec_evals;             // slice tests run beyond the logical ones (group-parallel rounds)
  long long rounds, active_rounds;  // slice-test rounds of the chain groups' warps, and those each group took part in
  int iter, done, status, metric_status;
  float logLstar;
  int stepped;                      // at least one iteration since create/import
  int finalised;
  int pad_;
  double logZ_mean, logZ_std, lw_norm;
};

struct WorkItem {                   // one warp's worth of chains of one run
  int run, c0, c1, pad_;
};

struct Dev {
  const RunDesc* desc;
  RunState* st;
  float* f;
  int* i;
  double* dd;
};

}  // namespace nss
