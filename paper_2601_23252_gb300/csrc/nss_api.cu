// nss_api.cu -- the C ABI of include/nss.h: context creation, the host loop of
// outer iterations, finalisation, state import/export and traces.
//
// The host never touches sampler arithmetic: it validates arguments, lays out
// the per-run pools, uploads the problem, enqueues kernels on the context's
// stream and copies results out.  The only host-side numerics are constants
// of the problem (likelihood normalisations, the unrolled live-count tables
// of App. D.1 and the slice-width rule of App. E), computed once at create.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nss.h"
#include "nss_internal.h"
#include "nss_kernels.h"

using nss::RunDesc;
using nss::RunState;
using nss::WorkItem;

struct EvRec {
  cudaEvent_t a, b;
  int kind, cfg;
};

struct LRWork {
  int run = -1;
  int rows_pad = 0, cols_pad = 0, emax = 0;
  __nv_bfloat16* Xb = nullptr;
  uint32_t* ybits = nullptr;
  float *zx = nullptr, *zv = nullptr, *xc = nullptr, *vdir = nullptr, *lc = nullptr;
  __nv_bfloat16* parts = nullptr;
  float *center = nullptr, *zref = nullptr;
  int* err = nullptr;
  CUtensorMap mapX, mapU;
  nss::LRArgs args;
  // the plain path's direct evaluation: per-chain step state, the count of
  // chains still testing (device, and its pinned host mirror)
  nss::LRDirect* lrd = nullptr;
  int* d_active = nullptr;
  int* h_active = nullptr;
};

struct GPWork {
  int run = -1;
  float *t = nullptr, *y = nullptr;
  nss::GPArgs args;
};

struct nss_ctx {
  int n_runs = 0;
  std::vector<GPWork> gp;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<LRWork> lr;
  // captured chunks of outer iterations (one graph per chunk length and
  // profiling flag); with profiling on, the graph carries its own event
  // record nodes, read back after each replay
  struct ChunkGraph {
    int n = 0;
    bool prof = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<EvRec> evs;
    long long launches = 0;
  };
  std::vector<ChunkGraph> graphs;
  std::vector<int> replayed;          // graphs replayed since the last harvest
  bool capturing = false;
  std::vector<EvRec> cap_evs;
  int device = 0, num_sms = 1;
  std::vector<RunDesc> desc;
  std::vector<double> widths;
  std::vector<double> sigmas;       // likelihood width of Gaussian / mixture runs
  std::vector<uint32_t> run_ids;
  RunDesc* d_desc = nullptr;
  RunState* d_state = nullptr;
  RunState* h_state = nullptr;  // pinned mirror
  float* fpool = nullptr;
  int* ipool = nullptr;
  double* dpool = nullptr;
  long long nf = 0, ni = 0, nd = 0;
  // sweep work lists, one per (configuration, mixture bound): list q * 3 + b
  // holds the chains of configuration q whose runs have mixture bound kKC[b]
  static constexpr int kKC[3] = {1, 4, 8};
  static constexpr int kLists = nss::kNumCfgs * 3;
  // run groups: contiguous ranges of runs, each iterated on a stream of its
  // own, so the latency-bound sweep of one group overlaps the direction
  // draws and prologue of another.  Group g holds runs [g_r0[g], g_r0[g+1]);
  // its sweep lists are g * kLists + list, its direction lists
  // g * kDirClasses + class.
  static constexpr int kMaxGroups = 2;
  int n_groups = 1;
  int g_r0[kMaxGroups + 1] = {};
  cudaStream_t gstream[kMaxGroups] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kMaxGroups] = {};
  cudaStream_t cur = nullptr;  // stream of the launches being enqueued
  // Inside one group's iteration, the directions and sweeps of each
  // dimension class (8 << ci) run as their own chain of launches: class ci
  // on the group's stream (the first class in use) or on one of its side
  // streams, forked after the prologue and joined before the termination
  // test, so the latency-bound sweeps of different classes overlap.  With
  // profiling on every launch stays on the group's stream.
  static constexpr int kSide = 4;  // one per dimension class beyond the first
  cudaStream_t side[kMaxGroups][kSide] = {};
  cudaEvent_t side_fork[kMaxGroups] = {}, side_join[kMaxGroups][kSide] = {};
  std::vector<WorkItem> init_items[nss::kNumCfgs], sweep_items[kMaxGroups * kLists];
  WorkItem* d_init[nss::kNumCfgs] = {};
  WorkItem* d_sweep[kMaxGroups * kLists] = {};
  int* d_queue = nullptr;
  int sweep_grid[kMaxGroups * kLists] = {};
  // direction generation: items of up to 32 chains, per dimension class 8..128
  static constexpr int kDirClasses = 5;
  static_assert(kSide == kDirClasses - 1, "one side stream per dimension class beyond the first");
  std::vector<WorkItem> dir_items[kMaxGroups * kDirClasses];
  WorkItem* d_dir[kMaxGroups * kDirClasses] = {};
  // ... and on the tensor cores (nss_dirgen_tc.cu): tiles of 128 steps of one
  // run, list g * 2 + (KC - 1) for 16 < d <= 32 (KC = 1) and 32 < d <= 64 (KC = 2)
  bool dir_fp32 = false;  // NSS options dir_fp32: every direction on the CUDA cores
  std::vector<WorkItem> dir_tc_items[kMaxGroups * 2];
  WorkItem* d_dir_tc[kMaxGroups * 2] = {};
  int dir_tc_grid[2] = {1, 1};
  size_t prologue_smem = 0, final_smem = 0;
  // volume simulation scratch
  int R = 100;
  int vol_cap_tiles = 0;
  double* d_vol = nullptr;
  int2* d_tiles = nullptr;
  int* d_vbase = nullptr;
  // profiling
  bool profiling = false;
  std::vector<EvRec> pending;
  std::vector<cudaEvent_t> ev_pool;
  nss_profile prof{};
  double cfg_ms[nss::kNumCfgs] = {};
  double tune_cost[nss::kNumCfgs] = {};
  int max_p = 1;   // last autotune: device ms per 1e6 evaluations
  long long launches = 0;
  bool plain = false;   // the plain single-run path (NSS_PATH_PLAIN)
  // set by a tensor-core kernel whose bounded wait ran out; read at every sync
  int* d_tc_err = nullptr;
  int* h_tc_err = nullptr;
  bool broken = false;
  std::string err;
};

namespace {

long long align16(long long n) { return (n + 15) & ~15LL; }

nss_status set_err(nss_ctx* c, nss_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

nss_status cuda_fail(nss_ctx* c, cudaError_t e, const char* where) {
  if (c) c->broken = true;
  return set_err(c, e == cudaErrorMemoryAllocation ? NSS_ERR_OOM : NSS_ERR_CUDA, "%s: %s", where,
                 cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

nss::Dev dev_of(nss_ctx* c) {
  nss::Dev D;
  D.desc = c->d_desc;
  D.st = c->d_state;
  D.f = c->fpool;
  D.i = c->ipool;
  D.dd = c->dpool;
  return D;
}

// Sweep configurations able to hold d dimensions with the least padding:
// G lanes x DPL dimensions = the smallest power of two >= max(d, 4).
std::vector<int> candidate_cfgs(int d) {
  int cap = 4;
  while (cap < d) cap <<= 1;
  std::vector<int> out;
  for (int q = 0; q < nss::kNumCfgs; ++q)
    if (nss::cfg_g(q) * nss::cfg_dpl(q) == cap) out.push_back(q);
  return out;
}

// Dimension class index ci (directions of d <= 8 << ci) of the runs a sweep
// configuration serves: its capacity G x DPL (a power of two >= max(4, d)),
// at least 8.
int sweep_class(int cfg) {
  const int cap = std::max(8, nss::cfg_g(cfg) * nss::cfg_dpl(cfg));
  int ci = 0;
  while ((8 << ci) < cap) ++ci;
  return ci;
}

// Before tuning: the widest chain group (fewest chains per warp, least
// divergence between chains of a warp).
int default_cfg(int d) {
  int best = -1;
  for (int q : candidate_cfgs(d))
    if (best < 0 || nss::cfg_g(q) > nss::cfg_g(best)) best = q;
  return best;
}

// ---- slice-width rule helpers (App. E), host FP64 -------------------------
// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-15) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// integral of f over [a, b] by `panels` panels of an n-point rule
template <class F>
double integrate(F f, double a, double b, int panels, const std::vector<double>& gx,
                 const std::vector<double>& gw) {
  double s = 0.0, h = (b - a) / panels;
  for (int p = 0; p < panels; ++p) {
    const double c = a + (p + 0.5) * h;
    for (size_t i = 0; i < gx.size(); ++i) s += gw[i] * f(c + 0.5 * h * gx[i]);
  }
  return s * 0.5 * h;
}

// kappa_inf = 1/2 + E[R ln(1 + kappa/R)], R = q / E[q], q ~ chi_3 (the
// square root of the Gamma(3/2, 2) variable of the ellipsoid theorem).
double kappa_inf_host() {
  std::vector<double> gx, gw;
  gauss_legendre(20, gx, gw);
  const double c = 2.0 * std::sqrt(2.0 / M_PI);
  auto dens = [](double q) { return std::sqrt(2.0 / M_PI) * q * q * std::exp(-0.5 * q * q); };
  double k = 1.0;
  for (int it = 0; it < 500; ++it) {
    auto f = [&](double q) { return q <= 0 ? 0.0 : (q / c) * std::log1p(k * c / q) * dens(q); };
    const double nk = 0.5 + integrate(f, 0.0, 14.0, 200, gx, gw);
    if (std::fabs(nk - k) < 1e-14) return nk;
    k = nk;
  }
  return k;
}

// mean chord of a uniform point in a d-ball of radius Rb along a uniform
// direction, with rho = (r/Rb)^d uniform and theta weighted by sin^(d-2).
double mean_chord_host(int d, double Rb) {
  if (d == 1) return 2.0 * Rb;
  std::vector<double> gx, gw;
  gauss_legendre(16, gx, gw);
  auto wt = [&](double th) { return d == 2 ? 1.0 : std::pow(std::sin(th), d - 2); };
  const double norm = integrate(wt, 0.0, M_PI, 200, gx, gw);
  auto inner = [&](double th) {
    const double s2 = std::sin(th) * std::sin(th);
    auto g = [&](double rho) {
      const double v = 1.0 - std::pow(rho, 2.0 / d) * s2;
      return 2.0 * Rb * std::sqrt(v > 0 ? v : 0.0);
    };
    return wt(th) * integrate(g, 0.0, 1.0, 100, gx, gw);
  };
  return integrate(inner, 0.0, M_PI, 200, gx, gw) / norm;
}

nss_status validate(nss_ctx* c, const nss_prior& pr, const nss_loglik& lk, int m, int k, int p,
                    const nss_options& o, int run) {
  if (pr.d < 1 || pr.d > nss::kMaxD) return set_err(c, NSS_ERR_ARG, "run %d: d=%d outside [1,%d]", run, pr.d, nss::kMaxD);
  if (m < 2 || m > nss::kMaxLive) return set_err(c, NSS_ERR_ARG, "run %d: n_live=%d outside [2,%d]", run, m, nss::kMaxLive);
  if (k < 1 || k >= m) return set_err(c, NSS_ERR_ARG, "run %d: k=%d outside [1,n_live)", run, k);
  if (p < 1) return set_err(c, NSS_ERR_ARG, "run %d: p=%d < 1", run, p);
  if (!pr.a || !pr.b) return set_err(c, NSS_ERR_ARG, "run %d: prior bounds missing", run);
  if (pr.kind != NSS_PRIOR_UNIFORM_BOX && pr.kind != NSS_PRIOR_GAUSS_DIAG)
    return set_err(c, NSS_ERR_ARG, "run %d: unknown prior kind %d", run, pr.kind);
  for (int i = 0; i < pr.d; ++i) {
    if (!std::isfinite(pr.a[i]) || !std::isfinite(pr.b[i]))
      return set_err(c, NSS_ERR_ARG, "run %d: non-finite prior bound", run);
    if (pr.kind == NSS_PRIOR_UNIFORM_BOX && !(pr.a[i] < pr.b[i]))
      return set_err(c, NSS_ERR_ARG, "run %d: empty box in dimension %d", run, i);
    if (pr.kind == NSS_PRIOR_GAUSS_DIAG && !(pr.b[i] > 0))
      return set_err(c, NSS_ERR_ARG, "run %d: prior sd <= 0 in dimension %d", run, i);
  }
  switch (lk.kind) {
    case NSS_LOGLIK_GAUSS_ISO:
    case NSS_LOGLIK_TEST_FAULT:
      if (!lk.mu || !(lk.sigma > 0)) return set_err(c, NSS_ERR_ARG, "run %d: Gaussian needs mu and sigma > 0", run);
      if (lk.kind == NSS_LOGLIK_TEST_FAULT && lk.fault_mode != 1 && lk.fault_mode != 2)
        return set_err(c, NSS_ERR_ARG, "run %d: fault_mode must be 1 or 2", run);
      break;
    case NSS_LOGLIK_GMM_ISO_EQUAL:
      if (!lk.mu || !(lk.sigma > 0) || lk.n_comp < 1 || lk.n_comp > 8)
        return set_err(c, NSS_ERR_ARG, "run %d: mixture needs mu, sigma > 0, 1 <= n_comp <= 8", run);
      break;
    case NSS_LOGLIK_FLAT:
      break;
    case NSS_LOGLIK_RASTRIGIN:
      if (!(lk.alpha >= 0.0 && lk.alpha <= 1.0)) return set_err(c, NSS_ERR_ARG, "run %d: Rastrigin alpha outside [0,1]", run);
      break;
    case NSS_LOGLIK_LOGREG:
      if (!lk.X || !lk.y || lk.n_data < 1 || lk.n_data > 20 * 512)
        return set_err(c, NSS_ERR_ARG, "run %d: logistic regression needs X, y and 1 <= n_data <= 10240", run);
      if (pr.kind != NSS_PRIOR_GAUSS_DIAG)
        return set_err(c, NSS_ERR_ARG, "run %d: logistic regression takes the Gaussian prior", run);
      break;
    case NSS_LOGLIK_GP_RBF_WHITE:
      if (!lk.gp_t || !lk.gp_y || lk.n_data < 1 || lk.n_data > 256)
        return set_err(c, NSS_ERR_ARG, "run %d: GP needs gp_t, gp_y and 1 <= n_data <= 256", run);
      if (pr.d != 3 || pr.kind != NSS_PRIOR_UNIFORM_BOX)
        return set_err(c, NSS_ERR_ARG, "run %d: GP hyperparameters are 3 log-parameters under a box prior", run);
      break;
    default:
      return set_err(c, NSS_ERR_ARG, "run %d: unknown likelihood kind %d", run, lk.kind);
  }
  if (!(o.tol > 0 && o.tol < 1)) return set_err(c, NSS_ERR_ARG, "run %d: tol outside (0,1)", run);
  if (o.max_iter < 1) return set_err(c, NSS_ERR_ARG, "run %d: max_iter < 1", run);
  if (o.w_rule == NSS_W_FIXED && !(o.w > 0)) return set_err(c, NSS_ERR_ARG, "run %d: w <= 0", run);
  if (o.w_rule != NSS_W_FIXED && o.w_rule != NSS_W_THEORY) return set_err(c, NSS_ERR_ARG, "run %d: unknown w_rule", run);
  if (o.dir_norm != NSS_DIR_MAHAL && o.dir_norm != NSS_DIR_EUCLID) return set_err(c, NSS_ERR_ARG, "run %d: unknown dir_norm", run);
  if (o.n_sim < 2 || o.n_sim > 1024) return set_err(c, NSS_ERR_ARG, "run %d: n_sim outside [2,1024]", run);
  if (!(o.cov_eps >= 0)) return set_err(c, NSS_ERR_ARG, "run %d: cov_eps < 0", run);
  if (o.dead_capacity < 0) return set_err(c, NSS_ERR_ARG, "run %d: dead_capacity < 0", run);
  if (o.kernel != NSS_KERNEL_HRSS && o.kernel != NSS_KERNEL_RW) return set_err(c, NSS_ERR_ARG, "run %d: unknown kernel", run);
  if (o.kernel == NSS_KERNEL_RW) {
    if (!(o.rw_scale >= 0) || !std::isfinite(o.rw_scale)) return set_err(c, NSS_ERR_ARG, "run %d: rw_scale < 0", run);
    if (lk.kind == NSS_LOGLIK_LOGREG || lk.kind == NSS_LOGLIK_GP_RBF_WHITE)
      return set_err(c, NSS_ERR_ARG, "run %d: the random-walk kernel takes Gaussian, mixture or flat likelihoods", run);
  }
  if (o.path != NSS_PATH_BATCHED && o.path != NSS_PATH_PLAIN) return set_err(c, NSS_ERR_ARG, "run %d: unknown path", run);
  if (o.run_groups != 0 && o.run_groups != 1) return set_err(c, NSS_ERR_ARG, "run %d: run_groups must be 0 or 1", run);
  if (o.path == NSS_PATH_PLAIN) {
    if (o.kernel != NSS_KERNEL_HRSS) return set_err(c, NSS_ERR_ARG, "run %d: the plain path runs the HRSS kernel", run);
    if (lk.kind != NSS_LOGLIK_GAUSS_ISO && lk.kind != NSS_LOGLIK_GMM_ISO_EQUAL && lk.kind != NSS_LOGLIK_FLAT &&
        lk.kind != NSS_LOGLIK_LOGREG)
      return set_err(c, NSS_ERR_ARG, "run %d: the plain path takes Gaussian, mixture, flat or logistic likelihoods",
                     run);
    if (k > 1024) return set_err(c, NSS_ERR_ARG, "run %d: the plain path takes k <= 1024", run);
    if (o.sweep_cfg >= nss::kLaneCfg0) return set_err(c, NSS_ERR_ARG, "run %d: the plain path takes a grouped sweep configuration", run);
  }
  if (o.sweep_cfg >= 0) {
    bool fits = false;
    for (int q : candidate_cfgs(pr.d)) fits |= (q == o.sweep_cfg);
    if (!fits) return set_err(c, NSS_ERR_ARG, "run %d: sweep_cfg %d does not fit d=%d", run, o.sweep_cfg, pr.d);
  }
  return NSS_OK;
}

void free_ctx(nss_ctx* c) {
  if (!c) return;
  cudaFree(c->d_desc);
  cudaFree(c->d_state);
  if (c->h_state) cudaFreeHost(c->h_state);
  cudaFree(c->fpool);
  cudaFree(c->ipool);
  cudaFree(c->dpool);
  for (int q = 0; q < nss::kNumCfgs; ++q) cudaFree(c->d_init[q]);
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kLists; ++q) cudaFree(c->d_sweep[q]);
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kDirClasses; ++q) cudaFree(c->d_dir[q]);
  for (int q = 0; q < nss_ctx::kMaxGroups * 2; ++q) cudaFree(c->d_dir_tc[q]);
  for (int g = 0; g < nss_ctx::kMaxGroups; ++g) {
    if (c->gstream[g]) cudaStreamDestroy(c->gstream[g]);
    if (c->join_ev[g]) cudaEventDestroy(c->join_ev[g]);
    if (c->side_fork[g]) cudaEventDestroy(c->side_fork[g]);
    for (int k = 0; k < nss_ctx::kSide; ++k) {
      if (c->side[g][k]) cudaStreamDestroy(c->side[g][k]);
      if (c->side_join[g][k]) cudaEventDestroy(c->side_join[g][k]);
    }
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  cudaFree(c->d_queue);
  cudaFree(c->d_vol);
  cudaFree(c->d_tiles);
  cudaFree(c->d_vbase);
  for (auto& e : c->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto& w : c->lr) {
    cudaFree(w.Xb);
    cudaFree(w.ybits);
    cudaFree(w.lrd);
    cudaFree(w.d_active);
    if (w.h_active) cudaFreeHost(w.h_active);
    cudaFree(w.zx);
    cudaFree(w.zv);
    cudaFree(w.xc);
    cudaFree(w.vdir);
    cudaFree(w.lc);
    cudaFree(w.parts);
    cudaFree(w.center);
    cudaFree(w.zref);
    cudaFree(w.err);
  }
  for (auto& g : c->gp) {
    cudaFree(g.t);
    cudaFree(g.y);
  }
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& e : g.evs) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// ---- profiling: an event pair around each launch while enabled -------------
cudaEvent_t take_event(nss_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct Rec {
  nss_ctx* c;
  int kind, cfg;
  cudaEvent_t a = nullptr;
  Rec(nss_ctx* c_, int k_, int cfg_ = -1) : c(c_), kind(k_), cfg(cfg_) {
    c->launches++;
    c->prof.total_launches++;
    c->prof.launches[kind]++;
    if (c->profiling) {
      a = take_event(c);
      if (c->capturing) cudaEventRecordWithFlags(a, c->cur, cudaEventRecordExternal);
      else cudaEventRecord(a, c->cur);
    }
  }
  ~Rec() {
    if (a) {
      cudaEvent_t b = take_event(c);
      if (c->capturing) {
        cudaEventRecordWithFlags(b, c->cur, cudaEventRecordExternal);
        c->cap_evs.push_back({a, b, kind, cfg});
      } else {
        cudaEventRecord(b, c->cur);
        c->pending.push_back({a, b, kind, cfg});
      }
    }
  }
};

void harvest(nss_ctx* c) {  // after a stream synchronisation
  for (int gi : c->replayed) {
    for (auto& e : c->graphs[gi].evs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
        c->prof.ms[e.kind] += ms;
        if (e.cfg >= 0) c->cfg_ms[e.cfg] += ms;
      }
    }
  }
  c->replayed.clear();
  for (auto& e : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      c->prof.ms[e.kind] += ms;
      if (e.cfg >= 0) c->cfg_ms[e.cfg] += ms;
    }
    c->ev_pool.push_back(e.a);
    c->ev_pool.push_back(e.b);
  }
  c->pending.clear();
}

nss_status sync_state(nss_ctx* c) {
  CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(RunState) * c->n_runs, cudaMemcpyDeviceToHost,
                     c->stream), "state readback");
  CK(cudaMemcpyAsync(c->h_tc_err, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag readback");
  c->prof.d2h_bytes += (long long)sizeof(RunState) * c->n_runs + (long long)sizeof(int);
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  harvest(c);
  if (*c->h_tc_err) {
    c->broken = true;
    return set_err(c, NSS_ERR_CUDA, "a tensor-core kernel's bounded wait ran out (code %d)", *c->h_tc_err);
  }
  return NSS_OK;
}

// One outer iteration of the runs of group g, enqueued on c->cur.
nss_status enqueue_iteration(nss_ctx* c, int g = 0) {
  nss::Dev D = dev_of(c);
  const int r0 = c->g_r0[g], nr = c->g_r0[g + 1] - r0;
  cudaStream_t st = c->cur;
  {
    Rec r(c, NSS_K_PROLOGUE);
    CK(nss::launch_prologue(D, r0, nr, c->prologue_smem, st), "prologue launch");
  }
  // per dimension class: directions (CUDA cores, or tensor cores for the
  // classes 32 and 64), then the sweeps of the configurations of that class
  cudaStream_t cs[nss_ctx::kDirClasses] = {};
  bool used[nss_ctx::kDirClasses] = {};
  for (int ci = 0; ci < nss_ctx::kDirClasses; ++ci) {
    used[ci] = !c->dir_items[g * nss_ctx::kDirClasses + ci].empty() ||
               ((ci == 2 || ci == 3) && !c->dir_tc_items[g * 2 + ci - 2].empty());
    for (int q = 0; q < nss_ctx::kLists && !used[ci]; ++q)
      used[ci] = !c->sweep_items[g * nss_ctx::kLists + q].empty() && sweep_class(q / 3) == ci;
  }
  int nside = 0;
  bool first = true;
  for (int ci = 0; ci < nss_ctx::kDirClasses; ++ci) {
    if (!used[ci]) continue;
    if (first || c->profiling) {
      cs[ci] = st;
      first = false;
    } else {
      cs[ci] = c->side[g][nside++];
    }
  }
  if (nside > 0) {
    CK(cudaEventRecord(c->side_fork[g], st), "class fork");
    for (int k = 0; k < nside; ++k) CK(cudaStreamWaitEvent(c->side[g][k], c->side_fork[g], 0), "class fork");
  }
  for (int ci = 0; ci < nss_ctx::kDirClasses; ++ci) {
    if (!used[ci]) continue;
    c->cur = cs[ci];
    const int L = g * nss_ctx::kDirClasses + ci;
    if (!c->dir_items[L].empty()) {
      Rec rd(c, NSS_K_DIRGEN);
      CK(nss::launch_dirgen(8 << ci, D, c->d_dir[L], (int)c->dir_items[L].size(), c->max_p, c->cur),
         "direction launch");
    }
    if (ci == 2 || ci == 3) {
      const int kc = ci - 1, T = g * 2 + kc - 1;
      if (!c->dir_tc_items[T].empty()) {
        Rec rd(c, NSS_K_DIRGEN);
        CK(nss::launch_dirgen_tc(kc, D, c->d_dir_tc[T], (int)c->dir_tc_items[T].size(), c->dir_tc_grid[kc - 1],
                                 c->d_tc_err, c->cur), "tensor-core direction launch");
      }
    }
    for (int q = 0; q < nss_ctx::kLists; ++q) {
      const int LS = g * nss_ctx::kLists + q;
      if (c->sweep_items[LS].empty() || sweep_class(q / 3) != ci) continue;
      CK(cudaMemsetAsync(c->d_queue + LS, 0, sizeof(int), c->cur), "queue reset");
      Rec r(c, NSS_K_SWEEP, q / 3);
      CK(nss::launch_sweep(q / 3, nss_ctx::kKC[q % 3], D, c->d_sweep[LS], (int)c->sweep_items[LS].size(),
                           c->d_queue + LS, c->sweep_grid[LS], c->cur), "sweep launch");
    }
  }
  c->cur = st;
  for (int k = 0; k < nside; ++k) {
    CK(cudaEventRecord(c->side_join[g][k], c->side[g][k]), "class join");
    CK(cudaStreamWaitEvent(st, c->side_join[g][k], 0), "class join");
  }
  if (g == 0) {  // logistic and GP runs keep one group
    for (auto& gw : c->gp) {
      const RunDesc& R = c->desc[gw.run];
      Rec r(c, NSS_K_GP_SWEEP);
      CK(nss::launch_gp_sweep_tc(D, gw.args, gw.run, R.k, R.n_data, c->num_sms, c->d_tc_err, st),
         "GP sweep launch");
    }
    for (auto& w : c->lr) {
      const RunDesc& R = c->desc[w.run];
      const int* done = &c->d_state[w.run].done;
      {
        Rec r(c, NSS_K_OTHER);
        CK(nss::launch_lr_center(D, w.args, w.run, R.n_data, st), "logistic centre launch");
      }
      {
        Rec r(c, NSS_K_OTHER);
        CK(nss::launch_lr_parents(D, w.args, w.run, R.k, st), "logistic parents launch");
      }
      {
        Rec r(c, NSS_K_LOGITS);
        CK(nss::launch_logits(w.mapX, w.mapU, w.rows_pad, w.cols_pad, w.zx, w.rows_pad, R.n_data, R.k, w.err, done,
                              w.zref, st), "logits launch");
      }
      for (int s = 0; s < R.p; ++s) {
        {
          Rec r(c, NSS_K_OTHER);
          CK(nss::launch_lr_dir(D, w.args, w.run, R.k, s, st), "logistic direction launch");
        }
        {
          Rec r(c, NSS_K_LOGITS);
          CK(nss::launch_logits(w.mapX, w.mapU, w.rows_pad, w.cols_pad, w.zv, w.rows_pad, R.n_data, R.k, w.err,
                                done, nullptr, st), "logits launch");
        }
        {
          Rec r(c, NSS_K_LR_SLICE);
          CK(nss::launch_lr_slice(D, w.args, w.run, R.k, s, w.emax, st), "logistic slice launch");
        }
      }
      {
        Rec r(c, NSS_K_OTHER);
        CK(nss::launch_lr_replace(D, w.args, w.run, R.k, st), "logistic replace launch");
      }
    }
  }
  {
    Rec r(c, NSS_K_TERMINATE);
    CK(nss::launch_terminate(D, r0, nr, st), "terminate launch");
  }
  return NSS_OK;
}

// The plain path's logistic HRSS steps: per step the directions, then
// lockstep evaluation rounds (candidate parts, one logits GEMM over all
// chains' candidates, evaluation and transition) until every chain has
// finished the step; the host reads the count of chains still testing after
// each round.
nss_status enqueue_plain_logreg_steps(nss_ctx* c, LRWork& w) {
  nss::Dev D = dev_of(c);
  const RunDesc& R = c->desc[w.run];
  cudaStream_t st = c->stream;
  const int* done = &c->d_state[w.run].done;
  {
    Rec r(c, NSS_K_OTHER);
    CK(nss::launch_lr_center(D, w.args, w.run, R.n_data, st), "logistic centre launch");
  }
  {
    Rec r(c, NSS_K_OTHER);
    CK(nss::launch_lr_parents(D, w.args, w.run, R.k, st), "logistic parents launch");
  }
  const int max_rounds = 2 * nss::kStepOutCap + nss::kShrinkCap + 2;
  for (int s = 0; s < R.p; ++s) {
    {
      Rec r(c, NSS_K_OTHER);
      CK(nss::launch_lr_dir(D, w.args, w.run, R.k, s, st), "logistic direction launch");
    }
    {
      Rec r(c, NSS_K_OTHER);
      CK(nss::launch_lr_direct_init(D, w.args, w.lrd, w.run, R.k, s, st), "logistic step start launch");
    }
    for (int round = 0; round < max_rounds; ++round) {
      CK(cudaMemsetAsync(w.d_active, 0, sizeof(int), st), "round counter reset");
      {
        Rec r(c, NSS_K_OTHER);
        CK(nss::launch_lr_direct_cand(D, w.args, w.lrd, w.run, R.k, st), "logistic candidate launch");
      }
      {
        Rec r(c, NSS_K_LOGITS);
        CK(nss::launch_logits(w.mapX, w.mapU, w.rows_pad, w.cols_pad, w.zx, w.rows_pad, R.n_data, R.k, w.err, done,
                              w.zref, st), "logits launch");
      }
      {
        Rec r(c, NSS_K_LR_SLICE);
        CK(nss::launch_lr_direct_eval(D, w.args, w.lrd, w.run, R.k, s, w.emax, w.d_active, st),
           "logistic evaluation launch");
      }
      CK(cudaMemcpyAsync(w.h_active, w.d_active, sizeof(int), cudaMemcpyDeviceToHost, st), "round counter read");
      CK(cudaStreamSynchronize(st), "round synchronise");
      c->prof.d2h_bytes += (long long)sizeof(int);
      if (*w.h_active == 0) break;
    }
  }
  {
    Rec r(c, NSS_K_OTHER);
    CK(nss::launch_lr_replace(D, w.args, w.run, R.k, st), "logistic replace launch");
  }
  return NSS_OK;
}

// One outer iteration of the plain single-run path (NSS_PATH_PLAIN): one
// launch per phase, one HRSS launch per step, on c->stream.
nss_status enqueue_plain_iteration(nss_ctx* c) {
  nss::Dev D = dev_of(c);
  const RunDesc& R = c->desc[0];
  cudaStream_t st = c->stream;
  for (int ph = 0; ph < 4; ++ph) {
    Rec r(c, NSS_K_PROLOGUE);
    CK(nss::launch_plain_phase(ph, D, 0, R.k, c->prologue_smem, st), "plain phase launch");
  }
  if (!c->lr.empty()) {
    nss_status s = enqueue_plain_logreg_steps(c, c->lr[0]);
    if (s != NSS_OK) return s;
    Rec r(c, NSS_K_TERMINATE);
    CK(nss::launch_terminate(D, 0, 1, st), "terminate launch");
    return NSS_OK;
  }
  for (int q = 0; q < nss_ctx::kDirClasses; ++q) {
    if (c->dir_items[q].empty()) continue;
    Rec rd(c, NSS_K_DIRGEN);
    CK(nss::launch_dirgen(8 << q, D, c->d_dir[q], (int)c->dir_items[q].size(), c->max_p, st), "direction launch");
  }
  for (int kc = 1; kc <= 2; ++kc) {
    if (c->dir_tc_items[kc - 1].empty()) continue;
    Rec rd(c, NSS_K_DIRGEN);
    CK(nss::launch_dirgen_tc(kc, D, c->d_dir_tc[kc - 1], (int)c->dir_tc_items[kc - 1].size(),
                             c->dir_tc_grid[kc - 1], c->d_tc_err, st), "tensor-core direction launch");
  }
  const int G = nss::cfg_g(R.cfg), DPL = nss::cfg_dpl(R.cfg);
  for (int s = 0; s < R.p; ++s) {
    Rec r(c, NSS_K_SWEEP, R.cfg);
    CK(nss::launch_plain_hrss(D, 0, R.k, s, G, DPL, st), "plain HRSS launch");
  }
  {
    Rec r(c, NSS_K_TERMINATE);
    CK(nss::launch_terminate(D, 0, 1, st), "terminate launch");
  }
  return NSS_OK;
}

// n outer iterations of every group.  With one group they go on c->stream;
// with several, each group's iterations go on its own stream between a fork
// and a join on c->stream, so the groups run ahead of one another freely.
nss_status enqueue_iterations(nss_ctx* c, int n) {
  if (c->n_groups == 1) {
    c->cur = c->stream;
    for (int i = 0; i < n; ++i) {
      nss_status st = enqueue_iteration(c, 0);
      if (st != NSS_OK) return st;
    }
    return NSS_OK;
  }
  CK(cudaEventRecord(c->fork_ev, c->stream), "fork");
  for (int g = 0; g < c->n_groups; ++g) CK(cudaStreamWaitEvent(c->gstream[g], c->fork_ev, 0), "fork");
  for (int i = 0; i < n; ++i)
    for (int g = 0; g < c->n_groups; ++g) {
      c->cur = c->gstream[g];
      nss_status st = enqueue_iteration(c, g);
      if (st != NSS_OK) {
        c->cur = c->stream;
        return st;
      }
    }
  c->cur = c->stream;
  for (int g = 0; g < c->n_groups; ++g) {
    CK(cudaEventRecord(c->join_ev[g], c->gstream[g]), "join");
    CK(cudaStreamWaitEvent(c->stream, c->join_ev[g], 0), "join");
  }
  return NSS_OK;
}

void drop_graphs(nss_ctx* c) {  // the captured chunks refer to the work lists
  if (!c->graphs.empty()) cudaStreamSynchronize(c->stream);
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& e : g.evs) {
      c->ev_pool.push_back(e.a);
      c->ev_pool.push_back(e.b);
    }
  }
  c->graphs.clear();
  c->replayed.clear();
}

// n outer iterations, replayed from a captured CUDA graph of the whole chunk
// (every group's launches, forks and joins; a run that is done skips its
// kernels on the device).  Captured on first use for each chunk length and
// profiling flag.  The autotuner enqueues launch by launch instead.
nss_status run_iteration(nss_ctx* c, int n = 1) {
  int gi = -1;
  for (int q = 0; q < (int)c->graphs.size(); ++q)
    if (c->graphs[q].n == n && c->graphs[q].prof == c->profiling) gi = q;
  if (gi < 0) {
    nss_ctx::ChunkGraph g;
    g.n = n;
    g.prof = c->profiling;
    const long long l0 = c->launches, t0 = c->prof.total_launches;
    long long k0[NSS_PROFILE_KINDS];
    std::memcpy(k0, c->prof.launches, sizeof k0);
    c->cap_evs.clear();
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    c->capturing = true;
    nss_status st = enqueue_iterations(c, n);
    c->capturing = false;
    cudaGraph_t cg = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &cg);
    if (st != NSS_OK) {
      if (cg) cudaGraphDestroy(cg);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture end");
    e = cudaGraphInstantiate(&g.exec, cg, 0);
    cudaGraphDestroy(cg);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    g.launches = c->launches - l0;
    g.evs.swap(c->cap_evs);
    c->launches = l0;
    c->prof.total_launches = t0;
    std::memcpy(c->prof.launches, k0, sizeof k0);
    c->graphs.push_back(std::move(g));
    gi = (int)c->graphs.size() - 1;
  }
  // one replay per harvest keeps every launch's event pair readable
  if (c->profiling && std::find(c->replayed.begin(), c->replayed.end(), gi) != c->replayed.end()) {
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    harvest(c);
  }
  CK(cudaGraphLaunch(c->graphs[gi].exec, c->stream), "graph launch");
  c->launches += c->graphs[gi].launches;
  c->prof.total_launches += c->graphs[gi].launches;
  for (const auto& e : c->graphs[gi].evs) c->prof.launches[e.kind]++;
  if (c->profiling) c->replayed.push_back(gi);
  return NSS_OK;
}

// Work lists of the init and sweep kernels: 32/G slots or chains of one run
// per warp, grouped by sweep configuration, costliest runs first.
nss_status build_work(nss_ctx* c) {
  drop_graphs(c);
  for (int q = 0; q < nss::kNumCfgs; ++q) {
    c->init_items[q].clear();
    cudaFree(c->d_init[q]);
    c->d_init[q] = nullptr;
  }
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kLists; ++q) {
    c->sweep_items[q].clear();
    cudaFree(c->d_sweep[q]);
    c->d_sweep[q] = nullptr;
  }
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kDirClasses; ++q) {
    c->dir_items[q].clear();
    cudaFree(c->d_dir[q]);
    c->d_dir[q] = nullptr;
  }
  for (int q = 0; q < nss_ctx::kMaxGroups * 2; ++q) {
    c->dir_tc_items[q].clear();
    cudaFree(c->d_dir_tc[q]);
    c->d_dir_tc[q] = nullptr;
  }
  for (int r = 0; r < c->n_runs; ++r) {
    const RunDesc& R = c->desc[r];
    const int per = 32 / nss::cfg_g(R.cfg);
    // the prior draw always runs in a grouped configuration
    const int icfg = nss::cfg_dpl(R.cfg) > 4 ? default_cfg(R.d) : R.cfg;
    const int iper = 32 / nss::cfg_g(icfg);
    for (int s = 0; s < R.m; s += iper) c->init_items[icfg].push_back({r, s, std::min(s + iper, R.m), 0});
    if (R.lik_kind == nss::kLikLogreg || R.lik_kind == nss::kLikGp) continue;  // own sweep kernels
    int g = 0;
    while (r >= c->g_r0[g + 1]) ++g;
    const int kc = nss::sweep_kc(R.lik_kind, R.n_comp);
    const int list = g * nss_ctx::kLists + R.cfg * 3 + (kc == 1 ? 0 : kc == 4 ? 1 : 2);
    for (int j = 0; j < R.k; j += per) c->sweep_items[list].push_back({r, j, std::min(j + per, R.k), 0});
    int dq = 0;
    while ((8 << dq) < nss::dirgen_class(R.d)) ++dq;
    if (!c->dir_fp32 && R.d > 16 && R.d <= 64) {
      // tiles of 128 rows q = chain * p + step
      const int kc = R.d <= 32 ? 1 : 2;
      const int rows = R.k * R.p;
      for (int q0 = 0; q0 < rows; q0 += 128)
        c->dir_tc_items[g * 2 + kc - 1].push_back({r, q0, std::min(q0 + 128, rows), 0});
      continue;
    }
    for (int j = 0; j < R.k; j += 32)
      c->dir_items[g * nss_ctx::kDirClasses + dq].push_back({r, j, std::min(j + 32, R.k), 0});
  }
  for (int q = 0; q < nss_ctx::kMaxGroups * 2; ++q) {
    if (c->dir_tc_items[q].empty()) continue;
    CK(cudaMalloc(&c->d_dir_tc[q], sizeof(WorkItem) * c->dir_tc_items[q].size()), "work list allocation");
    CK(cudaMemcpyAsync(c->d_dir_tc[q], c->dir_tc_items[q].data(), sizeof(WorkItem) * c->dir_tc_items[q].size(),
                       cudaMemcpyHostToDevice, c->stream), "work list upload");
  }
  for (int kc = 1; kc <= 2; ++kc) c->dir_tc_grid[kc - 1] = nss::dirgen_tc_blocks_per_sm(kc) * c->num_sms;
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kDirClasses; ++q) {
    if (c->dir_items[q].empty()) continue;
    CK(cudaMalloc(&c->d_dir[q], sizeof(WorkItem) * c->dir_items[q].size()), "work list allocation");
    CK(cudaMemcpyAsync(c->d_dir[q], c->dir_items[q].data(), sizeof(WorkItem) * c->dir_items[q].size(),
                       cudaMemcpyHostToDevice, c->stream), "work list upload");
  }
  for (int q = 0; q < nss::kNumCfgs; ++q) {
    if (!c->init_items[q].empty()) {
      CK(cudaMalloc(&c->d_init[q], sizeof(WorkItem) * c->init_items[q].size()), "work list allocation");
      CK(cudaMemcpyAsync(c->d_init[q], c->init_items[q].data(), sizeof(WorkItem) * c->init_items[q].size(),
                         cudaMemcpyHostToDevice, c->stream), "work list upload");
    }
  }
  for (int q = 0; q < nss_ctx::kMaxGroups * nss_ctx::kLists; ++q) {
    auto cost = [&](const WorkItem& w) { return (double)c->desc[w.run].p * c->desc[w.run].d; };
    std::stable_sort(c->sweep_items[q].begin(), c->sweep_items[q].end(),
                     [&](const WorkItem& a, const WorkItem& b) { return cost(a) > cost(b); });
    if (!c->sweep_items[q].empty()) {
      CK(cudaMalloc(&c->d_sweep[q], sizeof(WorkItem) * c->sweep_items[q].size()), "work list allocation");
      CK(cudaMemcpyAsync(c->d_sweep[q], c->sweep_items[q].data(), sizeof(WorkItem) * c->sweep_items[q].size(),
                         cudaMemcpyHostToDevice, c->stream), "work list upload");
      const int ql = q % nss_ctx::kLists;
      const int per_sm = nss::sweep_blocks_per_sm(ql / 3, nss_ctx::kKC[ql % 3]);
      const int wpb = nss::sweep_warps_per_block(ql / 3);
      const int warps_needed = (int)c->sweep_items[q].size();
      const int blocks_needed = (warps_needed + wpb - 1) / wpb;
      c->sweep_grid[q] = std::max(1, std::min(blocks_needed, per_sm * c->num_sms));
    }
  }
  CK(cudaMemcpyAsync(c->d_desc, c->desc.data(), sizeof(RunDesc) * c->n_runs, cudaMemcpyHostToDevice, c->stream),
     "descriptor upload");
  CK(cudaStreamSynchronize(c->stream), "work list upload");
  return NSS_OK;
}

nss_status gp_initial_loglik(nss_ctx* c, GPWork& g) {
  const RunDesc& R = c->desc[g.run];
  Rec rr(c, NSS_K_INIT);
  CK(nss::launch_gp_init(dev_of(c), g.args, g.run, R.m, R.n_data, c->stream), "GP init launch");
  return NSS_OK;
}

nss_status setup_gp(nss_ctx* c, int run, const nss_loglik& lk) {
  const RunDesc& R = c->desc[run];
  std::vector<float> t(R.n_data), y(R.n_data);
  for (int i = 0; i < R.n_data; ++i) {
    t[i] = (float)lk.gp_t[i];
    y[i] = (float)lk.gp_y[i];
  }
  GPWork g;
  g.run = run;
  CK(cudaMalloc(&g.t, sizeof(float) * R.n_data), "GP data");
  CK(cudaMalloc(&g.y, sizeof(float) * R.n_data), "GP data");
  c->gp.push_back(g);
  GPWork& G = c->gp.back();
  CK(cudaMemcpyAsync(G.t, t.data(), sizeof(float) * R.n_data, cudaMemcpyHostToDevice, c->stream), "GP data upload");
  CK(cudaMemcpyAsync(G.y, y.data(), sizeof(float) * R.n_data, cudaMemcpyHostToDevice, c->stream), "GP data upload");
  CK(cudaStreamSynchronize(c->stream), "GP data upload");
  c->prof.h2d_bytes += (long long)(2 * sizeof(float) * R.n_data);
  G.args.t = G.t;
  G.args.y = G.y;
  return gp_initial_loglik(c, G);
}

// logL of the m initial live points of a logistic run: split, contract, reduce.
nss_status lr_initial_loglik(nss_ctx* c, LRWork& w) {
  const RunDesc& R = c->desc[w.run];
  nss::Dev D = dev_of(c);
  Rec rr(c, NSS_K_INIT);
  CK(nss::launch_lr_center(D, w.args, w.run, R.n_data, c->stream), "logistic centre launch");
  CK(nss::launch_lr_live_parts(D, w.args, w.run, R.m, c->stream), "logistic live split launch");
  CK(nss::launch_logits(w.mapX, w.mapU, w.rows_pad, w.cols_pad, w.zx, w.rows_pad, R.n_data, R.m, w.err, nullptr,
                        w.zref, c->stream), "logits launch");
  CK(nss::launch_lr_rowll(D, w.args, w.run, R.m, w.emax, c->stream), "logistic row likelihood launch");
  return NSS_OK;
}

// Workspace of a logistic-regression run: bf16 design matrix [rows_pad][128],
// label bits in the slice kernel's thread layout, logits of chain points and
// directions, the bf16 split buffer, and the TMA descriptors.
nss_status setup_logreg(nss_ctx* c, int run, const nss_loglik& lk) {
  const RunDesc& R = c->desc[run];
  LRWork w;
  w.run = run;
  w.rows_pad = (R.n_data + 127) / 128 * 128;
  w.cols_pad = (std::max(R.m, R.k) + 127) / 128 * 128;
  w.emax = (R.n_data + 511) / 512 <= 4 ? 4 : 20;
  std::vector<__nv_bfloat16> xb((size_t)w.rows_pad * 128, __float2bfloat16_rn(0.0f));
  for (int n = 0; n < R.n_data; ++n)
    for (int i = 0; i < R.d; ++i) xb[(size_t)n * 128 + i] = __float2bfloat16_rn(lk.X[(size_t)n * R.d + i]);
  std::vector<uint32_t> yb(512, 0u);
  for (int n = 0; n < R.n_data; ++n)
    if (lk.y[n] > 0.5f) yb[n % 512] |= 1u << (n / 512);
  const size_t zsz = sizeof(float) * (size_t)w.cols_pad * w.rows_pad;
  CK(cudaMalloc(&w.Xb, sizeof(__nv_bfloat16) * xb.size()), "logistic workspace");
  CK(cudaMalloc(&w.ybits, sizeof(uint32_t) * 512), "logistic workspace");
  CK(cudaMalloc(&w.zx, zsz), "logistic workspace");
  CK(cudaMalloc(&w.zv, zsz), "logistic workspace");
  CK(cudaMalloc(&w.xc, sizeof(float) * w.cols_pad * 128), "logistic workspace");
  CK(cudaMalloc(&w.vdir, sizeof(float) * w.cols_pad * 128), "logistic workspace");
  CK(cudaMalloc(&w.lc, sizeof(float) * w.cols_pad), "logistic workspace");
  CK(cudaMalloc(&w.parts, sizeof(__nv_bfloat16) * 3 * (size_t)w.cols_pad * 128), "logistic workspace");
  CK(cudaMalloc(&w.err, sizeof(int)), "logistic workspace");
  CK(cudaMalloc(&w.center, sizeof(float) * 128), "logistic workspace");
  if (c->plain) {
    CK(cudaMalloc(&w.lrd, sizeof(nss::LRDirect) * w.cols_pad), "logistic workspace");
    CK(cudaMalloc(&w.d_active, sizeof(int)), "logistic workspace");
    CK(cudaMallocHost(&w.h_active, sizeof(int)), "logistic workspace");
  }
  CK(cudaMalloc(&w.zref, sizeof(float) * w.rows_pad), "logistic workspace");
  c->lr.push_back(w);  // owned by the context from here on (freed with it)
  LRWork& W = c->lr.back();
  CK(cudaMemcpyAsync(W.Xb, xb.data(), sizeof(__nv_bfloat16) * xb.size(), cudaMemcpyHostToDevice, c->stream),
     "design upload");
  CK(cudaMemcpyAsync(W.ybits, yb.data(), sizeof(uint32_t) * 512, cudaMemcpyHostToDevice, c->stream), "label upload");
  c->prof.h2d_bytes += (long long)(sizeof(__nv_bfloat16) * xb.size() + sizeof(uint32_t) * 512);
  CK(cudaMemsetAsync(W.zx, 0, zsz, c->stream), "workspace clear");
  CK(cudaMemsetAsync(W.zv, 0, zsz, c->stream), "workspace clear");
  CK(cudaMemsetAsync(W.parts, 0, sizeof(__nv_bfloat16) * 3 * (size_t)W.cols_pad * 128, c->stream), "workspace clear");
  CK(cudaMemsetAsync(W.xc, 0, sizeof(float) * W.cols_pad * 128, c->stream), "workspace clear");
  CK(cudaMemsetAsync(W.vdir, 0, sizeof(float) * W.cols_pad * 128, c->stream), "workspace clear");
  CK(cudaMemsetAsync(W.err, 0, sizeof(int), c->stream), "workspace clear");
  if (!nss::make_map_bf16(&W.mapX, W.Xb, (unsigned long long)W.rows_pad) ||
      !nss::make_map_bf16(&W.mapU, W.parts, 3ULL * W.cols_pad))
    return set_err(c, NSS_ERR_CUDA, "run %d: tensor map encoding failed", run);
  W.args.ybits = W.ybits;
  W.args.zx = W.zx;
  W.args.zv = W.zv;
  W.args.ldz = W.rows_pad;
  W.args.xc = W.xc;
  W.args.vdir = W.vdir;
  W.args.lc = W.lc;
  W.args.parts = W.parts;
  W.args.part_stride = (long long)W.cols_pad * 128;
  W.args.Xb = W.Xb;
  W.args.center = W.center;
  W.args.zref = W.zref;
  return lr_initial_loglik(c, W);
}

void clear_states(nss_ctx* c) {
  for (int r = 0; r < c->n_runs; ++r) {
    RunState& s = c->h_state[r];
    std::memset(&s, 0, sizeof s);
    s.logZ = -INFINITY;
    s.logX = 0.0;
    s.logLstar = -INFINITY;
  }
}

nss_status launch_inits(nss_ctx* c) {
  nss::Dev D = dev_of(c);
  for (int q = 0; q < nss::kNumCfgs; ++q) {
    if (c->init_items[q].empty()) continue;
    Rec rr(c, NSS_K_INIT);
    CK(nss::launch_init(q, D, c->d_init[q], (int)c->init_items[q].size(), c->stream), "init launch");
  }
  return NSS_OK;
}

bool all_done(const nss_ctx* c) {
  for (int r = 0; r < c->n_runs; ++r)
    if (!c->h_state[r].done) return false;
  return true;
}

void fill_info(const nss_ctx* c, nss_step_info* info) {
  if (!info) return;
  for (int r = 0; r < c->n_runs; ++r) {
    const RunState& s = c->h_state[r];
    nss_step_info& o = info[r];
    o.iter = s.iter;
    o.done = s.done;
    o.logLstar = s.logLstar;
    o.logZ = s.logZ;
    o.logX = s.logX;
    o.n_dead = s.n_dead;
    o.evals = s.evals;
    o.nulls = s.nulls;
    o.cap_out = s.cap_out;
    o.nan_evals = s.nan_evals;
    o.spec_evals = s.spec_evals;
    o.group_rounds = s.rounds;
    o.active_group_rounds = s.active_rounds;
    o.metric_status = s.metric_status;
    o.status = s.status;
  }
}

nss_status finalise_impl(nss_ctx* c, nss_result* res) {
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (!all_done(c)) return set_err(c, NSS_ERR_STATE, "finalise before every run terminated");
  nss::Dev D = dev_of(c);
  {
    Rec r(c, NSS_K_FINAL_SORT);
    CK(nss::launch_final_sort(D, c->n_runs, c->final_smem, c->stream), "final sort launch");
  }
  if ((st = sync_state(c)) != NSS_OK) return st;
  // tiles of kVolTile dead points, runs contiguous
  std::vector<int2> tiles;
  std::vector<int> vbase(c->n_runs);
  for (int r = 0; r < c->n_runs; ++r) {
    vbase[r] = (int)tiles.size();
    const long long n = c->h_state[r].n_dead;
    for (long long i = 0; i < n; i += nss::kVolTile) tiles.push_back(make_int2(r, (int)i));
  }
  const int nt = (int)tiles.size();
  if (nt > 0) {
    if (nt > c->vol_cap_tiles) {
      cudaFree(c->d_vol);
      cudaFree(c->d_tiles);
      c->d_vol = nullptr;
      c->d_tiles = nullptr;
      const int cap = nt + nt / 4 + 16;
      CK(cudaMalloc(&c->d_vol, sizeof(double) * 4 * (size_t)c->R * cap), "volume scratch");
      CK(cudaMalloc(&c->d_tiles, sizeof(int2) * cap), "tile list");
      c->vol_cap_tiles = cap;
    }
    CK(cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int2) * nt, cudaMemcpyHostToDevice, c->stream), "tiles upload");
    c->prof.h2d_bytes += (long long)(sizeof(int2) * nt + sizeof(int) * c->n_runs);
    CK(cudaMemcpyAsync(c->d_vbase, vbase.data(), sizeof(int) * c->n_runs, cudaMemcpyHostToDevice, c->stream), "vbase upload");
    nss::VolLaunch V;
    V.tiles = c->d_tiles;
    V.vbase = c->d_vbase;
    V.n_tiles = nt;
    V.R = c->R;
    const size_t blk = (size_t)c->R * nt;
    V.tsum = c->d_vol;
    V.toff = c->d_vol + blk;
    V.tmax = c->d_vol + 2 * blk;
    V.tacc = c->d_vol + 3 * blk;
    Rec r(c, NSS_K_VOLSIM);
    CK(nss::launch_volsim(D, V, c->n_runs, c->stream), "volume simulation launch");
  }
  if ((st = sync_state(c)) != NSS_OK) return st;
  nss_status worst = NSS_OK;
  for (int r = 0; r < c->n_runs; ++r) {
    const RunState& s = c->h_state[r];
    if (res) {
      nss_result& o = res[r];
      o.logZ = s.logZ_mean;
      o.logZ_err = s.logZ_std;
      o.logZ_det = s.logZ;
      o.n_dead = s.n_dead;
      o.iters = s.iter;
      o.evals = s.evals;
      o.nulls = s.nulls;
      o.cap_out = s.cap_out;
      o.nan_evals = s.nan_evals;
      o.spec_evals = s.spec_evals;
      o.group_rounds = s.rounds;
      o.active_group_rounds = s.active_rounds;
      o.status = s.status;
    }
    if (s.status == NSS_ERR_CAPACITY) worst = NSS_ERR_CAPACITY;
    if (s.status == NSS_ERR_NUMERIC && worst == NSS_OK) worst = NSS_ERR_NUMERIC;
  }
  if (worst != NSS_OK) return set_err(c, worst, "a run ended with status %d", (int)worst);
  return NSS_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

void nss_options_default(nss_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->seed = 0;
  o->run_id = 0;
  o->w = 1.0;
  o->w_rule = NSS_W_FIXED;
  o->dir_norm = NSS_DIR_MAHAL;
  o->tol = 1e-3;
  o->max_iter = 100000;
  o->dead_capacity = 0;
  o->n_sim = 100;
  o->cov_eps = 1e-6;
  o->cuda_stream = nullptr;
  o->sweep_cfg = -1;
  o->kernel = NSS_KERNEL_HRSS;
  o->rw_scale = 0.0;
  o->path = NSS_PATH_BATCHED;
  o->run_groups = 0;
  o->dir_fp32 = 0;
}

int nss_abi_version(void) { return NSS_ABI_VERSION; }

const char* nss_status_string(nss_status s) {
  switch (s) {
    case NSS_OK: return "ok";
    case NSS_DONE: return "done";
    case NSS_ERR_ARG: return "invalid argument";
    case NSS_ERR_CUDA: return "CUDA error";
    case NSS_ERR_OOM: return "out of device memory";
    case NSS_ERR_CAPACITY: return "dead-point store full";
    case NSS_ERR_TIMEOUT: return "iteration cap reached";
    case NSS_ERR_NUMERIC: return "non-finite evidence";
    case NSS_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* nss_last_error(const nss_ctx* c) { return c ? c->err.c_str() : "no context"; }

int nss_n_runs(const nss_ctx* c) { return c ? c->n_runs : 0; }

nss_status nss_wait_selftest(unsigned max_polls, int* outcome) {
  if (!outcome || max_polls < 1 || max_polls > (1u << 20)) return NSS_ERR_ARG;
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) e = nss::launch_wait_selftest(d, max_polls, 0);
  if (e == cudaSuccess) e = cudaMemcpy(outcome, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? NSS_OK : NSS_ERR_CUDA;
}

nss_status nss_logreg_logits(const float* X, int n, int d, const float* U, int nu, float* Z) {
  if (!X || !U || !Z || d < 1 || d > 128 || n < 1 || n > (1 << 20) || nu < 1 || nu > (1 << 16)) return NSS_ERR_ARG;
  const int rows_pad = (n + 127) / 128 * 128, cols_pad = (nu + 127) / 128 * 128;
  std::vector<__nv_bfloat16> xb((size_t)rows_pad * 128, __float2bfloat16_rn(0.0f));
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < d; ++i) xb[(size_t)r * 128 + i] = __float2bfloat16_rn(X[(size_t)r * d + i]);
  // three-part split of U on the host, the same rounding as the device split
  std::vector<__nv_bfloat16> parts(3 * (size_t)cols_pad * 128, __float2bfloat16_rn(0.0f));
  const size_t ps = (size_t)cols_pad * 128;
  for (int j = 0; j < nu; ++j)
    for (int i = 0; i < d; ++i) {
      const float u = U[(size_t)j * d + i];
      const __nv_bfloat16 h = __float2bfloat16_rn(u);
      const float r1 = u - __bfloat162float(h);
      const __nv_bfloat16 m = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(m);
      parts[(size_t)j * 128 + i] = h;
      parts[ps + (size_t)j * 128 + i] = m;
      parts[2 * ps + (size_t)j * 128 + i] = __float2bfloat16_rn(r2);
    }
  __nv_bfloat16 *dX = nullptr, *dP = nullptr;
  float* dZ = nullptr;
  int* dErr = nullptr;
  nss_status st = NSS_OK;
  cudaError_t e = cudaMalloc(&dX, sizeof(__nv_bfloat16) * xb.size());
  if (e == cudaSuccess) e = cudaMalloc(&dP, sizeof(__nv_bfloat16) * parts.size());
  // the device copy of Z has rows of rows_pad floats (the TMA stores want 16-byte row strides)
  if (e == cudaSuccess) e = cudaMalloc(&dZ, sizeof(float) * (size_t)nu * rows_pad);
  if (e == cudaSuccess) e = cudaMalloc(&dErr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dX, xb.data(), sizeof(__nv_bfloat16) * xb.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dP, parts.data(), sizeof(__nv_bfloat16) * parts.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(int));
  if (e == cudaSuccess) e = nss::setup_logits_attributes();
  CUtensorMap mx, mu;
  if (e == cudaSuccess) {
    if (!nss::make_map_bf16(&mx, dX, (unsigned long long)rows_pad) ||
        !nss::make_map_bf16(&mu, dP, 3ULL * cols_pad)) st = NSS_ERR_CUDA;
  }
  if (e == cudaSuccess && st == NSS_OK)
    e = nss::launch_logits(mx, mu, rows_pad, cols_pad, dZ, rows_pad, n, nu, dErr, nullptr, nullptr, 0);
  if (e == cudaSuccess && st == NSS_OK) e = cudaDeviceSynchronize();
  int herr = 0;
  if (e == cudaSuccess && st == NSS_OK) e = cudaMemcpy(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st == NSS_OK)
    e = cudaMemcpy2D(Z, sizeof(float) * (size_t)n, dZ, sizeof(float) * (size_t)rows_pad, sizeof(float) * (size_t)n, nu,
                     cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = (e == cudaErrorMemoryAllocation) ? NSS_ERR_OOM : NSS_ERR_CUDA;
  if (st == NSS_OK && herr != 0) st = NSS_ERR_TIMEOUT;
  cudaFree(dX);
  cudaFree(dP);
  cudaFree(dZ);
  cudaFree(dErr);
  return st;
}

nss_status nss_gp_loglik(const double* t, const double* y, int n, const double* theta, int m, float* out) {
  if (!t || !y || !theta || !out || n < 1 || n > 256 || m < 1 || m > (1 << 20)) return NSS_ERR_ARG;
  std::vector<float> ht(n), hy(n), hth(3 * (size_t)m);
  for (int i = 0; i < n; ++i) {
    ht[i] = (float)t[i];
    hy[i] = (float)y[i];
  }
  for (size_t i = 0; i < hth.size(); ++i) hth[i] = (float)theta[i];
  float *dt = nullptr, *dy = nullptr, *dth = nullptr, *dout = nullptr;
  int* dErr = nullptr;
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&dt, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dth, sizeof(float) * hth.size());
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(float) * m);
  if (e == cudaSuccess) e = cudaMalloc(&dErr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dt, ht.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dy, hy.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dth, hth.data(), sizeof(float) * hth.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(int));
  if (e == cudaSuccess) e = nss::setup_gp_tc_attributes();
  if (e == cudaSuccess) e = nss::launch_gp_loglik_tc(dt, dy, n, dth, m, dout, sms, dErr, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(float) * m, cudaMemcpyDeviceToHost);
  nss_status st = NSS_OK;
  if (e != cudaSuccess) st = (e == cudaErrorMemoryAllocation) ? NSS_ERR_OOM : NSS_ERR_CUDA;
  if (st == NSS_OK && herr != 0) st = NSS_ERR_TIMEOUT;
  cudaFree(dt);
  cudaFree(dy);
  cudaFree(dth);
  cudaFree(dout);
  cudaFree(dErr);
  return st;
}

double nss_run_width(const nss_ctx* c, int run) {
  if (!c || run < 0 || run >= c->n_runs) return NAN;
  return c->widths[run];
}

nss_status nss_create_batch(int n_runs, const nss_prior* prior, const nss_loglik* loglik,
                            const int* n_live, const int* kk, const int* pp, const nss_options* opt,
                            nss_ctx** out) {
  if (!out) return NSS_ERR_ARG;
  *out = nullptr;
  if (n_runs < 1 || !prior || !loglik || !n_live || !kk || !pp || !opt) return NSS_ERR_ARG;
  nss_ctx* c = new nss_ctx();
  c->n_runs = n_runs;
  for (int r = 0; r < n_runs; ++r) {
    nss_status s = validate(c, prior[r], loglik[r], n_live[r], kk[r], pp[r], opt[r], r);
    if (s != NSS_OK) {
      std::string msg = c->err;
      delete c;
      std::fprintf(stderr, "nss_create: %s\n", msg.c_str());
      return s;
    }
  }
  c->R = opt[0].n_sim;
  for (int r = 1; r < n_runs; ++r)
    if (opt[r].n_sim != c->R || opt[r].path != opt[0].path || opt[r].run_groups != opt[0].run_groups ||
        opt[r].dir_fp32 != opt[0].dir_fp32) {
      delete c;
      return NSS_ERR_ARG;
    }
  c->plain = opt[0].path == NSS_PATH_PLAIN;
  c->dir_fp32 = opt[0].dir_fp32 != 0;
  if (c->plain && n_runs != 1) {
    delete c;
    std::fprintf(stderr, "nss_create: the plain path runs a single run\n");
    return NSS_ERR_ARG;
  }
  c->stream = static_cast<cudaStream_t>(opt[0].cuda_stream);
  if (!c->stream) {
    cudaError_t es = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (es != cudaSuccess) {
      nss_status s_ = cuda_fail(c, es, "stream creation");
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());
      delete c;
      return s_;
    }
    c->own_stream = true;
  }
  c->cur = c->stream;

  // ---- layout -------------------------------------------------------------
  c->desc.resize(n_runs);
  c->widths.resize(n_runs);
  c->sigmas.assign(n_runs, 0.0);
  c->run_ids.resize(n_runs);
  double kappa = -1.0;
  for (int r = 0; r < n_runs; ++r) {
    const nss_prior& pr = prior[r];
    const nss_loglik& lk = loglik[r];
    const nss_options& o = opt[r];
    RunDesc& R = c->desc[r];
    std::memset(&R, 0, sizeof R);
    R.d = pr.d;
    R.dpad = (pr.d + 3) & ~3;
    R.m = n_live[r];
    R.k = kk[r];
    R.p = pp[r];
    c->max_p = std::max(c->max_p, R.p);
    int m2 = 1;
    while (m2 < R.m) m2 <<= 1;
    R.m2 = m2;
    R.prior_kind = pr.kind;
    R.lik_kind = lk.kind;
    R.n_comp = (lk.kind == NSS_LOGLIK_GMM_ISO_EQUAL) ? lk.n_comp : 1;
    R.n_data = lk.n_data;
    R.dir_norm = o.dir_norm;
    R.cfg = default_cfg(R.d);
    for (int q : candidate_cfgs(R.d))
      if (q == o.sweep_cfg) R.cfg = q;
    R.fault_mode = lk.fault_mode;
    R.fault_param = (float)lk.fault_param;
    R.max_iter = o.max_iter;
    R.kernel = o.kernel;
    if (lk.kind == NSS_LOGLIK_RASTRIGIN) {
      // the Gaussian part exp(-|x|^2/2) through the line coefficients (mean 0, sigma 1)
      R.inv2s2 = 0.5f;
      R.lognorm = 0.0f;
      R.ras_la = lk.alpha > 0.0 ? (float)std::log(lk.alpha) : -INFINITY;
      R.ras_l1a = lk.alpha < 1.0 ? (float)std::log1p(-lk.alpha) : -INFINITY;
    }
    R.rw_scale = (float)(o.rw_scale > 0 ? o.rw_scale : 2.38 / std::sqrt((double)R.d));
    double w = o.w;
    if (o.w_rule == NSS_W_THEORY) {
      if (kappa < 0) kappa = kappa_inf_host();
      w = kappa * mean_chord_host(R.d, std::sqrt(R.d + 2.0));
    }
    c->widths[r] = (double)(float)w;
    R.w = (float)w;
    R.cov_eps = (float)o.cov_eps;
    R.tol = o.tol;
    R.key0 = (uint32_t)o.seed;
    R.key1 = (uint32_t)(o.seed >> 32) ^ o.run_id;
    c->run_ids[r] = o.run_id;
    if (lk.kind == NSS_LOGLIK_GAUSS_ISO || lk.kind == NSS_LOGLIK_GMM_ISO_EQUAL ||
        lk.kind == NSS_LOGLIK_TEST_FAULT) {
      const double s2 = lk.sigma * lk.sigma;
      c->sigmas[r] = lk.sigma;
      R.inv2s2 = (float)(1.0 / (2.0 * s2));
      R.lognorm = (float)(-0.5 * R.d * std::log(2.0 * M_PI * s2) - std::log((double)R.n_comp));
    }
    if (pr.kind == NSS_PRIOR_GAUSS_DIAG) {
      double pc = 0.0;
      for (int i = 0; i < R.d; ++i) pc += -std::log(pr.b[i]) - 0.5 * std::log(2.0 * M_PI);
      R.prior_const = (float)pc;
    }
    long long cap = o.dead_capacity > 0 ? o.dead_capacity : (long long)R.k * 2000 + R.m;
    cap = std::max(cap, (long long)R.m);
    R.dead_cap = cap;
    // FP32 pool
    R.o_x = c->nf; c->nf += align16((long long)R.m * R.dpad);
    R.o_logL = c->nf; c->nf += align16(R.m);
    R.o_birth = c->nf; c->nf += align16(R.m);
    R.o_dx = c->nf; c->nf += align16(cap * R.dpad);
    R.o_dlogL = c->nf; c->nf += align16(cap);
    R.o_dbirth = c->nf; c->nf += align16(cap);
    R.o_a = c->nf; c->nf += align16(R.dpad);
    R.o_b = c->nf; c->nf += align16(R.dpad);
    R.o_mu = c->nf; c->nf += align16((long long)R.n_comp * R.dpad);
    R.o_L = c->nf; c->nf += align16((long long)R.dpad * R.dpad);
    const bool own_sweep = lk.kind != NSS_LOGLIK_LOGREG && lk.kind != NSS_LOGLIK_GP_RBF_WHITE;
    R.o_V = c->nf; c->nf += own_sweep ? align16((long long)R.k * R.p * R.dpad) : 16;
    // INT32 pool
    R.o_dn = c->ni; c->ni += align16(cap);
    R.o_dead = c->ni; c->ni += align16(R.k);
    R.o_parent = c->ni; c->ni += align16(R.k);
    R.o_stats = c->ni; c->ni += align16(6LL * R.k);
    {
      const bool own = lk.kind != NSS_LOGLIK_LOGREG && lk.kind != NSS_LOGLIK_GP_RBF_WHITE;
      R.o_wd = c->ni; c->ni += own ? align16((long long)R.k * R.p * nss::kStepWords) : 16;
    }
    R.o_surv = c->ni; c->ni += align16(R.m);
    // FP64 pool
    R.o_cum = c->nd; c->nd += align16(R.m + 1);
    R.o_lnd = c->nd; c->nd += align16(R.m);
    R.o_lw = c->nd; c->nd += align16(cap);
    // shared memory of the prologue: sort keys + survivors/flags, or the
    // covariance reductions and the two d x d matrices
    const size_t sortb = (size_t)R.m2 * 8 + (size_t)R.m2 * 4 + (size_t)R.m * 4;
    const int nt = R.dpad / 4, ntp = nt * (nt + 1) / 2, parts2 = std::max(1, nss::kPrologueThreads / ntp);
    const size_t covb = sizeof(float) * ((size_t)parts2 * ntp * 16 + (size_t)R.dpad * (2 * R.dpad + 1));
    const size_t meanb = sizeof(float) * nss::kPrologueThreads;
    c->prologue_smem = std::max(c->prologue_smem, std::max(sortb, std::max(covb, meanb)));
    c->final_smem = std::max(c->final_smem, (size_t)R.m2 * 8);
  }
  // ---- device allocation and upload --------------------------------------
  cudaError_t e;
#define CKC(call, where)                                           \
  do {                                                             \
    e = (call);                                                    \
    if (e != cudaSuccess) {                                        \
      nss_status s_ = cuda_fail(c, e, where);                      \
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());    \
      free_ctx(c);                                                 \
      return s_;                                                   \
    }                                                              \
  } while (0)
  CKC(cudaGetDevice(&c->device), "cudaGetDevice");
  CKC(nss::setup_kernel_attributes(), "kernel attributes");
  CKC(nss::setup_logits_attributes(), "kernel attributes");
  CKC(nss::setup_gp_attributes(), "kernel attributes");
  CKC(nss::setup_gp_tc_attributes(), "kernel attributes");
  CKC(nss::setup_dirgen_attributes(), "kernel attributes");
  CKC(nss::setup_dirgen_tc_attributes(), "kernel attributes");
  CKC(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device), "device attribute");
  CKC(cudaMalloc(&c->d_desc, sizeof(RunDesc) * n_runs), "descriptor allocation");
  CKC(cudaMalloc(&c->d_state, sizeof(RunState) * n_runs), "state allocation");
  CKC(cudaMallocHost(&c->h_state, sizeof(RunState) * n_runs), "pinned state allocation");
  CKC(cudaMalloc(&c->fpool, sizeof(float) * std::max(c->nf, 16LL)), "FP32 pool allocation");
  CKC(cudaMalloc(&c->ipool, sizeof(int) * std::max(c->ni, 16LL)), "INT32 pool allocation");
  CKC(cudaMalloc(&c->dpool, sizeof(double) * std::max(c->nd, 16LL)), "FP64 pool allocation");
  CKC(cudaMalloc(&c->d_queue, sizeof(int) * nss_ctx::kMaxGroups * nss_ctx::kLists), "queue allocation");
  CKC(cudaMalloc(&c->d_vbase, sizeof(int) * n_runs), "vbase allocation");
  CKC(cudaMalloc(&c->d_tc_err, sizeof(int)), "flag allocation");
  CKC(cudaMallocHost(&c->h_tc_err, sizeof(int)), "flag allocation");
  CKC(cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream), "flag clear");
  *c->h_tc_err = 0;
  CKC(cudaMemsetAsync(c->fpool, 0, sizeof(float) * std::max(c->nf, 16LL), c->stream), "pool clear");
  CKC(cudaMemsetAsync(c->ipool, 0, sizeof(int) * std::max(c->ni, 16LL), c->stream), "pool clear");
  CKC(cudaMemsetAsync(c->dpool, 0, sizeof(double) * std::max(c->nd, 16LL), c->stream), "pool clear");
  // host staging of the problem constants
  {
    std::vector<float> hf;
    std::vector<double> hd;
    for (int r = 0; r < n_runs; ++r) {
      const RunDesc& R = c->desc[r];
      const nss_prior& pr = prior[r];
      const nss_loglik& lk = loglik[r];
      std::vector<float> seg((size_t)(R.o_L - R.o_a), 0.0f);
      for (int i = 0; i < R.d; ++i) {
        seg[i] = (float)pr.a[i];
        seg[(R.o_b - R.o_a) + i] = (float)pr.b[i];
      }
      const bool has_mu = lk.kind == NSS_LOGLIK_GAUSS_ISO || lk.kind == NSS_LOGLIK_GMM_ISO_EQUAL ||
                          lk.kind == NSS_LOGLIK_TEST_FAULT;
      if (has_mu)
        for (int q = 0; q < R.n_comp; ++q)
          for (int i = 0; i < R.d; ++i) seg[(R.o_mu - R.o_a) + (size_t)q * R.dpad + i] = (float)lk.mu[(size_t)q * R.d + i];
      CKC(cudaMemcpyAsync(c->fpool + R.o_a, seg.data(), sizeof(float) * seg.size(), cudaMemcpyHostToDevice,
                          c->stream), "problem upload");
      c->prof.h2d_bytes += (long long)(sizeof(float) * seg.size() + sizeof(double) * (2 * R.m + 1));
      // unrolled live-count tables (App. D.1)
      std::vector<double> cum(R.m + 1), lnd(R.m);
      double acc = 0.0;
      for (int j = 0; j < R.m; ++j) {
        cum[j] = acc;
        const double n = (double)(R.m - j);
        lnd[j] = std::log(-std::expm1(-1.0 / n));
        acc += 1.0 / n;
      }
      cum[R.m] = acc;
      CKC(cudaMemcpyAsync(c->dpool + R.o_cum, cum.data(), sizeof(double) * cum.size(), cudaMemcpyHostToDevice,
                          c->stream), "table upload");
      CKC(cudaMemcpyAsync(c->dpool + R.o_lnd, lnd.data(), sizeof(double) * lnd.size(), cudaMemcpyHostToDevice,
                          c->stream), "table upload");
    }
    (void)hf;
    (void)hd;
  }
  CKC(cudaMemcpyAsync(c->d_desc, c->desc.data(), sizeof(RunDesc) * n_runs, cudaMemcpyHostToDevice, c->stream),
      "descriptor upload");
  c->prof.h2d_bytes += (long long)(sizeof(RunDesc) + sizeof(RunState)) * n_runs;
  clear_states(c);
  CKC(cudaMemcpyAsync(c->d_state, c->h_state, sizeof(RunState) * n_runs, cudaMemcpyHostToDevice, c->stream),
      "state upload");
  // run groups: two streams when every run uses the generic sweep, split
  // into contiguous halves of about equal sweep cost
  {
    bool generic = n_runs >= 2 && !c->plain && opt[0].run_groups == 0;
    double total = 0.0;
    for (int r = 0; r < n_runs; ++r) {
      const RunDesc& R = c->desc[r];
      if (R.lik_kind == nss::kLikLogreg || R.lik_kind == nss::kLikGp) generic = false;
      total += (double)R.k * R.p * R.d;
    }
    c->g_r0[0] = 0;
    c->n_groups = 1;
    if (generic) {
      double acc = 0.0;
      int cut = 1;
      for (int r = 0; r < n_runs - 1; ++r) {
        acc += (double)c->desc[r].k * c->desc[r].p * c->desc[r].d;
        cut = r + 1;
        if (acc >= 0.5 * total) break;
      }
      c->g_r0[1] = cut;
      c->n_groups = 2;
      CKC(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming), "event creation");
      for (int g = 0; g < 2; ++g) {
        CKC(cudaStreamCreateWithFlags(&c->gstream[g], cudaStreamNonBlocking), "stream creation");
        CKC(cudaEventCreateWithFlags(&c->join_ev[g], cudaEventDisableTiming), "event creation");
      }
    }
    c->g_r0[c->n_groups] = n_runs;
    for (int g = 0; g < c->n_groups; ++g) {
      CKC(cudaEventCreateWithFlags(&c->side_fork[g], cudaEventDisableTiming), "event creation");
      for (int k = 0; k < nss_ctx::kSide; ++k) {
        CKC(cudaStreamCreateWithFlags(&c->side[g][k], cudaStreamNonBlocking), "stream creation");
        CKC(cudaEventCreateWithFlags(&c->side_join[g][k], cudaEventDisableTiming), "event creation");
      }
    }
  }
  {
    nss_status sw = build_work(c);
    if (sw != NSS_OK) {
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());
      free_ctx(c);
      return sw;
    }
  }
  // initial live points
  {
    nss_status si = launch_inits(c);
    if (si != NSS_OK) {
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());
      free_ctx(c);
      return si;
    }
  }
  // GP data and the initial likelihoods
  for (int r = 0; r < n_runs; ++r) {
    if (c->desc[r].lik_kind != nss::kLikGp) continue;
    nss_status sg = setup_gp(c, r, loglik[r]);
    if (sg != NSS_OK) {
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());
      free_ctx(c);
      return sg;
    }
  }
  // logistic-regression workspaces and the initial likelihoods
  for (int r = 0; r < n_runs; ++r) {
    if (c->desc[r].lik_kind != nss::kLikLogreg) continue;
    nss_status sl = setup_logreg(c, r, loglik[r]);
    if (sl != NSS_OK) {
      std::fprintf(stderr, "nss_create: %s\n", c->err.c_str());
      free_ctx(c);
      return sl;
    }
  }
  CKC(cudaStreamSynchronize(c->stream), "init synchronize");
  harvest(c);
#undef CKC
  *out = c;
  return NSS_OK;
}

nss_status nss_create(const nss_prior* prior, const nss_loglik* loglik, int n_live, int k, int p,
                      const nss_options* opt, nss_ctx** out) {
  nss_options o;
  if (opt) o = *opt; else nss_options_default(&o);
  return nss_create_batch(1, prior, loglik, &n_live, &k, &p, &o, out);
}

nss_status nss_step(nss_ctx* c, nss_step_info* info) {
  if (!c) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (!all_done(c)) {
    if ((st = c->plain ? enqueue_plain_iteration(c) : run_iteration(c)) != NSS_OK) return st;
    if ((st = sync_state(c)) != NSS_OK) return st;
  }
  fill_info(c, info);
  for (int r = 0; r < c->n_runs; ++r)
    if (c->h_state[r].status == NSS_ERR_CAPACITY) return set_err(c, NSS_ERR_CAPACITY, "run %d: dead store full", r);
  return all_done(c) ? NSS_DONE : NSS_OK;
}

nss_status nss_run(nss_ctx* c, nss_result* res) {
  if (!c) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (c->plain) {
    // the plain path's host loop waits for every iteration
    while (!all_done(c)) {
      if ((st = enqueue_plain_iteration(c)) != NSS_OK) return st;
      if ((st = sync_state(c)) != NSS_OK) return st;
    }
    return finalise_impl(c, res);
  }
  int chunk = 4;
  while (!all_done(c)) {
    if ((st = run_iteration(c, chunk)) != NSS_OK) return st;
    if ((st = sync_state(c)) != NSS_OK) return st;
    chunk = std::min(chunk * 2, 16);
  }
  return finalise_impl(c, res);
}

nss_status nss_reset(nss_ctx* c, const uint64_t* seeds) {
  if (!c) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (seeds) {
    for (int r = 0; r < c->n_runs; ++r) {
      c->desc[r].key0 = (uint32_t)seeds[r];
      c->desc[r].key1 = (uint32_t)(seeds[r] >> 32) ^ c->run_ids[r];
    }
    CK(cudaMemcpyAsync(c->d_desc, c->desc.data(), sizeof(RunDesc) * c->n_runs, cudaMemcpyHostToDevice,
                       c->stream), "descriptor upload");
    c->prof.h2d_bytes += (long long)sizeof(RunDesc) * c->n_runs;
    CK(cudaStreamSynchronize(c->stream), "descriptor upload");
  }
  clear_states(c);
  CK(cudaMemcpyAsync(c->d_state, c->h_state, sizeof(RunState) * c->n_runs, cudaMemcpyHostToDevice,
                     c->stream), "state upload");
  c->prof.h2d_bytes += (long long)sizeof(RunState) * c->n_runs;
  if ((st = launch_inits(c)) != NSS_OK) return st;
  for (auto& w : c->lr)
    if ((st = lr_initial_loglik(c, w)) != NSS_OK) return st;
  for (auto& g : c->gp)
    if ((st = gp_initial_loglik(c, g)) != NSS_OK) return st;
  return NSS_OK;
}

int nss_cfg_lanes(int cfg) { return (cfg >= 0 && cfg < nss::kNumCfgs) ? nss::cfg_g(cfg) : 0; }
int nss_cfg_dims(int cfg) { return (cfg >= 0 && cfg < nss::kNumCfgs) ? nss::cfg_dpl(cfg) : 0; }

int nss_get_cfg(const nss_ctx* c, int run) {
  if (!c || run < 0 || run >= c->n_runs) return -1;
  return c->desc[run].cfg;
}

nss_status nss_autotune_report(const nss_ctx* c, double* cost) {
  if (!c || !cost) return NSS_ERR_ARG;
  for (int q = 0; q < nss::kNumCfgs; ++q) cost[q] = c->tune_cost[q];
  return NSS_OK;
}

nss_status nss_set_cfg(nss_ctx* c, int run, int cfg) {
  if (!c || run < 0 || run >= c->n_runs) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  bool fits = false;
  for (int q : candidate_cfgs(c->desc[run].d)) fits |= (q == cfg);
  if (!fits) return set_err(c, NSS_ERR_ARG, "configuration %d does not fit d=%d", cfg, c->desc[run].d);
  if (c->plain && cfg >= nss::kLaneCfg0) return set_err(c, NSS_ERR_ARG, "the plain path takes a grouped configuration");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  c->desc[run].cfg = cfg;
  return build_work(c);
}

nss_status nss_autotune(nss_ctx* c, int iters, int* cfg_out) {
  if (!c || iters < 1) return NSS_ERR_ARG;
  if (c->plain) return set_err(c, NSS_ERR_ARG, "the plain path is not autotuned");
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  // runs grouped by the capacity G x DPL their dimension needs
  std::vector<int> caps;
  for (int r = 0; r < c->n_runs; ++r) {
    int cap = 4;
    while (cap < c->desc[r].d) cap <<= 1;
    if (std::find(caps.begin(), caps.end(), cap) == caps.end()) caps.push_back(cap);
  }
  const bool prof_saved = c->profiling;
  const nss_profile prof_saved_v = c->prof;
  c->profiling = true;
  for (int cap : caps) {
    std::vector<int> runs;
    for (int r = 0; r < c->n_runs; ++r) {
      int cr = 4;
      while (cr < c->desc[r].d) cr <<= 1;
      if (cr == cap) runs.push_back(r);
    }
    int best = -1;
    double best_cost = INFINITY;
    for (int q : candidate_cfgs(cap)) {
      for (int r : runs) c->desc[r].cfg = q;
      if ((st = build_work(c)) != NSS_OK) return st;
      if ((st = nss_reset(c, nullptr)) != NSS_OK) return st;
      if ((st = sync_state(c)) != NSS_OK) return st;
      c->cfg_ms[q] = 0.0;
      if ((st = enqueue_iterations(c, iters)) != NSS_OK) return st;
      if ((st = sync_state(c)) != NSS_OK) return st;
      double ev = 0.0;
      for (int r : runs) ev += (double)c->h_state[r].evals;
      const double cost = c->cfg_ms[q] / std::max(1.0, ev);
      c->tune_cost[q] = cost * 1e6;
      if (cost < best_cost) {
        best_cost = cost;
        best = q;
      }
    }
    for (int r : runs) c->desc[r].cfg = best;
  }
  c->profiling = prof_saved;
  c->prof = prof_saved_v;
  if ((st = build_work(c)) != NSS_OK) return st;
  if ((st = nss_reset(c, nullptr)) != NSS_OK) return st;
  if (cfg_out)
    for (int r = 0; r < c->n_runs; ++r) cfg_out[r] = c->desc[r].cfg;
  return sync_state(c);
}

nss_status nss_finalise(nss_ctx* c, nss_result* res) {
  if (!c) return NSS_ERR_ARG;
  return finalise_impl(c, res);
}

nss_status nss_posterior_expectation(nss_ctx* c, int run, int kind, double* out, int n_out) {
  if (!c || run < 0 || run >= c->n_runs || !out) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (!c->h_state[run].finalised) return set_err(c, NSS_ERR_STATE, "posterior expectations before finalisation");
  const RunDesc& R = c->desc[run];
  const long long n = c->h_state[run].n_dead;
  const bool gauss = R.lik_kind == nss::kLikGauss || R.lik_kind == nss::kLikGmm;
  const int K = R.lik_kind == nss::kLikGmm ? R.n_comp : 1;
  int count = -1;
  switch (kind) {
    case NSS_GRAD_LIK_SIGMA: count = gauss ? 1 : -1; break;
    case NSS_GRAD_LIK_MU: count = gauss ? K * R.d : -1; break;
    case NSS_GRAD_PRIOR_LOG_PREC: count = R.prior_kind == nss::kPriorGauss ? 1 : -1; break;
    case NSS_GRAD_GP_NOISE_SCALE: count = R.lik_kind == nss::kLikGp ? 1 : -1; break;
    case NSS_MOMENT_MEAN: count = R.d; break;
    default: break;
  }
  if (count < 0) return set_err(c, NSS_ERR_ARG, "kind %d does not apply to run %d", kind, run);
  if (n_out != count) return set_err(c, NSS_ERR_ARG, "kind %d gives %d values, n_out = %d", kind, count, n_out);
  if (n <= 0) return set_err(c, NSS_ERR_STATE, "run %d has no dead points", run);
  double *coef = nullptr, *dout = nullptr;
  int* didx = nullptr;
  auto release = [&]() {
    cudaFree(coef);
    cudaFree(dout);
    cudaFree(didx);
  };
  cudaError_t e = cudaMalloc(&coef, sizeof(double) * (size_t)n * K);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * count);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "posterior scratch");
  }
  nss::PostArgs A;
  A.x = c->fpool + R.o_dx;
  A.lw = c->dpool + R.o_lw;
  A.n = n;
  A.d = R.d;
  A.ld = R.dpad;
  A.kind = kind;
  A.K = K;
  A.mu = c->fpool + R.o_mu;
  A.pa = c->fpool + R.o_a;
  A.pb = c->fpool + R.o_b;
  A.sigma = c->sigmas[run];
  if (kind == NSS_GRAD_GP_NOISE_SCALE) {
    // dead points whose weight is above 1e-12 of the largest
    std::vector<double> lw((size_t)n);
    e = cudaMemcpyAsync(lw.data(), c->dpool + R.o_lw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(c, e, "weights copy");
    }
    c->prof.d2h_bytes += (long long)sizeof(double) * n;
    double mx = -INFINITY;
    for (double v : lw) mx = std::max(mx, v);
    std::vector<int> idx;
    for (long long i = 0; i < n; ++i)
      if (lw[i] > mx - 27.631021115928547) idx.push_back((int)i);  // ln 1e12
    const GPWork* gw = nullptr;
    for (const auto& g : c->gp)
      if (g.run == run) gw = &g;
    e = cudaMemsetAsync(coef, 0, sizeof(double) * n, c->stream);
    if (e == cudaSuccess && !idx.empty()) e = cudaMalloc(&didx, sizeof(int) * idx.size());
    if (e == cudaSuccess && !idx.empty())
      e = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && gw)
      e = nss::launch_gp_noise_grad(dev_of(c), gw->args, run, didx, (int)idx.size(), R.n_data, coef, c->stream);
    if (e == cudaSuccess) e = nss::launch_post_sum(coef, n, dout, c->stream);
    c->prof.h2d_bytes += (long long)sizeof(int) * (long long)idx.size();
  } else {
    e = nss::launch_post(A, coef, dout, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "posterior expectation");
  c->prof.d2h_bytes += (long long)sizeof(double) * count;
  return NSS_OK;
}

nss_status nss_reweight(nss_ctx* c, int run, double beta, double* out) {
  if (!c || run < 0 || run >= c->n_runs || !out || !std::isfinite(beta) || !(beta > 0.0)) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  if (!c->h_state[run].finalised) return set_err(c, NSS_ERR_STATE, "reweighting before finalisation");
  const RunDesc& R = c->desc[run];
  const long long n = c->h_state[run].n_dead;
  if (n < 1) return set_err(c, NSS_ERR_STATE, "run %d has no dead points", run);
  // the run's tiles alone, through the context's own volume-simulation
  // scratch (finalisation sized it for every run's tiles)
  std::vector<int2> tiles;
  for (long long i = 0; i < n; i += nss::kVolTile) tiles.push_back(make_int2(run, (int)i));
  const int nt = (int)tiles.size();
  if (nt > c->vol_cap_tiles || !c->d_vol) return set_err(c, NSS_ERR_STATE, "volume scratch not sized for run %d", run);
  float* lb = nullptr;
  double *lw = nullptr, *aux = nullptr;
  auto release = [&]() {
    cudaFree(lb);
    cudaFree(lw);
    cudaFree(aux);
  };
  cudaError_t e = cudaMalloc(&lb, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&lw, sizeof(double) * n * 2);
  if (e == cudaSuccess) e = cudaMalloc(&aux, sizeof(double) * 4);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "reweighting scratch");
  }
  e = nss::launch_scale_logL(c->fpool + R.o_dlogL, (float)beta, n, lb, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(int2) * nt, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_vbase + run, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) {
    nss::VolLaunch V;
    V.tiles = c->d_tiles;
    V.vbase = c->d_vbase;
    V.n_tiles = nt;
    V.R = c->R;
    const size_t blk = (size_t)c->R * nt;
    V.tsum = c->d_vol;
    V.toff = c->d_vol + blk;
    V.tmax = c->d_vol + 2 * blk;
    V.tacc = c->d_vol + 3 * blk;
    V.run = run;
    V.logL_in = lb;
    V.lw_out = lw;
    V.stats_out = aux;
    e = nss::launch_volsim(dev_of(c), V, c->n_runs, c->stream);
  }
  if (e == cudaSuccess) e = nss::launch_sq_weights(lw, n, lw + n, c->stream);
  if (e == cudaSuccess) e = nss::launch_post_sum(lw + n, n, aux + 3, c->stream);
  double h[4] = {0.0, 0.0, 0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, aux, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "reweighting");
  c->prof.h2d_bytes += (long long)(sizeof(int2) * nt);
  c->prof.d2h_bytes += (long long)sizeof(double) * 4;
  out[0] = h[0];
  out[1] = h[1];
  out[2] = 1.0 / h[3];
  return NSS_OK;
}

nss_status nss_get_dead(nss_ctx* c, int run, float* x, float* logL, double* log_w, float* birth,
                        int* nlive, size_t cap, size_t* n_out) {
  if (!c || run < 0 || run >= c->n_runs) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  const RunDesc& R = c->desc[run];
  const long long n = c->h_state[run].n_dead;
  if (n_out) *n_out = (size_t)n;
  if (cap == 0) return NSS_OK;
  if (cap < (size_t)n) return set_err(c, NSS_ERR_ARG, "cap %zu < %lld dead points", cap, n);
  if (n == 0) return NSS_OK;
  c->prof.d2h_bytes += n * ((x ? (long long)sizeof(float) * R.d : 0) + (logL ? 4 : 0) + (birth ? 4 : 0) +
                            (nlive ? 4 : 0) + (log_w ? 8 : 0));
  if (x)
    CK(cudaMemcpy2DAsync(x, sizeof(float) * R.d, c->fpool + R.o_dx, sizeof(float) * R.dpad,
                         sizeof(float) * R.d, (size_t)n, cudaMemcpyDefault, c->stream), "dead x copy");
  if (logL) CK(cudaMemcpyAsync(logL, c->fpool + R.o_dlogL, sizeof(float) * n, cudaMemcpyDefault, c->stream), "dead logL copy");
  if (birth) CK(cudaMemcpyAsync(birth, c->fpool + R.o_dbirth, sizeof(float) * n, cudaMemcpyDefault, c->stream), "dead birth copy");
  if (nlive) CK(cudaMemcpyAsync(nlive, c->ipool + R.o_dn, sizeof(int) * n, cudaMemcpyDefault, c->stream), "dead n copy");
  if (log_w) {
    if (!c->h_state[run].finalised) return set_err(c, NSS_ERR_STATE, "weights before finalisation");
    CK(cudaMemcpyAsync(log_w, c->dpool + R.o_lw, sizeof(double) * n, cudaMemcpyDefault, c->stream), "weights copy");
  }
  CK(cudaStreamSynchronize(c->stream), "copy synchronize");
  return NSS_OK;
}

nss_status nss_export_state(nss_ctx* c, int run, float* x, float* logL, float* birth, nss_state* s) {
  if (!c || run < 0 || run >= c->n_runs) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  const RunDesc& R = c->desc[run];
  if (x)
    CK(cudaMemcpy2DAsync(x, sizeof(float) * R.d, c->fpool + R.o_x, sizeof(float) * R.dpad,
                         sizeof(float) * R.d, (size_t)R.m, cudaMemcpyDefault, c->stream), "live x copy");
  if (logL) CK(cudaMemcpyAsync(logL, c->fpool + R.o_logL, sizeof(float) * R.m, cudaMemcpyDefault, c->stream), "live logL copy");
  if (birth) CK(cudaMemcpyAsync(birth, c->fpool + R.o_birth, sizeof(float) * R.m, cudaMemcpyDefault, c->stream), "live birth copy");
  CK(cudaStreamSynchronize(c->stream), "copy synchronize");
  if (s) {
    const RunState& h = c->h_state[run];
    s->iter = h.iter;
    s->logZ = h.logZ;
    s->logX = h.logX;
    s->n_dead = h.n_dead;
  }
  return NSS_OK;
}

nss_status nss_import_state(nss_ctx* c, int run, const float* x, const float* logL, const float* birth,
                            const nss_state* s) {
  if (!c || run < 0 || run >= c->n_runs || !x || !logL || !s) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  const RunDesc& R = c->desc[run];
  if (s->iter < 0 || s->n_dead < 0 || s->n_dead > R.dead_cap) return set_err(c, NSS_ERR_ARG, "invalid imported scalars");
  for (int i = 0; i < R.m; ++i)
    if (std::isnan(logL[i])) return set_err(c, NSS_ERR_ARG, "NaN logL in imported state");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  CK(cudaMemsetAsync(c->fpool + R.o_x, 0, sizeof(float) * (size_t)R.m * R.dpad, c->stream), "live clear");
  CK(cudaMemcpy2DAsync(c->fpool + R.o_x, sizeof(float) * R.dpad, x, sizeof(float) * R.d,
                       sizeof(float) * R.d, (size_t)R.m, cudaMemcpyDefault, c->stream), "live x upload");
  CK(cudaMemcpyAsync(c->fpool + R.o_logL, logL, sizeof(float) * R.m, cudaMemcpyDefault, c->stream), "live logL upload");
  if (birth) {
    CK(cudaMemcpyAsync(c->fpool + R.o_birth, birth, sizeof(float) * R.m, cudaMemcpyDefault, c->stream), "live birth upload");
  } else {
    std::vector<float> nb(R.m, -INFINITY);
    CK(cudaMemcpyAsync(c->fpool + R.o_birth, nb.data(), sizeof(float) * R.m, cudaMemcpyHostToDevice, c->stream), "live birth upload");
    CK(cudaStreamSynchronize(c->stream), "upload synchronize");
  }
  RunState& h = c->h_state[run];
  RunState ns;
  std::memset(&ns, 0, sizeof ns);
  ns.iter = s->iter;
  ns.logZ = s->logZ;
  ns.logX = s->logX;
  ns.n_dead = s->n_dead;
  ns.logLstar = -INFINITY;
  ns.evals = h.evals;
  CK(cudaMemcpyAsync(c->d_state + run, &ns, sizeof ns, cudaMemcpyHostToDevice, c->stream), "state upload");
  return sync_state(c);
}

nss_status nss_step_trace(nss_ctx* c, int run, nss_trace* tr) {
  if (!c || run < 0 || run >= c->n_runs || !tr) return NSS_ERR_ARG;
  if (c->broken) return set_err(c, NSS_ERR_STATE, "context is unusable after an earlier CUDA error");
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  const RunState& h = c->h_state[run];
  if (!h.stepped) return set_err(c, NSS_ERR_STATE, "no step since create or import");
  const RunDesc& R = c->desc[run];
  std::vector<int> dead(R.k), stats(6 * (size_t)R.k);
  CK(cudaMemcpyAsync(dead.data(), c->ipool + R.o_dead, sizeof(int) * R.k, cudaMemcpyDeviceToHost, c->stream), "trace copy");
  CK(cudaMemcpyAsync(stats.data(), c->ipool + R.o_stats, sizeof(int) * 6 * R.k, cudaMemcpyDeviceToHost, c->stream), "trace copy");
  if (tr->parent) CK(cudaMemcpyAsync(tr->parent, c->ipool + R.o_parent, sizeof(int) * R.k, cudaMemcpyDefault, c->stream), "trace copy");
  if (tr->L)
    CK(cudaMemcpy2DAsync(tr->L, sizeof(float) * R.d, c->fpool + R.o_L, sizeof(float) * R.dpad,
                         sizeof(float) * R.d, (size_t)R.d, cudaMemcpyDefault, c->stream), "trace copy");
  std::vector<float> lx((size_t)R.m * R.dpad), ll(R.m);
  CK(cudaMemcpyAsync(lx.data(), c->fpool + R.o_x, sizeof(float) * lx.size(), cudaMemcpyDeviceToHost, c->stream), "trace copy");
  CK(cudaMemcpyAsync(ll.data(), c->fpool + R.o_logL, sizeof(float) * R.m, cudaMemcpyDeviceToHost, c->stream), "trace copy");
  CK(cudaStreamSynchronize(c->stream), "trace synchronize");
  if (tr->dead_idx) std::memcpy(tr->dead_idx, dead.data(), sizeof(int) * R.k);
  int* dst[6] = {tr->evals, tr->accepts, tr->nulls, tr->expansions, tr->shrinks, tr->cap_out};
  for (int q = 0; q < 6; ++q)
    if (dst[q]) std::memcpy(dst[q], stats.data() + (size_t)q * R.k, sizeof(int) * R.k);
  for (int j = 0; j < R.k; ++j) {
    const int slot = dead[j];
    if (tr->new_x) std::memcpy(tr->new_x + (size_t)j * R.d, lx.data() + (size_t)slot * R.dpad, sizeof(float) * R.d);
    if (tr->new_logL) tr->new_logL[j] = ll[slot];
  }
  tr->logLstar = h.logLstar;
  return NSS_OK;
}

nss_status nss_set_profiling(nss_ctx* c, int on) {
  if (!c) return NSS_ERR_ARG;
  c->profiling = on != 0;
  if (on) std::memset(&c->prof, 0, sizeof c->prof);
  return NSS_OK;
}

nss_status nss_get_profile(nss_ctx* c, nss_profile* p) {
  if (!c || !p) return NSS_ERR_ARG;
  nss_status st = sync_state(c);
  if (st != NSS_OK) return st;
  *p = c->prof;
  return NSS_OK;
}

void nss_destroy(nss_ctx* c) {
  if (!c) return;
  if (!c->broken) cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"
