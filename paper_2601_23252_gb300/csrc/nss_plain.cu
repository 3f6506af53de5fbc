// nss_plain.cu -- the plain single-run FP32 path's HRSS phase: one kernel
// launch per HRSS step, one thread per chain, the run's k chains advancing
// in lockstep evaluation rounds (Sec. 3.1: all chains evaluate the
// likelihood together as one batched operation), for sm_103a.
//
// This is the comparator of the batched sweep (nss_sweep_chain.cuh), not a
// production path.  Per step of chain j:
//   - the direction v (drawn ahead by k_dirgen) and the step's words;
//   - stepping out to the left, then to the right, then shrinkage (App. B.4),
//     each a loop of rounds that ends when every chain of the run has left
//     it (a block-wide vote per round); a chain evaluates one candidate per
//     round and a chain that is done waits for the others;
//   - every candidate's likelihood is evaluated from scratch: the squared
//     distance of x + t v to each component mean, the box interval of the
//     line and the prior term are recomputed over all d coordinates for
//     each evaluation (O(d K) work per evaluation, as a batched likelihood
//     call over the k candidate points does).
// The FP32 expressions and their reduction order are those of the batched
// sweep in sweep configuration (G, DPL): per G lanes a sequential fmaf
// chain over DPL coordinates, then the lanes' pairwise (butterfly) sums.  So
// the two paths take the same decisions and produce bit-identical dead
// points; they differ in schedule and work, not in results.
//
// The chain's state between step launches lives in its dead slot of the
// live set (never a parent: parents are survivors), its counters in the
// per-chain statistics of the iteration.
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {
namespace {

constexpr int kPlainMaxThreads = 1024;

// The butterfly sum of G lane partials p[0..G): at every stage lane l adds
// lane l ^ o's value, so every lane ends with lane 0's total; formed here in
// place as lane 0 sees it.
__device__ __forceinline__ float lanes_sum(float* p, int G) {
  for (int o = G >> 1; o > 0; o >>= 1)
    for (int l = 0; l < o; ++l) p[l] = p[l] + p[l + o];
  return p[0];
}

struct PlainChain {
  const RunDesc* R;
  const float* x;    // [dpad]
  const float* v;    // [dpad]
  const float* mu;   // [n_comp][dpad]
  const float* pa;   // prior lower bound / mean [dpad]
  const float* pb;   // prior upper bound / sd [dpad]
  int G, DPL, K;
  bool box;
  float lstar, qh;   // threshold; Gaussian prior: log u of the slice height

  // coordinate i of a lane slice, zero past the padded row
  __device__ __forceinline__ float at(const float* a, int i) const { return i < R->dpad ? a[i] : 0.0f; }

  // one slice test at x + t v, from scratch
  __device__ bool test(float t, float& ll, bool& isn) const {
    const int d = R->d;
    float part[32];
    bool ok = true;
    if (box) {
      float t_lo = -INFINITY, t_hi = INFINITY;
      for (int i = 0; i < d; ++i) {
        const float xi = x[i], vi = v[i];
        const float ai = pa[i] - xi, bi = pb[i] - xi;
        const float rv = __fdividef(1.0f, vi);
        const float ta = ai * rv, tb = bi * rv;
        t_lo = fmaxf(t_lo, fminf(ta, tb));
        t_hi = fminf(t_hi, fmaxf(ta, tb));
      }
      ok = t >= t_lo && t <= t_hi;
    } else {
      float P[3];
      for (int q = 0; q < 3; ++q) {
        for (int g = 0; g < G; ++g) {
          float a = 0.0f;
          for (int e = 0; e < DPL; ++e) {
            const int i = g * DPL + e;
            if (i < d) {
              const float ib = 1.0f / pb[i];
              const float u = (x[i] - pa[i]) * ib, w = v[i] * ib;
              a = fmaf(q == 0 ? u : q == 1 ? u : w, q == 0 ? u : w, a);
            }
          }
          part[g] = a;
        }
        P[q] = lanes_sum(part, G);
      }
      const float q3 = fmaf(-0.5f, P[0], R->prior_const) + qh;
      const float lp = fmaf(-0.5f, fmaf(t, fmaf(t, P[2], 2.0f * P[1]), P[0]), R->prior_const);
      ok = lp > q3;
    }
    if (R->lik_kind == kLikFlat) {
      ll = 0.0f;
    } else {
      for (int g = 0; g < G; ++g) {
        float a = 0.0f;
        for (int e = 0; e < DPL; ++e) {
          const float vi = at(v, g * DPL + e);
          a = fmaf(vi, vi, a);
        }
        part[g] = a;
      }
      const float Cv = lanes_sum(part, G);
      float vc[8];
      float M = -INFINITY;
      for (int c = 0; c < K; ++c) {
        const float* m = mu + (long long)c * R->dpad;
        float pe[32];
        for (int g = 0; g < G; ++g) {
          float dq = 0.0f, de = 0.0f;
          for (int e = 0; e < DPL; ++e) {
            const int i = g * DPL + e;
            const float ei = at(x, i) - at(m, i);
            dq = fmaf(ei, ei, dq);
            de = fmaf(ei, at(v, i), de);
          }
          part[g] = dq;
          pe[g] = de;
        }
        const float Dc = lanes_sum(part, G), Ec = lanes_sum(pe, G);
        vc[c] = -fmaf(t, fmaf(t, Cv, 2.0f * Ec), Dc) * R->inv2s2;
        M = fmaxf(M, vc[c]);
      }
      if (K == 1) {
        ll = M + R->lognorm;
      } else {
        float S = 0.0f;
        for (int c = 0; c < K; ++c) S += __expf(vc[c] - M);
        ll = M + __logf(S) + R->lognorm;
      }
    }
    const bool nan_ll = isnan(ll);
    ll = nan_ll ? -INFINITY : ll;
    isn = ok && nan_ll;
    return ok && ll > lstar;
  }
};

__global__ void __launch_bounds__(kPlainMaxThreads) k_plain_hrss(Dev D, int run, int s, int G, int DPL) {
  const RunDesc& R = D.desc[run];
  RunState* S = D.st + run;
  if (S->done) return;
  const int j = threadIdx.x;
  const bool live = j < R.k;
  const int d = R.d, ld = R.dpad;
  const uint32_t iter = (uint32_t)S->iter;
  float x[kMaxD], v[kMaxD];
  float lx = 0.0f;
  int acc = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  int slot = 0;
  const int* st = D.i + R.o_stats;
  if (live) {
    slot = D.i[R.o_dead + j];
    const int src = (s == 0) ? D.i[R.o_parent + j] : slot;
    for (int i = 0; i < ld; ++i) x[i] = D.f[R.o_x + (long long)src * ld + i];
    lx = D.f[R.o_logL + src];
    const float* vr = D.f + R.o_V + ((long long)j * R.p + s) * ld;
    for (int i = 0; i < ld; ++i) v[i] = vr[i];
    if (s > 0) {
      acc = st[R.k + j];
      exps = st[3 * R.k + j];
      shr = st[4 * R.k + j];
      capo = st[5 * R.k + j];
    }
  }
  const int* ws = D.i + R.o_wd + ((long long)j * R.p + s) * kStepWords;
  const uint32_t nz = 2u * (uint32_t)((d + 1) >> 1);
  PlainChain C;
  C.R = &R;
  C.x = x;
  C.v = v;
  C.mu = D.f + R.o_mu;
  C.pa = D.f + R.o_a;
  C.pb = D.f + R.o_b;
  C.G = G;
  C.DPL = DPL;
  C.K = (R.lik_kind == kLikGmm) ? R.n_comp : 1;
  C.box = R.prior_kind == kPriorBox;
  C.lstar = S->logLstar;
  C.qh = live && !C.box ? logf(u24((uint32_t)ws[1])) : 0.0f;
  const float w = R.w;
  const float tl0 = live ? -w * u24((uint32_t)ws[0]) : 0.0f;
  float ends[2] = {tl0, tl0 + w};
  // stepping out, the left side then the right, in lockstep rounds
  for (int q = 0; q < 2; ++q) {
    const float delta = q ? w : -w;
    float t = ends[q];
    int n = 0;
    bool active = live;
    while (__syncthreads_or(active)) {
      if (active) {
        bool isn = false;
        float ll = 0.0f;
        const bool in = C.test(t, ll, isn);
        nanc += isn;
        if (in) {
          t += delta;
          ++n;
          if (n == kStepOutCap) {
            ++capo;
            active = false;
          }
        } else {
          active = false;
        }
      }
    }
    ends[q] = t;
    exps += n;
  }
  // shrinkage, at most kShrinkCap proposals, then a null move
  float tl = ends[0], tr = ends[1], tacc = 0.0f, llacc = 0.0f;
  bool ok = false, active = live;
  int r = 0;
  while (__syncthreads_or(active)) {
    if (active) {
      const uint32_t ri = 3u + (uint32_t)r;
      uint32_t wr;
      if (ri < (uint32_t)kStepWords) {
        wr = (uint32_t)ws[ri];
      } else {
        const uint32_t wi = nz + ri;
        wr = pick(draw_block(R, iter, (uint32_t)j, (uint32_t)s, wi >> 2), wi & 3u);
      }
      const float t = fmaf(u24(wr), tr - tl, tl);
      ++shr;
      bool isn = false;
      float ll = 0.0f;
      const bool in = C.test(t, ll, isn);
      nanc += isn;
      if (in) {
        tacc = t;
        llacc = ll;
        ok = true;
        active = false;
      } else {
        if (t < 0.0f) tl = t;
        else tr = t;
        if (++r == kShrinkCap) active = false;
      }
    }
  }
  if (!live) return;
  if (ok) {
    for (int i = 0; i < ld; ++i) x[i] = fmaf(tacc, v[i], x[i]);
    lx = llacc;
    ++acc;
  }
  for (int i = 0; i < ld; ++i) D.f[R.o_x + (long long)slot * ld + i] = x[i];
  D.f[R.o_logL + slot] = lx;
  int* sw = D.i + R.o_stats;
  sw[R.k + j] = acc;
  sw[3 * R.k + j] = exps;
  sw[4 * R.k + j] = shr;
  sw[5 * R.k + j] = capo;
  if (nanc) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nan_evals), (unsigned long long)nanc);
  if (s == R.p - 1) {
    // (iv) the chain's point replaces dead slot j, born at logL*
    const int nul = R.p - acc;
    const int evals = exps + 2 * R.p - capo + shr;
    D.f[R.o_birth + slot] = C.lstar;
    sw[j] = evals;
    sw[2 * R.k + j] = nul;
    atomicAdd(reinterpret_cast<unsigned long long*>(&S->evals), (unsigned long long)evals);
    if (nul) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nulls), (unsigned long long)nul);
    if (capo) atomicAdd(reinterpret_cast<unsigned long long*>(&S->cap_out), (unsigned long long)capo);
  }
}

}  // namespace

cudaError_t launch_plain_hrss(const Dev& D, int run, int k, int s, int G, int DPL, cudaStream_t st) {
  if (k < 1 || k > kPlainMaxThreads || G < 1 || G > 32 || DPL < 1) return cudaErrorInvalidValue;
  const int threads = (k + 31) / 32 * 32;
  k_plain_hrss<<<1, threads, 0, st>>>(D, run, s, G, DPL);
  return cudaGetLastError();
}

}  // namespace nss
