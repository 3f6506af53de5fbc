// nss_kernels.cu -- the Nested Slice Sampling kernels for sm_103a.
//
// Per outer iteration (Sec. 3.1 (i)-(iv); Algorithm 1):
//   k_prologue  one block per run: select the k worst live points by a
//               bitonic sort of (logL, slot) keys, threshold logL*, survivors
//               in slot order, parents, dead-point append, unrolled evidence
//               update (FP64 accumulation), live-set covariance and its
//               Cholesky factor (the direction metric, Sec. 3.2).
//   k_sweep     persistent grid over (run, chain) work items: each chain group
//               of G lanes runs p Hit-and-Run Slice Sampling steps with the
//               likelihood evaluated inside the step (App. B.4) and writes the
//               new point into its dead slot (step (iv)).
//   k_terminate one block per run: remaining live evidence and the stopping
//               test (App. B.3).
// After termination:
//   k_final_sort  kill the live set in (logL, slot) order with n = m..1.
//   k_vol_*       post-hoc volume-shrinkage simulation, evidence error and
//                 posterior weights (App. D.2).
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {

// ---------------------------------------------------------------------------
// Likelihood of a chain group: lane gl owns dimensions [4 gl, 4 gl + 4).
// Padding dimensions hold zeros in x, v and the means, so they add nothing.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ float group_loglik(const RunDesc& R, const float* __restrict__ f,
                                              const float y[4], int gl, unsigned mask) {
  const int lk = R.lik_kind;
  const bool has = gl * 4 < R.dpad;
  if (lk == kLikFlat) return 0.0f;
  if (lk == kLikGauss || lk == kLikFault) {
    float q = 0.0f;
    if (has) {
      const float4 m = __ldg(reinterpret_cast<const float4*>(f + R.o_mu) + gl);
      const float e0 = y[0] - m.x, e1 = y[1] - m.y, e2 = y[2] - m.z, e3 = y[3] - m.w;
      q = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, e3 * e3)));
    }
    q = gsum<G>(q, mask);
    float ll = fmaf(-q, R.inv2s2, R.lognorm);
    if (lk == kLikFault) {
      const float x0 = __shfl_sync(mask, y[0], 0, G);
      if (x0 < R.fault_param) ll = (R.fault_mode == 1) ? __int_as_float(0x7fc00000) : INFINITY;
    }
    return ll;
  }
  // equal-weight isotropic mixture: online log-sum-exp over components
  float M = -INFINITY, S = 0.0f;
  const float4* mu = reinterpret_cast<const float4*>(f + R.o_mu);
  const int stride4 = R.dpad >> 2;
  for (int c = 0; c < R.n_comp; ++c) {
    float q = 0.0f;
    if (has) {
      const float4 m = __ldg(mu + c * stride4 + gl);
      const float e0 = y[0] - m.x, e1 = y[1] - m.y, e2 = y[2] - m.z, e3 = y[3] - m.w;
      q = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, e3 * e3)));
    }
    q = gsum<G>(q, mask);
    const float v = -q * R.inv2s2;
    if (v > M) {
      S = S * expf(M - v) + 1.0f;
      M = v;
    } else {
      S += expf(v - M);
    }
  }
  return M + logf(S) + R.lognorm;
}

// Per-chain constants held by every lane of a group.
struct ChainConst {
  float a[4], b[4];
  bool own[4];
  float lstar;
  bool box, nonflat;
};

template <int G>
__device__ __forceinline__ float group_logprior(const RunDesc& R, const ChainConst& C,
                                                const float y[4], unsigned mask) {
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (C.own[i]) {
      const float u = (y[i] - C.a[i]) / C.b[i];
      s = fmaf(-0.5f * u, u, s);
    }
  return gsum<G>(s, mask) + R.prior_const;
}

// One logical likelihood evaluation: y is in the slice when it is in the prior
// support, above the prior slice height (non-flat prior) and strictly above
// logL* (Sec. 3.1: E < E_batch).  Returns the decision, identical in all lanes.
template <int G>
__device__ __forceinline__ bool in_slice(const RunDesc& R, const float* __restrict__ f,
                                         const ChainConst& C, const float y[4], float height,
                                         int gl, unsigned mask, float& ll, int& nan_cnt) {
  if (C.box) {
    bool out = false;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (C.own[i] && !(y[i] >= C.a[i] && y[i] <= C.b[i])) out = true;
    if (__any_sync(mask, out)) return false;
  }
  if (C.nonflat) {
    const float lp = group_logprior<G>(R, C, y, mask);
    if (!(lp > height)) return false;
  }
  ll = group_loglik<G>(R, f, y, gl, mask);
  if (isnan(ll)) {
    ll = -INFINITY;
    ++nan_cnt;
  }
  return ll > C.lstar;
}

// Words of one HRSS step, cached one Philox block (four words) at a time.
struct WordCache {
  uint32_t blk;
  uint4 v;
};
__device__ __forceinline__ uint32_t step_word(const RunDesc& R, WordCache& wc, uint32_t iter,
                                              uint32_t chain, uint32_t step, uint32_t wi) {
  const uint32_t b = wi >> 2;
  if (b != wc.blk) {
    wc.v = draw_block(R, iter, chain, step, b);
    wc.blk = b;
  }
  return pick(wc.v, wi & 3u);
}

// ---------------------------------------------------------------------------
// Initial live set: m prior draws per run (Sec. 2.1), counter (0, slot,
// TAG_INIT, word/4); group lane gl draws dimensions [4 gl, 4 gl + 4).
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(128) k_init(Dev D, const WorkItem* __restrict__ items, int n_items) {
  const int lane = threadIdx.x & 31;
  const int gl = lane % G, grp = lane / G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = warp; it < n_items; it += nwarps) {
    const WorkItem wi = items[it];
    const RunDesc& R = D.desc[wi.run];
    const int slot = wi.c0 + grp;
    if (slot >= wi.c1) continue;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    const bool has = gl * 4 < R.dpad;
    const uint4 w = draw_block(R, 0u, (uint32_t)slot, kTagInit, (uint32_t)gl);
    if (R.prior_kind == kPriorBox) {
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int dim = gl * 4 + i;
        if (dim < R.d) {
          const float a = D.f[R.o_a + dim], b = D.f[R.o_b + dim];
          x[i] = fmaf(b - a, u24(ws[i]), a);
        }
      }
    } else {
      float z[4];
      box_muller(w.x, w.y, z[0], z[1]);
      box_muller(w.z, w.w, z[2], z[3]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int dim = gl * 4 + i;
        if (dim < R.d) x[i] = fmaf(D.f[R.o_b + dim], z[i], D.f[R.o_a + dim]);
      }
    }
    float ll = group_loglik<G>(R, D.f, x, gl, mask);
    if (isnan(ll)) ll = -INFINITY;
    if (has) {
      reinterpret_cast<float4*>(D.f + R.o_x + (long long)slot * R.dpad)[gl] =
          make_float4(x[0], x[1], x[2], x[3]);
    }
    if (gl == 0) {
      D.f[R.o_logL + slot] = ll;
      D.f[R.o_birth + slot] = -INFINITY;
    }
  }
}

// ---------------------------------------------------------------------------
// Unrolled evidence update for `cnt` deaths (App. D.1): the j-th death has
// n = m - j live points; with cum_j = sum_{j'<j} 1/(m - j') and
// lnd_j = log(1 - e^{-1/(m-j)}), its Delta-X term is
//   logL_j + logX_0 - cum_j + lnd_j  (Eq. eq:marginal with E[log t] = -1/n).
// The terms are combined by a block log-sum-exp: max and offsets in FP64,
// the exponentials of the (FP64) differences in FP32, the sum in FP64.
// ---------------------------------------------------------------------------
__device__ void evidence_update(const RunDesc& R, RunState& S, const float* __restrict__ dlogL,
                                const double* __restrict__ cum, const double* __restrict__ lnd,
                                int cnt, double* red) {
  const double lx0 = S.logX;
  double mx = -INFINITY;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const double t = (double)dlogL[j] + (lx0 - cum[j]) + lnd[j];
    mx = fmax(mx, t);
  }
  mx = block_max_d(mx, red);
  double s = 0.0;
  if (mx > -INFINITY) {
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const double t = (double)dlogL[j] + (lx0 - cum[j]) + lnd[j];
      s += (double)expf((float)(t - mx));
    }
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    if (mx > -INFINITY) S.logZ = logaddexp_d(S.logZ, mx + log(s));
    S.logX = lx0 - cum[cnt];
  }
  __syncthreads();
}

// Append the first `cnt` entries of the sorted key list to the dead store.
__device__ void append_dead(const Dev& D, const RunDesc& R, RunState& S,
                            const unsigned long long* keys, int cnt) {
  const long long base = S.n_dead;
  const int q4 = R.dpad >> 2;
  const float4* xs = reinterpret_cast<const float4*>(D.f + R.o_x);
  float4* xd = reinterpret_cast<float4*>(D.f + R.o_dx + base * R.dpad);
  for (int t = threadIdx.x; t < cnt * q4; t += blockDim.x) {
    const int j = t / q4, c = t - j * q4;
    const int slot = (int)(keys[j] & 0xffffffffu);
    xd[(long long)j * q4 + c] = xs[(long long)slot * q4 + c];
  }
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int slot = (int)(keys[j] & 0xffffffffu);
    D.f[R.o_dlogL + base + j] = D.f[R.o_logL + slot];
    D.f[R.o_dbirth + base + j] = D.f[R.o_birth + slot];
    D.i[R.o_dn + base + j] = R.m - j;
  }
}

// Cholesky factor of S + reg I into Lm (both [dpad][dpad] in shared memory);
// left-looking by columns; returns true on a non-positive pivot.
__device__ bool cholesky_smem(const float* S, float* Lm, int d, int ld, float reg, int* flag) {
  for (int t = threadIdx.x; t < ld * ld; t += blockDim.x) Lm[t] = 0.0f;
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < d; ++j) {
    if (wid == 0) {
      float s = 0.0f;
      for (int q = lane; q < j; q += 32) s = fmaf(Lm[j * ld + q], Lm[j * ld + q], s);
      s = warp_sum_f(s);
      if (lane == 0) {
        const float v = S[j * ld + j] + reg - s;
        if (!(v > 0.0f) || !isfinite(v)) *flag = 1;
        Lm[j * ld + j] = sqrtf(fmaxf(v, 0.0f));
      }
    }
    __syncthreads();
    if (*flag) return true;
    const float ljj = Lm[j * ld + j];
    for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) {
      float t = S[i * ld + j];
      for (int q = 0; q < j; ++q) t = fmaf(-Lm[i * ld + q], Lm[j * ld + q], t);
      Lm[i * ld + j] = t / ljj;
    }
    __syncthreads();
  }
  return false;
}

// Direction metric (Sec. 3.2): covariance of the m live points (divisor m-1)
// about a shifted mean, FP32 with 4x4 register tiles and a fixed-order
// reduction; regularised by eps * tr/d and factorised; a failed factorisation
// retries with 10x the jitter (up to 6 times); a zero or non-finite trace
// gives the identity.
__device__ void live_metric(const Dev& D, const RunDesc& R, RunState& S, char* smem) {
  const int d = R.d, ld = R.dpad, m = R.m, T = blockDim.x;
  const float* X = D.f + R.o_x;
  __shared__ float mu_s[kMaxD];
  __shared__ int flag_s;
  __shared__ double red_s[32];
  float* part = reinterpret_cast<float*>(smem);
  // mean of x - x_0 per dimension
  const int nparts = T / ld;
  {
    const int a = threadIdx.x % ld, pi = threadIdx.x / ld;
    float s = 0.0f;
    if (pi < nparts && a < d) {
      const float ref = X[a];
      for (int i = pi; i < m; i += nparts) s += X[(long long)i * ld + a] - ref;
    }
    if (pi < nparts) part[pi * ld + a] = s;
    __syncthreads();
    if (threadIdx.x < ld) {
      float t = 0.0f;
      for (int q = 0; q < nparts; ++q) t += part[q * ld + threadIdx.x];
      mu_s[threadIdx.x] = (threadIdx.x < d) ? t / (float)m : 0.0f;
    }
    __syncthreads();
  }
  // lower-triangular 4x4 tiles of sum_i c_i c_i^T, c_i = (x_i - x_0) - mu
  const int nt = ld >> 2, ntp = nt * (nt + 1) / 2;
  const int parts2 = max(1, T / ntp);
  float* red = part;                             // [parts2][ntp][16]
  float* Sm = part + (size_t)parts2 * ntp * 16;  // [ld][ld]
  float* Lm = Sm + ld * ld;                      // [ld][ld]
  for (int tpp = threadIdx.x; tpp < parts2 * ntp; tpp += T) {
    const int tp = tpp % ntp, pi = tpp / ntp;
    int ta = 0;
    while ((ta + 1) * (ta + 2) / 2 <= tp) ++ta;
    const int tb = tp - ta * (ta + 1) / 2;
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
    const float4 ra = reinterpret_cast<const float4*>(X)[ta];
    const float4 rb = reinterpret_cast<const float4*>(X)[tb];
    const float ma[4] = {mu_s[4 * ta], mu_s[4 * ta + 1], mu_s[4 * ta + 2], mu_s[4 * ta + 3]};
    const float mb[4] = {mu_s[4 * tb], mu_s[4 * tb + 1], mu_s[4 * tb + 2], mu_s[4 * tb + 3]};
    for (int i = pi; i < m; i += parts2) {
      const float4 xa = reinterpret_cast<const float4*>(X + (long long)i * ld)[ta];
      const float4 xb = reinterpret_cast<const float4*>(X + (long long)i * ld)[tb];
      const float ca[4] = {(xa.x - ra.x) - ma[0], (xa.y - ra.y) - ma[1], (xa.z - ra.z) - ma[2],
                           (xa.w - ra.w) - ma[3]};
      const float cb[4] = {(xb.x - rb.x) - mb[0], (xb.y - rb.y) - mb[1], (xb.z - rb.z) - mb[2],
                           (xb.w - rb.w) - mb[3]};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(ca[u], cb[v], acc[u * 4 + v]);
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) red[((size_t)pi * ntp + tp) * 16 + e] = acc[e];
  }
  __syncthreads();
  const float inv = 1.0f / (float)(m - 1);
  for (int e = threadIdx.x; e < ntp * 16; e += T) {
    const int tp = e >> 4, uv = e & 15;
    float s = 0.0f;
    for (int q = 0; q < parts2; ++q) s += red[((size_t)q * ntp + tp) * 16 + uv];
    int ta = 0;
    while ((ta + 1) * (ta + 2) / 2 <= tp) ++ta;
    const int tb = tp - ta * (ta + 1) / 2;
    const int a = 4 * ta + (uv >> 2), b = 4 * tb + (uv & 3);
    const float val = (a < d && b < d) ? s * inv : 0.0f;
    Sm[a * ld + b] = val;
    Sm[b * ld + a] = val;
  }
  __syncthreads();
  double tr = 0.0;
  for (int a = threadIdx.x; a < d; a += T) tr += (double)Sm[a * ld + a];
  tr = block_sum_d(tr, red_s);
  int status = 0;
  bool identity = false;
  if (!(tr > 0.0) || !isfinite(tr)) {
    identity = true;
    status = 1;
  } else {
    float reg = R.cov_eps * (float)tr / (float)d;
    bool fail = true;
    for (int attempt = 0; attempt <= 6; ++attempt) {
      fail = cholesky_smem(Sm, Lm, d, ld, reg, &flag_s);
      __syncthreads();
      if (!fail) break;
      reg *= 10.0f;
      status = 2;
    }
    if (fail) {
      identity = true;
      status = 3;
    }
  }
  float* Lg = D.f + R.o_L;
  for (int t = threadIdx.x; t < ld * ld; t += T) {
    const int a = t / ld, b = t - a * ld;
    Lg[t] = identity ? ((a == b && a < d) ? 1.0f : 0.0f) : Lm[t];
  }
  if (threadIdx.x == 0) S.metric_status = status;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Iteration prologue: steps (i), (ii), evidence and metric for one run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_prologue(Dev D) {
  const int run = blockIdx.x;
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  extern __shared__ __align__(16) char smem[];
  __shared__ double red_d[32];
  __shared__ int red_i[32];
  __shared__ int cap_fail;
  const int m = R.m, k = R.k, m2 = R.m2;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
  int* surv = reinterpret_cast<int*>(smem + (size_t)m2 * 8);
  const float* logL = D.f + R.o_logL;
  for (int i = threadIdx.x; i < m2; i += blockDim.x)
    keys[i] = (i < m) ? sort_key(logL[i], i) : ~0ull;
  bitonic_sort(keys, m2);
  // (i) dead slots, worst first; threshold = the k-th worst
  int* dead = D.i + R.o_dead;
  for (int j = threadIdx.x; j < k; j += blockDim.x) dead[j] = (int)(keys[j] & 0xffffffffu);
  if (threadIdx.x == 0) {
    S.logLstar = logL[(int)(keys[k - 1] & 0xffffffffu)];
    cap_fail = (S.n_dead + k > R.dead_cap);
  }
  __syncthreads();
  if (cap_fail) {
    if (threadIdx.x == 0) {
      S.done = 1;
      S.status = -4;
    }
    return;
  }
  // survivors in ascending slot order: flag the dead, compact the rest
  int* flag = surv + m2;  // [m]
  for (int i = threadIdx.x; i < m; i += blockDim.x) flag[i] = 1;
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) flag[(int)(keys[j] & 0xffffffffu)] = 0;
  __syncthreads();
  {
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    int c = 0;
    for (int i = i0; i < min(i0 + per, m); ++i) c += flag[i];
    int tot;
    int pos = block_exscan_i(c, red_i, &tot);
    for (int i = i0; i < min(i0 + per, m); ++i)
      if (flag[i]) surv[pos++] = i;
  }
  __syncthreads();
  // (ii) parents uniformly with replacement among the m-k survivors
  int* parent = D.i + R.o_parent;
  const uint32_t iter = (uint32_t)S.iter;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const uint32_t w = draw_block(R, iter, (uint32_t)j, kTagParent, 0u).x;
    parent[j] = surv[__umulhi(w, (uint32_t)(m - k))];
  }
  // dead store and unrolled evidence
  append_dead(D, R, S, keys, k);
  __syncthreads();
  evidence_update(R, S, D.f + R.o_dlogL + S.n_dead, D.dd + R.o_cum, D.dd + R.o_lnd, k, red_d);
  if (threadIdx.x == 0) S.n_dead += k;
  __syncthreads();
  // direction metric from the live set at the start of the iteration
  live_metric(D, R, S, smem);
}

// ---------------------------------------------------------------------------
// (iii)+(iv): the HRSS sweep.  One chain per group of G lanes; a warp takes
// 32/G chains of one run from the work queue.
// ---------------------------------------------------------------------------
template <int G>
__device__ void sweep_chain(const Dev& D, const RunDesc& R, RunState* Sw, int j, int gl,
                            unsigned mask, float* zs) {
  const RunState& S = *Sw;
  const float* __restrict__ f = D.f;
  const int d = R.d, ld = R.dpad;
  const bool has = gl * 4 < ld;
  const int parent = D.i[R.o_parent + j];
  const uint32_t iter = (uint32_t)S.iter;
  ChainConst C;
  C.box = R.prior_kind == kPriorBox;
  C.nonflat = !C.box;
  C.lstar = S.logLstar;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int dim = gl * 4 + i;
    C.own[i] = dim < d;
    C.a[i] = C.own[i] ? f[R.o_a + dim] : 0.f;
    C.b[i] = C.own[i] ? f[R.o_b + dim] : 1.f;
  }
  float x[4] = {0.f, 0.f, 0.f, 0.f};
  if (has) {
    const float4 p4 = reinterpret_cast<const float4*>(f + R.o_x + (long long)parent * ld)[gl];
    x[0] = p4.x; x[1] = p4.y; x[2] = p4.z; x[3] = p4.w;
  }
  float lx = f[R.o_logL + parent];
  const float w = R.w;
  const uint32_t nz = 2u * (uint32_t)((d + 1) >> 1);
  const float* Lg = f + R.o_L;
  int evals = 0, acc = 0, nul = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  for (int s = 0; s < R.p; ++s) {
    // direction: z ~ N(0, I), d~ = L z, v = d~ / |z| (or / |d~|)
    const uint4 wb = draw_block(R, iter, (uint32_t)j, (uint32_t)s, (uint32_t)gl);
    float z[4];
    box_muller(wb.x, wb.y, z[0], z[1]);
    box_muller(wb.z, wb.w, z[2], z[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (!C.own[i]) z[i] = 0.0f;
    zs[gl * 4 + 0] = z[0];
    zs[gl * 4 + 1] = z[1];
    zs[gl * 4 + 2] = z[2];
    zs[gl * 4 + 3] = z[3];
    __syncwarp(mask);
    const float zz = gsum<G>(fmaf(z[0], z[0], fmaf(z[1], z[1], fmaf(z[2], z[2], z[3] * z[3]))), mask);
    float dt[4] = {0.f, 0.f, 0.f, 0.f};
    if (has) {
      for (int bb = 0; bb <= gl; ++bb) {
        const float4 zb = reinterpret_cast<const float4*>(zs)[bb];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 l4 = __ldg(reinterpret_cast<const float4*>(Lg + (gl * 4 + r) * ld) + bb);
          dt[r] = fmaf(l4.x, zb.x, fmaf(l4.y, zb.y, fmaf(l4.z, zb.z, fmaf(l4.w, zb.w, dt[r]))));
        }
      }
    }
    __syncwarp(mask);
    float nrm;
    if (R.dir_norm == 0) {
      nrm = sqrtf(zz);
    } else {
      nrm = sqrtf(gsum<G>(fmaf(dt[0], dt[0], fmaf(dt[1], dt[1], fmaf(dt[2], dt[2], dt[3] * dt[3]))), mask));
    }
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = dt[i] / nrm;
    WordCache wc;
    wc.blk = 0xFFFFFFFFu;
    float height = 0.0f;
    if (C.nonflat) {
      const float uh = u24(step_word(R, wc, iter, (uint32_t)j, (uint32_t)s, nz + 1u));
      height = group_logprior<G>(R, C, x, mask) + logf(uh);
    }
    // randomised initial bracket of width w around t = 0
    const float U = u24(step_word(R, wc, iter, (uint32_t)j, (uint32_t)s, nz));
    float tl = -w * U;
    float tr = tl + w;
    float y[4], lly;
    // stepping out, at most 10 expansions per side
    for (int n = 0;; ++n) {
      if (n >= kStepOutCap) { ++capo; break; }
#pragma unroll
      for (int i = 0; i < 4; ++i) y[i] = fmaf(tl, v[i], x[i]);
      ++evals;
      if (!in_slice<G>(R, f, C, y, height, gl, mask, lly, nanc)) break;
      tl -= w;
      ++exps;
    }
    for (int n = 0;; ++n) {
      if (n >= kStepOutCap) { ++capo; break; }
#pragma unroll
      for (int i = 0; i < 4; ++i) y[i] = fmaf(tr, v[i], x[i]);
      ++evals;
      if (!in_slice<G>(R, f, C, y, height, gl, mask, lly, nanc)) break;
      tr += w;
      ++exps;
    }
    // shrinkage, at most 100 proposals, then a null move
    bool ok = false;
    for (int r = 0; r < kShrinkCap; ++r) {
      const float u = u24(step_word(R, wc, iter, (uint32_t)j, (uint32_t)s, nz + 3u + (uint32_t)r));
      const float t = fmaf(u, tr - tl, tl);
#pragma unroll
      for (int i = 0; i < 4; ++i) y[i] = fmaf(t, v[i], x[i]);
      ++evals;
      ++shr;
      if (in_slice<G>(R, f, C, y, height, gl, mask, lly, nanc)) {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = y[i];
        lx = lly;
        ok = true;
        break;
      }
      if (t < 0.0f) tl = t; else tr = t;
    }
    if (ok) ++acc; else ++nul;
  }
  // (iv) replace dead slot j, born at logL*
  const int slot = D.i[R.o_dead + j];
  if (has)
    reinterpret_cast<float4*>(D.f + R.o_x + (long long)slot * ld)[gl] = make_float4(x[0], x[1], x[2], x[3]);
  if (gl == 0) {
    D.f[R.o_logL + slot] = lx;
    D.f[R.o_birth + slot] = C.lstar;
    int* st = D.i + R.o_stats;
    st[j] = evals;
    st[R.k + j] = acc;
    st[2 * R.k + j] = nul;
    st[3 * R.k + j] = exps;
    st[4 * R.k + j] = shr;
    st[5 * R.k + j] = capo;
    atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->evals), (unsigned long long)evals);
    if (nul) atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->nulls), (unsigned long long)nul);
    if (capo) atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->cap_out), (unsigned long long)capo);
    if (nanc) atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->nan_evals), (unsigned long long)nanc);
  }
}

constexpr int kSweepThreads = 128;

template <int G>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(Dev D, const WorkItem* __restrict__ items,
                                                         int n_items, int* queue) {
  __shared__ __align__(16) float zbuf[kSweepThreads / 32][32 * 4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gl = lane % G, grp = lane / G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  float* zs = &zbuf[wid][grp * G * 4];
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const WorkItem wi = items[it];
    RunState* S = D.st + wi.run;
    if (S->done) continue;
    const int j = wi.c0 + grp;
    if (j < wi.c1) sweep_chain<G>(D, D.desc[wi.run], S, j, gl, mask, zs);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Termination (App. B.3, reading: live fraction): Z_live = X mean(L_live);
// stop when Z_live / (Z + Z_live) < tol.  Also counts the iteration.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_terminate(Dev D) {
  const int run = blockIdx.x;
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  __shared__ double red[32];
  const float* logL = D.f + R.o_logL;
  double mx = -INFINITY;
  for (int i = threadIdx.x; i < R.m; i += blockDim.x) mx = fmax(mx, (double)logL[i]);
  mx = block_max_d(mx, red);
  double s = 0.0;
  if (mx > -INFINITY)
    for (int i = threadIdx.x; i < R.m; i += blockDim.x) s += (double)expf((float)((double)logL[i] - mx));
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    const double lzl = (mx > -INFINITY) ? S.logX + mx + log(s) - log((double)R.m) : -INFINITY;
    const double tot = logaddexp_d(S.logZ, lzl);
    const bool stop = (lzl - tot) < log(R.tol);
    S.iter += 1;
    S.stepped = 1;
    if (stop) S.done = 1;
    else if (S.iter >= R.max_iter) { S.done = 1; S.status = -5; }
    if (!isfinite(S.logZ) && S.logZ != -INFINITY) { S.done = 1; S.status = -6; }
  }
}

// ---------------------------------------------------------------------------
// Final live set: kill in (logL, slot) order with n = m, ..., 1 (App. D.2,
// X_{N+1} := 0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_final_sort(Dev D) {
  const int run = blockIdx.x;
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.finalised || S.status == -4) return;
  extern __shared__ __align__(16) char smem[];
  __shared__ double red_d[32];
  __shared__ int cap_fail;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
  const float* logL = D.f + R.o_logL;
  for (int i = threadIdx.x; i < R.m2; i += blockDim.x)
    keys[i] = (i < R.m) ? sort_key(logL[i], i) : ~0ull;
  bitonic_sort(keys, R.m2);
  if (threadIdx.x == 0) cap_fail = (S.n_dead + R.m > R.dead_cap);
  __syncthreads();
  if (cap_fail) {
    if (threadIdx.x == 0) S.status = -4;
    return;
  }
  append_dead(D, R, S, keys, R.m);
  __syncthreads();
  evidence_update(R, S, D.f + R.o_dlogL + S.n_dead, D.dd + R.o_cum, D.dd + R.o_lnd, R.m, red_d);
  if (threadIdx.x == 0) {
    S.n_dead += R.m;
    S.finalised = 1;
  }
}

// ---------------------------------------------------------------------------
// Volume-shrinkage simulation (App. D.2).  Trajectory r draws
// log X_i = log X_{i-1} + log(u_{r,i}) / n_i, u from counter
// (r, i/2, TAG_VOLSIM, 0).  Each term is formed in FP32 (log of a uniform,
// one division) and accumulated in FP64.  Dead points are cut into tiles of
// kVolTile; thread r of a block owns trajectory r of one tile.
// ---------------------------------------------------------------------------
struct VolArgs {
  const int2* tiles;   // (run, first dead index) per tile
  const int* vbase;    // first tile of each run
  int n_tiles, R;
  double* tsum;        // [R][n_tiles] sum of the tile's terms
  double* toff;        // [R][n_tiles] log X before the tile
  double* tmax;        // [R][n_tiles] running log-sum-exp max of log w
  double* tacc;        // [R][n_tiles] running log-sum-exp sum
};

__device__ __forceinline__ float vol_term(const RunDesc& R, int r, long long i, int n) {
  const uint4 b = draw_block(R, (uint32_t)r, (uint32_t)(i >> 1), kTagVolsim, 0u);
  const double u = (i & 1) ? u53(b.z, b.w) : u53(b.x, b.y);
  return logf((float)u) / (float)n;
}

__global__ void k_vol_tilesum(Dev D, VolArgs A) {
  const int tile = blockIdx.x, r = threadIdx.x;
  if (r >= A.R) return;
  const int2 t = A.tiles[tile];
  const RunDesc& R = D.desc[t.x];
  const long long n = D.st[t.x].n_dead;
  const long long i0 = t.y, i1 = min((long long)t.y + kVolTile, n);
  double s = 0.0;
  const int* nl = D.i + R.o_dn;
  for (long long i = i0; i < i1; ++i) s += (double)vol_term(R, r, i, nl[i]);
  A.tsum[(size_t)r * A.n_tiles + tile] = s;
}

// exclusive scan of tile sums per (run, trajectory); tiles of a run are
// contiguous starting at vbase[run]
__global__ void k_vol_scan(Dev D, VolArgs A, int n_runs) {
  const int run = blockIdx.x, r = threadIdx.x;
  if (r >= A.R || run >= n_runs) return;
  const RunDesc& R = D.desc[run];
  const long long n = D.st[run].n_dead;
  const int nt = (int)((n + kVolTile - 1) / kVolTile);
  double acc = 0.0;
  for (int q = 0; q < nt; ++q) {
    const size_t o = (size_t)r * A.n_tiles + A.vbase[run] + q;
    A.toff[o] = acc;
    acc += A.tsum[o];
  }
}

// per tile: log w_i^(r) = logL_i + log dX_i^(r) (trapezoid), the running
// log-sum-exp of each trajectory, and the mean over r of log dX_i.
__global__ void k_vol_weights(Dev D, VolArgs A) {
  extern __shared__ double sh[];  // [R][32]
  const int tile = blockIdx.x, r = threadIdx.x;
  const int2 t = A.tiles[tile];
  const RunDesc& R = D.desc[t.x];
  const long long n = D.st[t.x].n_dead;
  const long long i0 = t.y, i1 = min((long long)t.y + kVolTile, n);
  const int* nl = D.i + R.o_dn;
  const float* lL = D.f + R.o_dlogL;
  double* lw = D.dd + R.o_lw;
  const bool act = r < A.R;
  double prev = act ? A.toff[(size_t)r * A.n_tiles + tile] : 0.0;  // log X_{i-1}
  double cur = act ? prev + (double)vol_term(R, r, i0, nl[i0]) : 0.0;
  double M = -INFINITY, Sacc = 0.0;
  const double ln2 = 0.69314718055994530942;
  for (long long c0 = i0; c0 < i1; c0 += 32) {
    const int cn = (int)min((long long)32, i1 - c0);
    if (act) {
      for (int q = 0; q < cn; ++q) {
        const long long i = c0 + q;
        double nxt = -INFINITY;
        if (i + 1 < n) nxt = cur + (double)vol_term(R, r, i + 1, nl[i + 1]);
        const double ldx = prev + (double)logf(-expm1f((float)(nxt - prev))) - ln2;
        const double v = (double)lL[i] + ldx;
        if (v == -INFINITY) {
          // a point outside every constraint set carries no weight
        } else if (v > M) {
          Sacc = Sacc * (double)expf((float)(M - v)) + 1.0;
          M = v;
        } else {
          Sacc += (double)expf((float)(v - M));
        }
        sh[r * 32 + q] = ldx;
        prev = cur;
        cur = nxt;
      }
    }
    __syncthreads();
    if (threadIdx.x < cn) {
      double s = 0.0;
      for (int q = 0; q < A.R; ++q) s += sh[q * 32 + threadIdx.x];
      lw[c0 + threadIdx.x] = (double)lL[c0 + threadIdx.x] + s / (double)A.R;
    }
    __syncthreads();
  }
  if (act) {
    A.tmax[(size_t)r * A.n_tiles + tile] = M;
    A.tacc[(size_t)r * A.n_tiles + tile] = Sacc;
  }
}

// per run: log Z^(r), their mean and standard deviation, the weight norm
__global__ void k_vol_final(Dev D, VolArgs A, int n_runs) {
  const int run = blockIdx.x;
  if (run >= n_runs) return;
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  __shared__ double red[32];
  __shared__ double lz[1024];
  const long long n = S.n_dead;
  const int nt = (int)((n + kVolTile - 1) / kVolTile);
  for (int r = threadIdx.x; r < A.R; r += blockDim.x) {
    double M = -INFINITY;
    for (int q = 0; q < nt; ++q) M = fmax(M, A.tmax[(size_t)r * A.n_tiles + A.vbase[run] + q]);
    double s = 0.0;
    for (int q = 0; q < nt; ++q) {
      const size_t o = (size_t)r * A.n_tiles + A.vbase[run] + q;
      if (A.tmax[o] > -INFINITY) s += A.tacc[o] * exp(A.tmax[o] - M);
    }
    lz[r] = M + log(s);
  }
  __syncthreads();
  double mean = 0.0;
  for (int r = threadIdx.x; r < A.R; r += blockDim.x) mean += lz[r];
  mean = block_sum_d(mean, red) / A.R;
  double var = 0.0;
  for (int r = threadIdx.x; r < A.R; r += blockDim.x) var += (lz[r] - mean) * (lz[r] - mean);
  var = block_sum_d(var, red) / (A.R > 1 ? A.R - 1 : 1);
  // normalisation of the geometric-mean weights
  const double* lw = D.dd + R.o_lw;
  double mx = -INFINITY;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, lw[i]);
  mx = block_max_d(mx, red);
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)expf((float)(lw[i] - mx));
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    S.logZ_mean = mean;
    S.logZ_std = sqrt(var);
    S.lw_norm = mx + log(s);
  }
}

__global__ void k_vol_norm(Dev D, int run) {
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  double* lw = D.dd + R.o_lw;
  const double c = S.lw_norm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n_dead;
       i += (long long)gridDim.x * blockDim.x)
    lw[i] -= c;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int G>
static cudaError_t launch_init_t(const Dev& D, const WorkItem* items, int n, cudaStream_t s) {
  const int blocks = (n * 32 + 127) / 128;
  k_init<G><<<blocks > 0 ? blocks : 1, 128, 0, s>>>(D, items, n);
  return cudaGetLastError();
}

cudaError_t launch_init(int cls, const Dev& D, const WorkItem* items, int n, cudaStream_t s) {
  switch (cls) {
    case 0: return launch_init_t<1>(D, items, n, s);
    case 1: return launch_init_t<2>(D, items, n, s);
    case 2: return launch_init_t<4>(D, items, n, s);
    case 3: return launch_init_t<8>(D, items, n, s);
    case 4: return launch_init_t<16>(D, items, n, s);
    default: return launch_init_t<32>(D, items, n, s);
  }
}

cudaError_t launch_prologue(const Dev& D, int n_runs, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_prologue, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_final_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_prologue<<<n_runs, 1024, smem, s>>>(D);
  return cudaGetLastError();
}

template <int G>
static cudaError_t launch_sweep_t(const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                                  cudaStream_t s) {
  k_sweep<G><<<grid, kSweepThreads, 0, s>>>(D, items, n, queue);
  return cudaGetLastError();
}

int sweep_blocks_per_sm(int cls) {
  int nb = 0;
  switch (cls) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<1>, kSweepThreads, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<2>, kSweepThreads, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<4>, kSweepThreads, 0); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<8>, kSweepThreads, 0); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<16>, kSweepThreads, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<32>, kSweepThreads, 0); break;
  }
  return nb > 0 ? nb : 1;
}

cudaError_t launch_sweep(int cls, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                         cudaStream_t s) {
  switch (cls) {
    case 0: return launch_sweep_t<1>(D, items, n, queue, grid, s);
    case 1: return launch_sweep_t<2>(D, items, n, queue, grid, s);
    case 2: return launch_sweep_t<4>(D, items, n, queue, grid, s);
    case 3: return launch_sweep_t<8>(D, items, n, queue, grid, s);
    case 4: return launch_sweep_t<16>(D, items, n, queue, grid, s);
    default: return launch_sweep_t<32>(D, items, n, queue, grid, s);
  }
}

cudaError_t launch_terminate(const Dev& D, int n_runs, cudaStream_t s) {
  k_terminate<<<n_runs, 256, 0, s>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_final_sort(const Dev& D, int n_runs, size_t smem, cudaStream_t s) {
  k_final_sort<<<n_runs, 1024, smem, s>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_volsim(const Dev& D, const VolLaunch& V, int n_runs, cudaStream_t s) {
  VolArgs A;
  A.tiles = V.tiles;
  A.vbase = V.vbase;
  A.n_tiles = V.n_tiles;
  A.R = V.R;
  A.tsum = V.tsum;
  A.toff = V.toff;
  A.tmax = V.tmax;
  A.tacc = V.tacc;
  const int bt = (V.R + 31) / 32 * 32;
  k_vol_tilesum<<<V.n_tiles, bt, 0, s>>>(D, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_vol_scan<<<n_runs, bt, 0, s>>>(D, A, n_runs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_vol_weights<<<V.n_tiles, bt, (size_t)bt * 32 * sizeof(double), s>>>(D, A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_vol_final<<<n_runs, 256, 0, s>>>(D, A, n_runs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int r = 0; r < n_runs; ++r) {
    k_vol_norm<<<64, 256, 0, s>>>(D, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nss
