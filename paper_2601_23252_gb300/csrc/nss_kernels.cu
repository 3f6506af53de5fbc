// nss_kernels.cu -- the Nested Slice Sampling kernels for sm_103a.
//
// Per outer iteration (Sec. 3.1 (i)-(iv); Algorithm 1):
//   k_prologue  two blocks per run: one selects the k worst live points by a
//               bitonic sort of (logL, slot) keys, threshold logL*, survivors
//               in slot order, parents, dead-point append, unrolled evidence
//               update (FP64 accumulation); the other forms the live-set
//               covariance and its Cholesky factor (the direction metric,
//               Sec. 3.2).
//   k_sweep     (nss_sweep.cu) the HRSS sweep with the likelihood fused in.
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

// Append `cnt` dead slots, worst first, to the dead store; slot_of(j) is
// the j-th dead slot.
template <class SlotOf>
__device__ void append_dead_by(const Dev& D, const RunDesc& R, RunState& S, SlotOf slot_of, int cnt) {
  const long long base = S.n_dead;
  const int q4 = R.dpad >> 2;
  const float4* xs = reinterpret_cast<const float4*>(D.f + R.o_x);
  float4* xd = reinterpret_cast<float4*>(D.f + R.o_dx + base * R.dpad);
  for (int t = threadIdx.x; t < cnt * q4; t += blockDim.x) {
    const int j = t / q4, c = t - j * q4;
    const int slot = slot_of(j);
    xd[(long long)j * q4 + c] = xs[(long long)slot * q4 + c];
  }
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int slot = slot_of(j);
    D.f[R.o_dlogL + base + j] = D.f[R.o_logL + slot];
    D.f[R.o_dbirth + base + j] = D.f[R.o_birth + slot];
    D.i[R.o_dn + base + j] = R.m - j;
  }
}

// ... from the first `cnt` entries of the sorted key list
__device__ void append_dead(const Dev& D, const RunDesc& R, RunState& S,
                            const unsigned long long* keys, int cnt) {
  append_dead_by(D, R, S, [keys](int j) { return (int)(keys[j] & 0xffffffffu); }, cnt);
}

// Cholesky factor of S + reg I ([ld][ld] in shared memory) into Lm
// ([ld][ld + 1]) by the whole block: right-looking column steps with one
// block barrier each.  At step j the warps take the rows i > j and their
// lanes the columns j < q <= i, A_iq -= (A_ij / l_jj)(A_qj / l_jj), while
// column j - 1 (read by no thread of this step) is scaled to its final
// values.  Every thread of the block calls it; returns true (for every
// thread) on a non-positive or non-finite pivot.
__device__ bool cholesky_block(const float* S, float* Lm, int d, int ld, float reg) {
  const int lw = ld + 1, T = blockDim.x, nw = T >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < ld * ld; t += T) {
    const int a = t / ld, b = t - a * ld;
    Lm[a * lw + b] = (b <= a && a < d) ? S[t] + (a == b ? reg : 0.0f) : 0.0f;
  }
  __syncthreads();
  bool bad = false;
  float lprev = 0.0f, iprev = 0.0f;
  for (int j = 0; j < d; ++j) {
    const float piv = Lm[j * lw + j];
    bad = !(piv > 0.0f) || !isfinite(piv);  // the same in every thread
    if (bad) break;
    const float ljj = sqrtf(piv), inv = 1.0f / ljj;
    for (int i = j + 1 + wid; i < d; i += nw) {
      const float lij = Lm[i * lw + j] * inv;
      for (int q = j + 1 + lane; q <= i; q += 32) Lm[i * lw + q] = fmaf(-lij, Lm[q * lw + j] * inv, Lm[i * lw + q]);
    }
    if (j > 0)
      for (int i = j - 1 + threadIdx.x; i < d; i += T)
        Lm[i * lw + j - 1] = (i == j - 1) ? lprev : Lm[i * lw + j - 1] * iprev;
    lprev = ljj;
    iprev = inv;
    __syncthreads();
  }
  if (!bad && threadIdx.x == 0) Lm[(d - 1) * lw + d - 1] = lprev;
  __syncthreads();
  return bad;
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
  __shared__ double red_s[32];
  float* part = reinterpret_cast<float*>(smem);
  // mean of x - x_0 per dimension
  const int nparts = T / ld;
  {
    const int a = threadIdx.x % ld, pi = threadIdx.x / ld;
    float s = 0.0f;
    if (pi < nparts && a < d) {
      const float ref = X[a];
#pragma unroll 4
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
  float* Lm = Sm + ld * ld;                      // [ld][ld + 1]
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
#pragma unroll 2
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
      fail = cholesky_block(Sm, Lm, d, ld, reg);
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
    Lg[t] = identity ? ((a == b && a < d) ? 1.0f : 0.0f) : Lm[a * (ld + 1) + b];
  }
  if (threadIdx.x == 0) S.metric_status = status;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Iteration prologue: steps (i), (ii), evidence and metric for one run.
// ---------------------------------------------------------------------------
// Two blocks per run: the even one selects, records the dead points, updates
// the evidence and draws the parents; the odd one forms the direction metric
// of the same live set (the two read the live set as the iteration starts
// and write disjoint state), so their chains of block barriers overlap.
__global__ void __launch_bounds__(kPrologueThreads) k_prologue(Dev D, int run0) {
  const int run = run0 + (blockIdx.x >> 1);
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  extern __shared__ __align__(16) char smem[];
  if (blockIdx.x & 1) {
    live_metric(D, R, S, smem);
    return;
  }
  __shared__ double red_d[32];
  __shared__ int red_i[32];
  __shared__ int cap_fail;
  const int m = R.m, k = R.k, m2 = R.m2;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
  int* surv = reinterpret_cast<int*>(smem + (size_t)m2 * 8);
  const float* logL = D.f + R.o_logL;
  for (int i = threadIdx.x; i < m2; i += blockDim.x)
    keys[i] = (i < m) ? sort_key(logL[i], i) : ~0ull;
  if (m2 <= (int)blockDim.x) bitonic_sort_reg(keys, m2);
  else bitonic_sort(keys, m2);
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
}

// ---------------------------------------------------------------------------
// The plain single-run path: the prologue's phases as separate kernels, one
// block of kPrologueThreads threads each, calling the same device functions
// (so every reduction runs in the same order and the results are
// bit-identical to k_prologue's).
// ---------------------------------------------------------------------------
// (i) selection: dead slots worst first, logL*, survivors in slot order
__global__ void __launch_bounds__(kPrologueThreads) k_plain_select(Dev D, int run) {
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  extern __shared__ __align__(16) char smem[];
  __shared__ int red_i[32];
  __shared__ int cap_fail;
  const int m = R.m, k = R.k, m2 = R.m2;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
  int* flag = reinterpret_cast<int*>(smem + (size_t)m2 * 8);
  const float* logL = D.f + R.o_logL;
  for (int i = threadIdx.x; i < m2; i += blockDim.x) keys[i] = (i < m) ? sort_key(logL[i], i) : ~0ull;
  if (m2 <= (int)blockDim.x) bitonic_sort_reg(keys, m2);
  else bitonic_sort(keys, m2);
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
  for (int i = threadIdx.x; i < m; i += blockDim.x) flag[i] = 1;
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) flag[(int)(keys[j] & 0xffffffffu)] = 0;
  __syncthreads();
  int* surv = D.i + R.o_surv;
  const int per = (m + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per;
  int c = 0;
  for (int i = i0; i < min(i0 + per, m); ++i) c += flag[i];
  int tot;
  int pos = block_exscan_i(c, red_i, &tot);
  for (int i = i0; i < min(i0 + per, m); ++i)
    if (flag[i]) surv[pos++] = i;
}

// dead-point append and the unrolled evidence update
__global__ void __launch_bounds__(kPrologueThreads) k_plain_evidence(Dev D, int run) {
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  __shared__ double red_d[32];
  const int* dead = D.i + R.o_dead;
  append_dead_by(D, R, S, [dead](int j) { return dead[j]; }, R.k);
  __syncthreads();
  evidence_update(R, S, D.f + R.o_dlogL + S.n_dead, D.dd + R.o_cum, D.dd + R.o_lnd, R.k, red_d);
  if (threadIdx.x == 0) S.n_dead += R.k;
}

// direction metric of the live set at the start of the iteration
__global__ void __launch_bounds__(kPrologueThreads) k_plain_metric(Dev D, int run) {
  const RunDesc& R = D.desc[run];
  RunState& S = D.st[run];
  if (S.done) return;
  extern __shared__ __align__(16) char smem[];
  live_metric(D, R, S, smem);
}

// (ii) parents uniformly with replacement among the m-k survivors
__global__ void k_plain_parents(Dev D, int run) {
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  if (S.done) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R.k) return;
  const uint32_t w = draw_block(R, (uint32_t)S.iter, (uint32_t)j, kTagParent, 0u).x;
  D.i[R.o_parent + j] = D.i[R.o_surv + __umulhi(w, (uint32_t)(R.m - R.k))];
}

// ---------------------------------------------------------------------------
// Termination (App. B.3, reading: live fraction): Z_live = X mean(L_live);
// stop when Z_live / (Z + Z_live) < tol.  Also counts the iteration.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_terminate(Dev D, int run0) {
  const int run = run0 + blockIdx.x;
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
  if (R.m2 <= (int)blockDim.x) bitonic_sort_reg(keys, R.m2);
  else bitonic_sort(keys, R.m2);
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
  int run0;            // block b of the per-run kernels serves run run0 + b
  double* tsum;        // [R][n_tiles] sum of the tile's terms
  double* toff;        // [R][n_tiles] log X before the tile
  double* tmax;        // [R][n_tiles] running log-sum-exp max of log w
  double* tacc;        // [R][n_tiles] running log-sum-exp sum
  // reweighting (one run): logL read from logL_in and the weights and
  // statistics written to lw_out / stats_out instead of the run's own store
  const float* logL_in;
  double* lw_out;
  double* stats_out;   // logZ mean, std, weight norm
};

__global__ void k_vol_tilesum(Dev D, VolArgs A) {
  const int tile = blockIdx.x, r = threadIdx.x;
  if (r >= A.R) return;
  const int2 t = A.tiles[tile];
  const RunDesc& R = D.desc[t.x];
  const long long n = D.st[t.x].n_dead;
  const long long i0 = t.y, i1 = min((long long)t.y + kVolTile, n);
  double s = 0.0;
  const int* nl = D.i + R.o_dn;
  uint4 blk;
  long long bi = -1;
  for (long long i = i0; i < i1; ++i) s += (double)vol_term_f(R.key0, R.key1, r, i, nl[i], blk, bi);
  A.tsum[(size_t)r * A.n_tiles + tile] = s;
}

// exclusive scan of tile sums per (run, trajectory); tiles of a run are
// contiguous starting at vbase[run]
__global__ void k_vol_scan(Dev D, VolArgs A, int n_runs) {
  const int run = A.run0 + blockIdx.x, r = threadIdx.x;
  if (r >= A.R || run >= n_runs) return;
  const long long n = D.st[run].n_dead;
  const int nt = (int)((n + kVolTile - 1) / kVolTile);
  double acc = 0.0;
  for (int q = 0; q < nt; ++q) {
    const size_t o = (size_t)r * A.n_tiles + A.vbase[run] + q;
    A.toff[o] = acc;
    acc += A.tsum[o];
  }
}

// per tile: log w_i^(r) = logL_i + log dX_i^(r) (trapezoid), the tile's part
// of each trajectory's log-sum-exp, and the mean over r of log dX_i.
//
// Within a tile everything is relative to two references, so the per-term
// work stays in FP32: log X at the tile start (FP64, from the scan) and the
// tile's largest logL.  rel_i = log dX_i - log X(start) sums the terms from
// the tile start (compensated FP32 sum) and the trapezoid factor; since
// log X only decreases and the factor is below 1/2, every log w_i is at most
// M = max logL + log X(start), and the tile's sum is sum exp(log w_i - M)
// with FP32 exponents accumulated in FP64.
__global__ void k_vol_weights(Dev D, VolArgs A) {
  extern __shared__ float shf[];  // [R][32] rel_i of the current chunk
  __shared__ double red[32];
  __shared__ double part_s[32 * 32];
  const int tile = blockIdx.x, r = threadIdx.x;
  const int2 t = A.tiles[tile];
  const RunDesc& R = D.desc[t.x];
  const long long n = D.st[t.x].n_dead;
  const long long i0 = t.y, i1 = min((long long)t.y + kVolTile, n);
  const int* nl = D.i + R.o_dn;
  const float* lL = A.logL_in ? A.logL_in : D.f + R.o_dlogL;
  double* lw = A.lw_out ? A.lw_out : D.dd + R.o_lw;
  const bool act = r < A.R;
  // the tile's largest logL, and the mean over r of log X at the tile start
  float lm = -INFINITY;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) lm = fmaxf(lm, lL[i]);
  lm = (float)block_max_d((double)lm, red);
  const double start = act ? A.toff[(size_t)r * A.n_tiles + tile] : 0.0;
  const double start_mean = block_sum_d(start, red) / (double)A.R;
  uint4 blk;
  long long bi = -1;
  float off = 0.0f, comp = 0.0f;  // log X_{i-1} - log X(start), compensated
  float tcur = act ? vol_term_f(R.key0, R.key1, r, i0, nl[i0], blk, bi) : 0.0f;
  double Sacc = 0.0;
  const float ln2f = 0.693147182f;
  for (long long c0 = i0; c0 < i1; c0 += 32) {
    const int cn = (int)min((long long)32, i1 - c0);
    if (act) {
      for (int q = 0; q < cn; ++q) {
        const long long i = c0 + q;
        const float tnxt = (i + 1 < n) ? vol_term_f(R.key0, R.key1, r, i + 1, nl[i + 1], blk, bi) : -INFINITY;
        // (X_{i-1} - X_{i+1}) / 2 = X_{i-1} (1 - e^{t_i + t_{i+1}}) / 2  (t_{N+1} = -inf: X_{N+1} = 0)
        const float rel = off + (logf(-expm1f(tcur + tnxt)) - ln2f);
        const float li = lL[i];
        // a point outside every constraint set carries no weight
        if (li > -INFINITY) Sacc += (double)expf((li - lm) + rel);
        shf[r * 32 + q] = rel;
        const float y = tcur - comp, tt = off + y;
        comp = (tt - off) - y;
        off = tt;
        tcur = tnxt;
      }
    }
    __syncthreads();
    // mean over the trajectories: one partial sum per warp and dead point,
    // then the partials combined in warp order
    {
      const int pt = threadIdx.x & 31, part = threadIdx.x >> 5, P = blockDim.x >> 5;
      double sp = 0.0;
      if (pt < cn)
        for (int q = part; q < A.R; q += P) sp += (double)shf[q * 32 + pt];
      part_s[part * 32 + pt] = sp;
      __syncthreads();
      if (threadIdx.x < cn) {
        double tot = 0.0;
        for (int q = 0; q < P; ++q) tot += part_s[q * 32 + threadIdx.x];
        lw[c0 + threadIdx.x] = (double)lL[c0 + threadIdx.x] + (start_mean + tot / (double)A.R);
      }
    }
    __syncthreads();
  }
  if (act) {
    A.tmax[(size_t)r * A.n_tiles + tile] = (lm > -INFINITY && Sacc > 0.0) ? (double)lm + start : -INFINITY;
    A.tacc[(size_t)r * A.n_tiles + tile] = Sacc;
  }
}

// per run: log Z^(r), their mean and standard deviation, the weight norm
__global__ void k_vol_final(Dev D, VolArgs A, int n_runs) {
  const int run = A.run0 + blockIdx.x;
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
  const double* lw = A.lw_out ? A.lw_out : D.dd + R.o_lw;
  double mx = -INFINITY;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, lw[i]);
  mx = block_max_d(mx, red);
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)expf((float)(lw[i] - mx));
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    if (A.stats_out) {
      A.stats_out[0] = mean;
      A.stats_out[1] = sqrt(var);
      A.stats_out[2] = mx + log(s);
    } else {
      S.logZ_mean = mean;
      S.logZ_std = sqrt(var);
      S.lw_norm = mx + log(s);
    }
  }
}

__global__ void k_vol_norm(Dev D, int run, double* lw_out, const double* stats_out) {
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  double* lw = lw_out ? lw_out : D.dd + R.o_lw;
  const double c = stats_out ? stats_out[2] : S.lw_norm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n_dead;
       i += (long long)gridDim.x * blockDim.x)
    lw[i] -= c;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t setup_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_prologue, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_plain_select, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_plain_metric, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  // up to 1024 trajectories: [1024][32] FP32 offsets
  e = cudaFuncSetAttribute(k_vol_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, 1024 * 32 * (int)sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_final_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_prologue(const Dev& D, int run0, int n_runs, size_t smem, cudaStream_t s) {
  k_prologue<<<2 * n_runs, kPrologueThreads, smem, s>>>(D, run0);
  return cudaGetLastError();
}

cudaError_t launch_plain_phase(int phase, const Dev& D, int run, int k, size_t smem, cudaStream_t s) {
  switch (phase) {
    case 0: k_plain_select<<<1, kPrologueThreads, smem, s>>>(D, run); break;
    case 1: k_plain_evidence<<<1, kPrologueThreads, 0, s>>>(D, run); break;
    case 2: k_plain_metric<<<1, kPrologueThreads, smem, s>>>(D, run); break;
    case 3: k_plain_parents<<<(k + 255) / 256, 256, 0, s>>>(D, run); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_terminate(const Dev& D, int run0, int n_runs, cudaStream_t s) {
  k_terminate<<<n_runs, 256, 0, s>>>(D, run0);
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
  A.logL_in = V.logL_in;
  A.lw_out = V.lw_out;
  A.stats_out = V.stats_out;
  // one run (reweighting) or all of them
  const bool one = V.run >= 0;
  A.run0 = one ? V.run : 0;
  const int nb = one ? 1 : n_runs;
  const int bt = (V.R + 31) / 32 * 32;
  k_vol_tilesum<<<V.n_tiles, bt, 0, s>>>(D, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_vol_scan<<<nb, bt, 0, s>>>(D, A, n_runs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_vol_weights<<<V.n_tiles, bt, (size_t)bt * 32 * sizeof(float), s>>>(D, A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_vol_final<<<nb, 256, 0, s>>>(D, A, n_runs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int r = A.run0; r < A.run0 + nb; ++r) {
    k_vol_norm<<<64, 256, 0, s>>>(D, r, A.lw_out, A.stats_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nss
