// nss_sweep.cu -- the initial prior draw (Sec. 2.1) in the sweep's lane
// layout, and the dispatch of the HRSS sweep over its configurations
// (nss_sweep_chain.cuh, nss_sweep_lane.cu), for sm_103a.
//
// A slot is owned by a group of G lanes of one warp; lane gl holds the DPL
// dimensions [gl*DPL, gl*DPL + DPL) of the point.  The likelihood of a draw
// is a group reduction (xor butterflies: every lane ends with the same value).
#include "nss_sweep_common.cuh"

namespace nss {

// ---- likelihood of a chain group ------------------------------------------
template <int G, int DPL>
struct Lik {
  float mu4[4][DPL];   // cached means of up to four mixture components
  bool cached;

  __device__ __forceinline__ void init(const RunDesc& R, const float* __restrict__ f, int gl, bool has) {
    cached = (R.lik_kind == kLikGmm && R.n_comp <= 4) || R.lik_kind == kLikGauss || R.lik_kind == kLikFault;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int i = 0; i < DPL; ++i) mu4[c][i] = 0.0f;
    if (!cached || !has) return;
    const int nc = (R.lik_kind == kLikGmm) ? R.n_comp : 1;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < nc) ldg_lane<DPL>(f + R.o_mu + (long long)c * R.dpad, gl, R.dpad, mu4[c]);
  }

  __device__ __forceinline__ static float sqdist(const float (&y)[DPL], const float (&m)[DPL]) {
    float q = 0.0f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
      const float e = y[i] - m[i];
      q = fmaf(e, e, q);
    }
    return q;
  }

  __device__ __forceinline__ float eval(const RunDesc& R, const float* __restrict__ f, const float (&y)[DPL],
                                        int gl, bool has, unsigned mask) const {
    const int lk = R.lik_kind;
    if (lk == kLikFlat) return 0.0f;
    if (lk == kLikRastrigin) {
      // App. F.3: alpha exp(-|y|^2/2) + (1 - alpha) exp(-A d + A sum cos(2 pi y_i)), A = 10
      float q = 0.0f, cs = 0.0f;
#pragma unroll
      for (int i = 0; i < DPL; ++i)
        if (has && gl * DPL + i < R.d) {
          q = fmaf(y[i], y[i], q);
          cs += cospif(2.0f * y[i]);
        }
      q = gsum<G>(q, mask);
      cs = gsum<G>(cs, mask);
      const float a1 = R.ras_la - 0.5f * q, a2 = R.ras_l1a + fmaf(10.0f, cs, -10.0f * (float)R.d);
      const float hi = fmaxf(a1, a2), lo = fminf(a1, a2);
      return (hi == -INFINITY) ? -INFINITY : hi + log1pf(expf(lo - hi));
    }
    if (lk == kLikGauss || lk == kLikFault) {
      const float q = gsum<G>(has ? sqdist(y, mu4[0]) : 0.0f, mask);
      float ll = fmaf(-q, R.inv2s2, R.lognorm);
      if (lk == kLikFault) {
        const float x0 = __shfl_sync(mask, y[0], 0, G);
        if (x0 < R.fault_param) ll = (R.fault_mode == 1) ? __int_as_float(0x7fc00000) : INFINITY;
      }
      return ll;
    }
    if constexpr (G >= 4) {
      if (R.n_comp == 4) {
        // four components: transposed butterfly.  After two exchange levels
        // lane gl holds the partial of component (gl & G/2 ? 2 : 0) +
        // (gl & G/4 ? 1 : 0); the remaining levels finish its sum.
        float q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = has ? sqdist(y, mu4[c]) : 0.0f;
        const bool h1 = gl & (G / 2);
        const float r0 = __shfl_xor_sync(mask, h1 ? q[0] : q[2], G / 2, G);
        const float r1 = __shfl_xor_sync(mask, h1 ? q[1] : q[3], G / 2, G);
        const float k0 = (h1 ? q[2] : q[0]) + r0;
        const float k1 = (h1 ? q[3] : q[1]) + r1;
        const bool h2 = gl & (G / 4);
        const float r2 = __shfl_xor_sync(mask, h2 ? k0 : k1, G / 4, G);
        float s = (h2 ? k1 : k0) + r2;
#pragma unroll
        for (int o = G / 8; o > 0; o >>= 1) s += __shfl_xor_sync(mask, s, o, G);
        const float v = -s * R.inv2s2;
        float M = fmaxf(v, __shfl_xor_sync(mask, v, G / 2, G));
        M = fmaxf(M, __shfl_xor_sync(mask, M, G / 4, G));
        float e = __expf(v - M);
        e += __shfl_xor_sync(mask, e, G / 2, G);
        e += __shfl_xor_sync(mask, e, G / 4, G);
        return M + __logf(e) + R.lognorm;
      }
    }
    // general mixture: one reduction per component, online log-sum-exp
    float M = -INFINITY, S = 0.0f;
    const int K = R.n_comp;
    if (cached) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < K) {
          const float q = gsum<G>(has ? sqdist(y, mu4[c]) : 0.0f, mask);
          const float v = -q * R.inv2s2;
          if (v > M) {
            S = S * expf(M - v) + 1.0f;
            M = v;
          } else {
            S += expf(v - M);
          }
        }
      }
    } else {
      for (int c = 0; c < K; ++c) {
        float mq[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) mq[i] = 0.0f;
        if (has) ldg_lane<DPL>(f + R.o_mu + (long long)c * R.dpad, gl, R.dpad, mq);
        const float q = gsum<G>(has ? sqdist(y, mq) : 0.0f, mask);
        const float v = -q * R.inv2s2;
        if (v > M) {
          S = S * expf(M - v) + 1.0f;
          M = v;
        } else {
          S += expf(v - M);
        }
      }
    }
    return M + logf(S) + R.lognorm;
  }
};

// ---------------------------------------------------------------------------
// Initial live set (Sec. 2.1): slot s draws x ~ Pi from counter
// (0, s, TAG_INIT, word/4) -- box: x_i = a_i + (b_i - a_i) u(word i);
// Gaussian: x_i = a_i + b_i z_i with Box-Muller pairs.
// ---------------------------------------------------------------------------
template <int G, int DPL>
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
    const bool has = gl * DPL < R.dpad;
    float x[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) x[i] = 0.0f;
    if (R.prior_kind == kPriorBox) {
      uint32_t u[DPL];
      lane_uniform_words<DPL>(R, 0u, (uint32_t)slot, kTagInit, gl, u);
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        const int dim = gl * DPL + i;
        if (dim < R.d) {
          const float a = D.f[R.o_a + dim], b = D.f[R.o_b + dim];
          x[i] = fmaf(b - a, u24(u[i]), a);
        }
      }
    } else {
      float z[DPL];
      lane_normals<DPL>(R, 0u, (uint32_t)slot, kTagInit, gl, z);
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        const int dim = gl * DPL + i;
        if (dim < R.d) x[i] = fmaf(D.f[R.o_b + dim], z[i], D.f[R.o_a + dim]);
      }
    }
    float ll = 0.0f;  // logistic regression and GP: filled by their own init pass
    if (R.lik_kind != kLikLogreg && R.lik_kind != kLikGp) {
      Lik<G, DPL> L;
      L.init(R, D.f, gl, has);
      ll = L.eval(R, D.f, x, gl, has, mask);
      if (isnan(ll)) ll = -INFINITY;
    }
    if (has) store_lane<DPL>(D.f + R.o_x + (long long)slot * R.dpad, gl, R.dpad, x);
    if (gl == 0) {
      D.f[R.o_logL + slot] = ll;
      D.f[R.o_birth + slot] = -INFINITY;
    }
  }
}

// ---------------------------------------------------------------------------
// configuration table and launchers
// ---------------------------------------------------------------------------
int cfg_g(int cfg) {
  if (cfg >= kLaneCfg0) return 1;
#define X(id, g, p) if (cfg == id) return g;
  NSS_CFGS(X)
#undef X
  return 32;
}

int cfg_dpl(int cfg) {
  if (cfg >= kLaneCfg0) return lane_dmax(cfg);
#define X(id, g, p) if (cfg == id) return p;
  NSS_CFGS(X)
#undef X
  return 4;
}

cudaError_t launch_init(int cfg, const Dev& D, const WorkItem* items, int n, cudaStream_t s) {
  const int blocks = (n * 32 + 127) / 128;
  switch (cfg) {
#define X(id, g, p) case id: k_init<g, p><<<blocks > 0 ? blocks : 1, 128, 0, s>>>(D, items, n); break;
    NSS_CFGS(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int sweep_warps_per_block(int cfg) { return cfg >= kLaneCfg0 ? sweep_lane_warps_per_block() : kSweepThreads / 32; }

template <int KC>
cudaError_t launch_sweep_kc(int cfg, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                            cudaStream_t s);
template <int KC>
int sweep_blocks_per_sm_kc(int cfg);

int sweep_blocks_per_sm(int cfg, int kc) {
  if (cfg >= kLaneCfg0) return sweep_lane_blocks_per_sm(lane_dmax(cfg), kc);
  return kc == 1 ? sweep_blocks_per_sm_kc<1>(cfg) : kc == 4 ? sweep_blocks_per_sm_kc<4>(cfg)
                                                            : sweep_blocks_per_sm_kc<8>(cfg);
}

cudaError_t launch_sweep(int cfg, int kc, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                         cudaStream_t s) {
  if (cfg >= kLaneCfg0) return launch_sweep_lane(lane_dmax(cfg), kc, D, items, n, queue, grid, s);
  switch (kc) {
    case 1: return launch_sweep_kc<1>(cfg, D, items, n, queue, grid, s);
    case 4: return launch_sweep_kc<4>(cfg, D, items, n, queue, grid, s);
    case 8: return launch_sweep_kc<8>(cfg, D, items, n, queue, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int sweep_kc(int lik_kind, int n_comp) {
  if (lik_kind == kLikGmm) return n_comp <= 1 ? 1 : n_comp <= 4 ? 4 : 8;
  return 1;
}

}  // namespace nss
