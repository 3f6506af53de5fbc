// nss_sweep.cu -- the Hit-and-Run Slice Sampling sweep (steps (iii)+(iv) of
// Sec. 3.1; HRSS of Sec. 3.2 and App. B.4) and the initial prior draw, for
// sm_103a.
//
// A chain is owned by a group of G lanes of one warp; lane gl holds the DPL
// dimensions [gl*DPL, gl*DPL + DPL) of the chain's position x, direction v
// and candidate y in registers.  A warp holds 32/G chains of one run.  The
// likelihood of a candidate is a group reduction (xor butterflies, so every
// lane of the group ends with the bitwise-identical value and the whole group
// takes the same branch).  Chains of a warp step in lockstep per HRSS step
// and diverge only inside the stepping-out and shrinkage loops; a persistent
// grid takes warps' worth of chains from an atomic ticket queue (costliest
// runs first), so a warp that finishes early takes the next chains instead
// of idling.  No lane ever waits on another block.
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {

// ---- lane-slice loads and stores of a point row ---------------------------
// Lane gl owns entries [gl*DPL, gl*DPL + DPL) of a row of ld floats (ld a
// multiple of 4).  For DPL >= 8 the lane's range can run past ld (d = 20 with
// 8 entries per lane): each float4 is guarded, and entries past ld read as 0
// and are never written.
template <int DPL>
__device__ __forceinline__ void load_lane(const float* __restrict__ row, int gl, int ld, float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      const float4 t = (DPL == 4 || 4 * b < ld) ? reinterpret_cast<const float4*>(row)[b]
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
    }
  } else if constexpr (DPL == 2) {
    const float2 t = reinterpret_cast<const float2*>(row)[gl];
    x[0] = t.x; x[1] = t.y;
  } else {
    x[0] = row[gl];
  }
}

template <int DPL>
__device__ __forceinline__ void ldg_lane(const float* __restrict__ row, int gl, int ld, float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      const float4 t = (DPL == 4 || 4 * b < ld) ? __ldg(reinterpret_cast<const float4*>(row) + b)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
    }
  } else if constexpr (DPL == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(row) + gl);
    x[0] = t.x; x[1] = t.y;
  } else {
    x[0] = __ldg(row + gl);
  }
}

template <int DPL>
__device__ __forceinline__ void store_lane(float* row, int gl, int ld, const float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      if (DPL == 4 || 4 * b < ld)
        reinterpret_cast<float4*>(row)[b] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
  } else if constexpr (DPL == 2) {
    reinterpret_cast<float2*>(row)[gl] = make_float2(x[0], x[1]);
  } else {
    row[gl] = x[0];
  }
}

// Standard normals of the lane's dimensions from words [0, 2 ceil(d/2)) of the
// counter stream (c0, c1, c2): dimension i uses Box-Muller pair i/2.
template <int DPL>
__device__ __forceinline__ void lane_normals(const RunDesc& R, uint32_t c0, uint32_t c1, uint32_t c2,
                                             int gl, float (&z)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl * (DPL / 4) + q));
      box_muller(w.x, w.y, z[4 * q], z[4 * q + 1]);
      box_muller(w.z, w.w, z[4 * q + 2], z[4 * q + 3]);
    }
  } else if constexpr (DPL == 2) {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl >> 1));
    if (gl & 1) box_muller(w.z, w.w, z[0], z[1]);
    else box_muller(w.x, w.y, z[0], z[1]);
  } else {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl >> 2));
    float a, b;
    if (gl & 2) box_muller(w.z, w.w, a, b);
    else box_muller(w.x, w.y, a, b);
    z[0] = (gl & 1) ? b : a;
  }
}

// Uniforms of the lane's dimensions, word i for dimension i.
template <int DPL>
__device__ __forceinline__ void lane_uniform_words(const RunDesc& R, uint32_t c0, uint32_t c1, uint32_t c2,
                                                   int gl, uint32_t (&u)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl * (DPL / 4) + q));
      u[4 * q] = w.x; u[4 * q + 1] = w.y; u[4 * q + 2] = w.z; u[4 * q + 3] = w.w;
    }
  } else {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)((gl * DPL) >> 2));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    const int o = (gl * DPL) & 3;
#pragma unroll
    for (int i = 0; i < DPL; ++i) u[i] = ws[o + i];
  }
}

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

// The words of one HRSS step: group lane b computes Philox block b of the
// step's counter stream (iteration, chain, step, b) once; a word w < 4G is
// then read from lane w/4 by a shuffle, a later word (a shrinkage proposal
// past the first 4G - nz - 3) is drawn on demand.
template <int G>
struct StepWords {
  uint4 mine;       // block base + gl of the step's counter stream
  uint32_t base;
  uint32_t cblk;    // one-block cache for words past the shared range
  uint4 cw;
  __device__ __forceinline__ void draw(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step, int gl,
                                       uint32_t base_) {
    base = base_;
    mine = draw_block(R, iter, chain, step, base + (uint32_t)gl);
    cblk = 0xFFFFFFFFu;
  }
  // word wi, uniform over the group
  __device__ __forceinline__ uint32_t word(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step,
                                           uint32_t wi, unsigned mask) {
    const uint32_t b = wi >> 2;
    if (b >= base && b - base < (uint32_t)G) return __shfl_sync(mask, pick(mine, wi & 3u), (int)(b - base), G);
    if (b != cblk) {
      cw = draw_block(R, iter, chain, step, b);
      cblk = b;
    }
    return pick(cw, wi & 3u);
  }
  // word wi, one per lane (consecutive lanes ask for consecutive words)
  __device__ __forceinline__ uint32_t lane_word(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step,
                                                uint32_t wi, unsigned mask) const {
    const uint32_t src = (wi >> 2) - base;
    const bool shared = src < (uint32_t)G;
    const int sl = shared ? (int)src : 0;
    const uint4 blk = make_uint4(__shfl_sync(mask, mine.x, sl, G), __shfl_sync(mask, mine.y, sl, G),
                                 __shfl_sync(mask, mine.z, sl, G), __shfl_sync(mask, mine.w, sl, G));
    if (shared) return pick(blk, wi & 3u);
    return pick(draw_block(R, iter, chain, step, wi >> 2), wi & 3u);
  }
  // all four words of block b (base <= b < base + G), for lane-specific picks
  __device__ __forceinline__ uint4 block(int b, unsigned mask) const {
    return make_uint4(__shfl_sync(mask, mine.x, b, G), __shfl_sync(mask, mine.y, b, G),
                      __shfl_sync(mask, mine.z, b, G), __shfl_sync(mask, mine.w, b, G));
  }
};

// Normals of the lane's dimensions for the step, from the shared blocks.
template <int G, int DPL>
__device__ __forceinline__ void step_normals(const StepWords<G>& W, const RunDesc& R, uint32_t iter, uint32_t chain,
                                             uint32_t step, int gl, unsigned mask, float (&z)[DPL]) {
  if constexpr (DPL > 4) {
    // the lane's own blocks gl*DPL/4 .. (the shared blocks hold the scalar words)
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const uint4 w = draw_block(R, iter, chain, step, (uint32_t)(gl * (DPL / 4) + q));
      box_muller(w.x, w.y, z[4 * q], z[4 * q + 1]);
      box_muller(w.z, w.w, z[4 * q + 2], z[4 * q + 3]);
    }
  } else if constexpr (DPL == 4) {
    box_muller(W.mine.x, W.mine.y, z[0], z[1]);
    box_muller(W.mine.z, W.mine.w, z[2], z[3]);
  } else if constexpr (DPL == 2) {
    const uint4 w = W.block(gl >> 1, mask);
    if (gl & 1) box_muller(w.z, w.w, z[0], z[1]);
    else box_muller(w.x, w.y, z[0], z[1]);
  } else {
    const uint4 w = W.block(gl >> 2, mask);
    float a, b;
    if (gl & 2) box_muller(w.z, w.w, a, b);
    else box_muller(w.x, w.y, a, b);
    z[0] = (gl & 1) ? b : a;
  }
}

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
// One chain: p HRSS steps from its parent, then replacement of dead slot j.
//
// Along the line y(t) = x + t v every quantity of the slice test is a
// polynomial in t of degree <= 2, so once per step the group reduces the
// coefficients and every evaluation of that step is scalar arithmetic:
//   |y - mu_c|^2 = D_c + t (2 E_c + t C),  D_c = |x - mu_c|^2,
//                  E_c = (x - mu_c).v,  C = |v|^2;
//   box support:   a <= y <= b  <=>  t_lo <= t <= t_hi;
//   Gaussian prior: sum ((y - a)/b)^2 = P0 + t (2 P1 + t P2).
// The moved point x + t v is formed coordinate by coordinate on acceptance.
// ---------------------------------------------------------------------------
constexpr int kMaxComp = 8;

template <int G, int DPL>
__device__ void sweep_chain(const Dev& D, const RunDesc& R, RunState* Sw, int j, int gl, unsigned mask) {
  const float* __restrict__ f = D.f;
  const int d = R.d, ld = R.dpad;
  const bool has = gl * DPL < ld;
  const int parent = D.i[R.o_parent + j];
  const uint32_t iter = (uint32_t)Sw->iter;
  const float lstar = Sw->logLstar;
  const bool box = R.prior_kind == kPriorBox, nonflat = !box;
  const int lk = R.lik_kind;
  const int K = (lk == kLikGmm) ? R.n_comp : ((lk == kLikGauss || lk == kLikFault) ? 1 : 0);
  bool own[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i) own[i] = gl * DPL + i < d;
  float x[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i) x[i] = 0.0f;
  if (has) load_lane<DPL>(f + R.o_x + (long long)parent * ld, gl, ld, x);
  float lx = f[R.o_logL + parent];
  const float w = R.w;
  const uint32_t nz = 2u * (uint32_t)((d + 1) >> 1);
  int evals = 0, acc = 0, nul = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  for (int s = 0; s < R.p; ++s) {
    // the step's direction, drawn ahead (nss_dirgen.cu); the scalar words
    // (U, slice height, shrinkage proposals) from blocks nz/4 + gl
    StepWords<G> W;
    W.draw(R, iter, (uint32_t)j, (uint32_t)s, gl, nz >> 2);
    float v[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) v[i] = 0.0f;
    if (has) ldg_lane<DPL>(f + R.o_V + ((long long)j * R.p + s) * ld, gl, ld, v);

    // coefficients of the step's line, reduced over the group
    float Cv = 0.0f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) Cv = fmaf(v[i], v[i], Cv);
    Cv = gsum<G>(Cv, mask);
    float Dc[kMaxComp], Ec[kMaxComp];
#pragma unroll
    for (int c = 0; c < kMaxComp; ++c) {
      Dc[c] = 0.0f;
      Ec[c] = 0.0f;
      if (c < K) {
        float m[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) m[i] = 0.0f;
        if (has) ldg_lane<DPL>(f + R.o_mu + (long long)c * ld, gl, ld, m);
        float dq = 0.0f, de = 0.0f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
          const float e = x[i] - m[i];
          dq = fmaf(e, e, dq);
          de = fmaf(e, v[i], de);
        }
        Dc[c] = gsum<G>(dq, mask);
        Ec[c] = gsum<G>(de, mask);
      }
    }
    float t_lo = -INFINITY, t_hi = INFINITY;
    float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f, height = 0.0f;
    if (box) {
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        if (own[i]) {
          const int dim = gl * DPL + i;
          const float ai = f[R.o_a + dim] - x[i], bi = f[R.o_b + dim] - x[i];
          const float rv = __frcp_rn(v[i]);
          if (v[i] > 0.0f) {
            t_lo = fmaxf(t_lo, ai * rv);
            t_hi = fminf(t_hi, bi * rv);
          } else if (v[i] < 0.0f) {
            t_lo = fmaxf(t_lo, bi * rv);
            t_hi = fminf(t_hi, ai * rv);
          } else if (!(ai <= 0.0f && bi >= 0.0f)) {
            t_lo = INFINITY;
          }
        }
      }
      t_lo = gmax<G>(t_lo, mask);
      t_hi = -gmax<G>(-t_hi, mask);
    } else {
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        if (own[i]) {
          const int dim = gl * DPL + i;
          const float ib = 1.0f / f[R.o_b + dim];
          const float u = (x[i] - f[R.o_a + dim]) * ib, q = v[i] * ib;
          P0 = fmaf(u, u, P0);
          P1 = fmaf(u, q, P1);
          P2 = fmaf(q, q, P2);
        }
      }
      P0 = gsum<G>(P0, mask);
      P1 = gsum<G>(P1, mask);
      P2 = gsum<G>(P2, mask);
      const float uh = u24(W.word(R, iter, (uint32_t)j, (uint32_t)s, nz + 1u, mask));
      height = fmaf(-0.5f, P0, R.prior_const) + logf(uh);
    }
    float x0 = 0.0f, v0 = 0.0f;  // coordinate 0 for the fault likelihood
    if (lk == kLikFault) {
      x0 = __shfl_sync(mask, x[0], 0, G);
      v0 = __shfl_sync(mask, v[0], 0, G);
    }
    // one slice test at x + t v: support, prior slice height, then
    // logL > logL* (Sec. 3.1: E < E_batch).  A NaN likelihood reads as -inf
    // and is flagged; nothing is counted here.
    auto probe = [&](float t, float& ll, bool& isn) -> bool {
      if (box && !(t >= t_lo && t <= t_hi)) return false;
      if (nonflat) {
        const float lp = fmaf(-0.5f, fmaf(t, fmaf(t, P2, 2.0f * P1), P0), R.prior_const);
        if (!(lp > height)) return false;
      }
      if (lk == kLikFlat) {
        ll = 0.0f;
      } else {
        float vc[kMaxComp];
        float M = -INFINITY;
#pragma unroll
        for (int c = 0; c < kMaxComp; ++c) {
          vc[c] = (c < K) ? -fmaf(t, fmaf(t, Cv, 2.0f * Ec[c]), Dc[c]) * R.inv2s2 : -INFINITY;
          M = fmaxf(M, vc[c]);
        }
        float S = 0.0f;
#pragma unroll
        for (int c = 0; c < kMaxComp; ++c)
          if (c < K) S += __expf(vc[c] - M);
        ll = (K == 1 ? M : M + __logf(S)) + R.lognorm;
        if (lk == kLikFault && fmaf(t, v0, x0) < R.fault_param)
          ll = (R.fault_mode == 1) ? __int_as_float(0x7fc00000) : INFINITY;
      }
      if (isnan(ll)) {
        ll = -INFINITY;
        isn = true;
      }
      return ll > lstar;
    };
    // Stepping out: an end moves by repeated FP32 steps of +-w while the
    // slice test at it passes, at most kStepOutCap tests.  The ends it visits
    // do not depend on the outcomes, so the group tests G consecutive ones at
    // once; the first that fails is where the one-at-a-time procedure stops,
    // and the counters are those of that procedure.
    auto step_out = [&](float start, float delta) -> float {
      int nfail = kStepOutCap;
      for (int b0 = 0; b0 < kStepOutCap; b0 += G) {
        const int idx = b0 + gl;
        float t = start;
#pragma unroll
        for (int i = 0; i < kStepOutCap - 1; ++i)
          if (i < idx) t += delta;
        const bool valid = idx < kStepOutCap;
        bool isn = false;
        float ll = 0.0f;
        const bool in = valid && probe(t, ll, isn);
        const unsigned outb = gballot<G>(valid && !in, mask);
        const unsigned nanb = gballot<G>(isn, mask);
        if (outb) {
          const int f = __ffs(outb) - 1;
          nfail = b0 + f;
          nanc += __popc(nanb & ((2u << f) - 1u));
          break;
        }
        nanc += __popc(nanb);
      }
      evals += min(nfail + 1, kStepOutCap);
      exps += nfail;
      if (nfail == kStepOutCap) ++capo;
      float t = start;
      for (int i = 0; i < nfail; ++i) t += delta;
      return t;
    };
    // randomised initial bracket of width w around t = 0
    const float U = u24(W.word(R, iter, (uint32_t)j, (uint32_t)s, nz, mask));
    float tl = -w * U;
    float tr = tl + w;
    tl = step_out(tl, -w);
    tr = step_out(tr, w);
    // Shrinkage, at most kShrinkCap proposals, then a null move.  Proposal r
    // is t_r = tl_r + u_r (tr_r - tl_r) and a rejection moves the end on
    // t_r's side to t_r, so the brackets of the proposals that follow
    // rejections are known before any test: each round the group forms G
    // consecutive proposals (a short scan over the shared u's) and tests
    // them at once; the first inside the slice is the sequential result.
    bool ok = false;
    float tacc = 0.0f, llacc = 0.0f;
    for (int b0 = 0; b0 < kShrinkCap; b0 += G) {
      const int idx = b0 + gl;
      const bool valid = idx < kShrinkCap;
      const float u = u24(W.lane_word(R, iter, (uint32_t)j, (uint32_t)s, nz + 3u + (uint32_t)idx, mask));
      float lo = tl, hi = tr, t = 0.0f;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const float ui = __shfl_sync(mask, u, i, G);
        const float ti = fmaf(ui, hi - lo, lo);
        if (i == gl) t = ti;
        if (ti < 0.0f) lo = ti;
        else hi = ti;
      }
      bool isn = false;
      float ll = 0.0f;
      const bool in = valid && probe(t, ll, isn);
      const unsigned inb = gballot<G>(in, mask);
      const unsigned nanb = gballot<G>(isn, mask);
      if (inb) {
        const int f = __ffs(inb) - 1;
        shr += f + 1;
        evals += f + 1;
        nanc += __popc(nanb & ((1u << f) - 1u));
        tacc = __shfl_sync(mask, t, f, G);
        llacc = __shfl_sync(mask, ll, f, G);
        ok = true;
        break;
      }
      const int nvalid = min(G, kShrinkCap - b0);
      shr += nvalid;
      evals += nvalid;
      nanc += __popc(nanb);
      tl = lo;
      tr = hi;
    }
    if (ok) {
#pragma unroll
      for (int i = 0; i < DPL; ++i) x[i] = fmaf(tacc, v[i], x[i]);
      lx = llacc;
    }
    if (ok) ++acc;
    else ++nul;
  }
  // (iv) replace dead slot j, born at logL*
  const int slot = D.i[R.o_dead + j];
  if (has) store_lane<DPL>(D.f + R.o_x + (long long)slot * ld, gl, ld, x);
  if (gl == 0) {
    D.f[R.o_logL + slot] = lx;
    D.f[R.o_birth + slot] = lstar;
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
// resident blocks per SM the register budget is tuned for
constexpr int sweep_min_blocks(int dpl) { return dpl <= 2 ? 5 : dpl == 4 ? 4 : dpl == 8 ? 4 : 3; }

template <int G, int DPL>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_blocks(DPL)) k_sweep(Dev D, const WorkItem* __restrict__ items, int n_items,
                                                         int* queue) {
  const int lane = threadIdx.x & 31;
  const int gl = lane % G, grp = lane / G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const WorkItem wi = items[it];
    RunState* S = D.st + wi.run;
    if (S->done) continue;
    const int j = wi.c0 + grp;
    if (j < wi.c1) sweep_chain<G, DPL>(D, D.desc[wi.run], S, j, gl, mask);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// configuration table and launchers
// ---------------------------------------------------------------------------
#define NSS_CFGS(X) \
  X(0, 1, 4) X(1, 2, 4) X(2, 4, 4) X(3, 8, 4) X(4, 16, 4) X(5, 32, 4) \
  X(6, 2, 2) X(7, 4, 2) X(8, 8, 2) X(9, 16, 2) X(10, 32, 2) \
  X(11, 4, 1) X(12, 8, 1) X(13, 16, 1) X(14, 32, 1) \
  X(15, 2, 8) X(16, 4, 8) X(17, 8, 8) X(18, 16, 8) \
  X(19, 2, 16) X(20, 4, 16) X(21, 8, 16)

// configurations 22..24: one chain per lane (nss_sweep_lane.cu), d <= 8, 16, 32
constexpr int kLaneCfg0 = 22;
static int lane_dmax(int cfg) { return cfg == 22 ? 8 : cfg == 23 ? 16 : 32; }

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

int sweep_blocks_per_sm(int cfg) {
  if (cfg >= kLaneCfg0) return sweep_lane_blocks_per_sm(lane_dmax(cfg));
  int nb = 0;
  switch (cfg) {
#define X(id, g, p) case id: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<g, p>, kSweepThreads, 0); break;
    NSS_CFGS(X)
#undef X
    default: break;
  }
  return nb > 0 ? nb : 1;
}

cudaError_t launch_sweep(int cfg, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                         cudaStream_t s) {
  if (cfg >= kLaneCfg0) return launch_sweep_lane(lane_dmax(cfg), D, items, n, queue, grid, s);
  switch (cfg) {
#define X(id, g, p) case id: k_sweep<g, p><<<grid, kSweepThreads, 0, s>>>(D, items, n, queue); break;
    NSS_CFGS(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace nss
