// nss_sweep_lane.cu -- the HRSS sweep with one chain per lane (d <= 32), for
// sm_103a.
//
// A lane holds its chain's whole position x and direction v in registers.
// Per HRSS step it loads its direction (drawn ahead for every step of the
// iteration), then forms the coefficients of the step's line:
//   |x + t v - mu_c|^2 = D_c + t (2 E_c + t C),   box: t in [t_lo, t_hi],
//   Gaussian prior: sum ((x + t v - a)/b)^2 = P0 + t (2 P1 + t P2),
// so every slice evaluation of the step is a few scalar FMAs and one
// log-sum-exp, with no communication between lanes.  The 32 chains of a warp
// belong to one run and step in lockstep per HRSS step.
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {
namespace {

constexpr int kLaneThreads = 32;   // one warp per block: few warps in total, spread over every SM
template <int DMAX, int KC>
__device__ void lane_chain(const Dev& D, const RunDesc& R, RunState* Sw, int j) {
  const float* __restrict__ f = D.f;
  const int d = R.d, ld = R.dpad;
  const int parent = D.i[R.o_parent + j];
  const uint32_t iter = (uint32_t)Sw->iter;
  const float lstar = Sw->logLstar;
  const bool box = R.prior_kind == kPriorBox, nonflat = !box;
  const int lk = R.lik_kind;
  const int K = (lk == kLikGmm) ? R.n_comp : ((lk == kLikGauss || lk == kLikFault || lk == kLikRastrigin) ? 1 : 0);
  float x[DMAX];
  {
    const float4* xp = reinterpret_cast<const float4*>(f + R.o_x + (long long)parent * ld);
#pragma unroll
    for (int b = 0; b < DMAX / 4; ++b) {
      const float4 t = (4 * b < ld) ? xp[b] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * b] = t.x; x[4 * b + 1] = t.y; x[4 * b + 2] = t.z; x[4 * b + 3] = t.w;
    }
  }
  float lx = f[R.o_logL + parent];
  const float w = R.w;
  // the run's scalars and offsets the steps use, read once
  const int P = R.p;
  const bool rw = R.kernel == kKernelRw;
  const float inv2s2 = R.inv2s2, lognorm = R.lognorm, pconst = R.prior_const, rws = R.rw_scale;
  const uint32_t key0 = R.key0, key1 = R.key1;
  const long long o_V = R.o_V, o_mu = R.o_mu, o_a = R.o_a, o_b = R.o_b, o_wd = R.o_wd;
  const uint32_t nz = 2u * (uint32_t)((d + 1) >> 1);
  int evals = 0, acc = 0, nul = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  for (int s = 0; s < P; ++s) {
    // the step's direction, drawn ahead (nss_dirgen.cu)
    float v[DMAX];
    float Cv = 0.0f;
    {
      const float4* vp = reinterpret_cast<const float4*>(f + o_V + ((long long)j * P + s) * ld);
#pragma unroll
      for (int b = 0; b < DMAX / 4; ++b) {
        const float4 t = (4 * b < ld) ? __ldg(vp + b) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * b] = t.x; v[4 * b + 1] = t.y; v[4 * b + 2] = t.z; v[4 * b + 3] = t.w;
      }
#pragma unroll
      for (int a = 0; a < DMAX; ++a) Cv = fmaf(v[a], v[a], Cv);
    }
    // mixture coefficients; components K..KC-1 read as infinitely far
    float Dc[KC], Ec[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      float dq = INFINITY, de = 0.0f;
      if (c < K) {
        dq = 0.0f;
        const float4* m4 = reinterpret_cast<const float4*>(f + o_mu + (long long)c * ld);
#pragma unroll
        for (int b = 0; b < DMAX / 4; ++b) {
          if (4 * b < ld) {
            const float4 m = __ldg(m4 + b);
            const float e0 = x[4 * b] - m.x, e1 = x[4 * b + 1] - m.y, e2 = x[4 * b + 2] - m.z, e3 = x[4 * b + 3] - m.w;
            dq = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, dq))));
            de = fmaf(e0, v[4 * b], fmaf(e1, v[4 * b + 1], fmaf(e2, v[4 * b + 2], fmaf(e3, v[4 * b + 3], de))));
          }
        }
      }
      Dc[c] = dq;
      Ec[c] = de;
    }
    // support interval of the box prior, or the Gaussian-prior quadratic
    float t_lo = -INFINITY, t_hi = INFINITY;
    float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f, height = 0.0f;
    if (box) {
#pragma unroll
      for (int i = 0; i < DMAX; ++i) {
        if (i < d) {
          const float ai = __ldg(f + o_a + i) - x[i], bi = __ldg(f + o_b + i) - x[i];
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
    } else {
#pragma unroll
      for (int i = 0; i < DMAX; ++i) {
        if (i < d) {
          const float ib = 1.0f / __ldg(f + o_b + i);
          const float u = (x[i] - __ldg(f + o_a + i)) * ib, q = v[i] * ib;
          P0 = fmaf(u, u, P0);
          P1 = fmaf(u, q, P1);
          P2 = fmaf(q, q, P2);
        }
      }
    }
    // step words beyond the normals: U, height, shrinkage proposals
    // words nz .. nz + 11 drawn ahead beside the directions; later ones now
    const int* ws = D.i + o_wd + ((long long)j * P + s) * kStepWords;
    uint32_t cblk = 0xFFFFFFFFu;
    uint4 cw = make_uint4(0u, 0u, 0u, 0u);
    auto word = [&](uint32_t wi) {
      if (wi - nz < (uint32_t)kStepWords) return (uint32_t)__ldg(ws + (wi - nz));
      if ((wi >> 2) != cblk) {
        cblk = wi >> 2;
        cw = philox4x32_10(make_uint4(iter, (uint32_t)j, (uint32_t)s, cblk), key0, key1);
      }
      return pick(cw, wi & 3u);
    };
    // HRSS: slice height (word nz + 1); RW: Metropolis threshold (word nz)
    if (nonflat) height = fmaf(-0.5f, P0, pconst) + logf(u24(word(rw ? nz : nz + 1u)));
    auto in_slice = [&](float t, float& ll) -> bool {
      ++evals;
      if (box && !(t >= t_lo && t <= t_hi)) return false;
      if (nonflat) {
        const float lp = fmaf(-0.5f, fmaf(t, fmaf(t, P2, 2.0f * P1), P0), pconst);
        if (!(lp > height)) return false;
      }
      if (lk == kLikFlat) {
        ll = 0.0f;
      } else {
        float vc[KC];
        float M = -INFINITY;
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          vc[c] = -fmaf(t, fmaf(t, Cv, 2.0f * Ec[c]), Dc[c]) * inv2s2;
          M = fmaxf(M, vc[c]);
        }
        if constexpr (KC == 1) {
          ll = M + lognorm;
        } else {
          float S = 0.0f;
#pragma unroll
          for (int c = 0; c < KC; ++c) S += __expf(vc[c] - M);
          ll = M + __logf(S) + lognorm;
        }
        if (lk == kLikFault && fmaf(t, v[0], x[0]) < R.fault_param)
          ll = (R.fault_mode == 1) ? __int_as_float(0x7fc00000) : INFINITY;
        if (lk == kLikRastrigin) {
          // App. F.3 mixture: the Gaussian part above (mean 0, sigma 1), the
          // cosine sum over the lane's dimensions
          float cs = 0.0f;
#pragma unroll
          for (int i = 0; i < DMAX; ++i)
            if (i < d) cs += cospif(2.0f * fmaf(t, v[i], x[i]));
          const float a1 = R.ras_la + ll, a2 = R.ras_l1a + fmaf(10.0f, cs, -10.0f * (float)d);
          const float hi = fmaxf(a1, a2), lo = fminf(a1, a2);
          ll = (hi == -INFINITY) ? -INFINITY : hi + log1pf(expf(lo - hi));
        }
      }
      if (isnan(ll)) {
        ll = -INFINITY;
        ++nanc;
      }
      return ll > lstar;
    };
    if (rw) {
      // constrained random walk: one proposal at the line point t = s
      const float ts = rws;
      float ll = 0.0f;
      if (in_slice(ts, ll)) {
#pragma unroll
        for (int i = 0; i < DMAX; ++i) x[i] = fmaf(ts, v[i], x[i]);
        lx = ll;
        ++acc;
      } else {
        ++nul;
      }
      continue;
    }
    const float U = u24(word(nz));
    float tl = -w * U, tr = tl + w, lly = 0.0f;
    for (int n = 0;; ++n) {
      if (n >= kStepOutCap) { ++capo; break; }
      if (!in_slice(tl, lly)) break;
      tl -= w;
      ++exps;
    }
    for (int n = 0;; ++n) {
      if (n >= kStepOutCap) { ++capo; break; }
      if (!in_slice(tr, lly)) break;
      tr += w;
      ++exps;
    }
    bool ok = false;
    for (int r = 0; r < kShrinkCap; ++r) {
      const float u = u24(word(nz + 3u + (uint32_t)r));
      const float t = fmaf(u, tr - tl, tl);
      ++shr;
      if (in_slice(t, lly)) {
#pragma unroll
        for (int i = 0; i < DMAX; ++i) x[i] = fmaf(t, v[i], x[i]);
        lx = lly;
        ok = true;
        break;
      }
      if (t < 0.0f) tl = t;
      else tr = t;
    }
    if (ok) ++acc;
    else ++nul;
  }
  // (iv) replace dead slot j, born at logL*
  const int slot = D.i[R.o_dead + j];
  float4* xo = reinterpret_cast<float4*>(D.f + R.o_x + (long long)slot * ld);
#pragma unroll
  for (int b = 0; b < DMAX / 4; ++b)
    if (4 * b < ld) xo[b] = make_float4(x[4 * b], x[4 * b + 1], x[4 * b + 2], x[4 * b + 3]);
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

template <int DMAX, int KC>
__global__ void __launch_bounds__(kLaneThreads, (DMAX >= 32 ? 8 : 16)) k_sweep_lane(Dev D, const WorkItem* __restrict__ items,
                                                                                int n_items, int* queue) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const WorkItem wi = items[it];
    RunState* S = D.st + wi.run;
    if (S->done) continue;
    const int j = wi.c0 + lane;
    if (j < wi.c1) lane_chain<DMAX, KC>(D, D.desc[wi.run], S, j);
    __syncwarp();
  }
}

template <int DMAX>
cudaError_t launch_lane_dmax(int kc, const Dev& D, const WorkItem* items, int n, int* queue, int grid, cudaStream_t s) {
  switch (kc) {
    case 1: k_sweep_lane<DMAX, 1><<<grid, kLaneThreads, 0, s>>>(D, items, n, queue); break;
    case 4: k_sweep_lane<DMAX, 4><<<grid, kLaneThreads, 0, s>>>(D, items, n, queue); break;
    case 8: k_sweep_lane<DMAX, 8><<<grid, kLaneThreads, 0, s>>>(D, items, n, queue); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int DMAX>
int lane_blocks_dmax(int kc) {
  int nb = 0;
  switch (kc) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_lane<DMAX, 1>, kLaneThreads, 0); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_lane<DMAX, 4>, kLaneThreads, 0); break;
    case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_lane<DMAX, 8>, kLaneThreads, 0); break;
    default: break;
  }
  return nb > 0 ? nb : 1;
}

}  // namespace

cudaError_t launch_sweep_lane(int dmax, int kc, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                              cudaStream_t s) {
  switch (dmax) {
    case 8: return launch_lane_dmax<8>(kc, D, items, n, queue, grid, s);
    case 16: return launch_lane_dmax<16>(kc, D, items, n, queue, grid, s);
    case 32: return launch_lane_dmax<32>(kc, D, items, n, queue, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int sweep_lane_warps_per_block() { return kLaneThreads / 32; }

int sweep_lane_blocks_per_sm(int dmax, int kc) {
  switch (dmax) {
    case 8: return lane_blocks_dmax<8>(kc);
    case 16: return lane_blocks_dmax<16>(kc);
    case 32: return lane_blocks_dmax<32>(kc);
    default: return 1;
  }
}

}  // namespace nss
