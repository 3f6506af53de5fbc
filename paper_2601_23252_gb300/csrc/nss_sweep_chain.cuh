// nss_sweep_chain.cuh -- the Hit-and-Run Slice Sampling sweep (steps
// (iii)+(iv) of Sec. 3.1; HRSS of Sec. 3.2 and App. B.4), for sm_103a.
//
// A chain is owned by a group of G lanes of one warp; lane gl holds the DPL
// dimensions [gl*DPL, gl*DPL + DPL) of the chain's position x and of the
// step's direction v in registers.  A warp holds 32/G chains of one run.
// Group reductions are xor butterflies, so every lane of the group ends with
// the bitwise-identical value and the whole group takes the same branch.
// The warp's chains step in lockstep and never split the warp: the
// stepping-out and shrinkage rounds loop until every group is done (a done
// group evaluates but changes nothing), so every shuffle and vote runs on
// the full warp.  A persistent grid takes warps' worth of chains from an
// atomic ticket queue (costliest runs first), so a warp that finishes early
// takes the next chains instead of idling.  No lane ever waits on another
// block.
//
// KC bounds the number of mixture components (1: one isotropic Gaussian or
// no likelihood; 4; 8).  Components K..KC-1 of a run with fewer read as
// infinitely far, so the component loops are fully unrolled and branch-free.
// Each KC is instantiated in its own translation unit (nss_sweep_k*.cu).
#pragma once
#include "nss_sweep_common.cuh"

namespace nss {

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
template <int G, int DPL, int KC>
__device__ void sweep_chain(const Dev& D, const RunDesc& R, RunState* Sw, int j, int gl, unsigned mask, bool live) {
  // Every lane of the warp runs here (a group without a chain of its own
  // repeats the warp's first chain and writes nothing), and all groups take
  // the same number of steps, so the per-step reductions and the grouped
  // slice-test rounds run on the whole warp (full-mask shuffles and votes,
  // warp-uniform round loops); `mask` (the group's lanes) serves the paths
  // whose groups run their tests one at a time.
  constexpr unsigned kAll = 0xffffffffu;
  const int gshift = (int)(threadIdx.x & 31) & ~(G - 1);  // first lane of the group
  const float* __restrict__ f = D.f;
  const int d = R.d, ld = R.dpad;
  const bool has = gl * DPL < ld;
  const int parent = D.i[R.o_parent + j];
  const uint32_t iter = (uint32_t)Sw->iter;
  const float lstar = Sw->logLstar;
  const bool box = R.prior_kind == kPriorBox, nonflat = !box;
  // runs with a mixture bound above 1 are mixture runs (sweep_kc), so their
  // instantiations compile the mixture likelihood alone
  const int lk = KC > 1 ? kLikGmm : R.lik_kind;
  const int K = (lk == kLikGmm) ? R.n_comp : ((lk == kLikGauss || lk == kLikFault || lk == kLikRastrigin) ? 1 : 0);
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
  // the run's scalars the steps use, read once
  const int P = R.p;
  const bool rw = R.kernel == kKernelRw;
  const float inv2s2 = R.inv2s2, lognorm = R.lognorm, pconst = R.prior_const, rws = R.rw_scale;
  // Per-chain counters.  Logical evaluations and null moves are not kept:
  // every step ends in an acceptance or a null move, so nul = p - acc, and
  // a side that stops after n expansions took min(n + 1, cap) tests, so an
  // HRSS chain's evals = exps + 2 p - capo + shr (a random-walk chain takes
  // one test per step: evals = p).
  int acc = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  int ran = 0;  // slice tests this lane ran (logical or speculative)
  // slice-test rounds of the warp, and those this group still needed (the
  // others are lockstep idle rounds of a group that is done)
  int rounds = 0, active = 0;
  // the steps' directions, drawn ahead (nss_dirgen.cu); the load of step
  // s + 1's is issued while step s runs
  const float* vrow = f + R.o_V + (long long)j * R.p * ld;
  // the steps' first scalar words (U, slice height, shrinkage proposals
  // 0..8), drawn ahead beside the directions; lane gl's first-round proposal
  // is word 3 + gl
  const int* wrow = D.i + R.o_wd + (long long)j * R.p * kStepWords;
  const bool wlane = 3 + gl < kStepWords;
  float vn[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i) vn[i] = 0.0f;
  if (has) ldg_lane<DPL>(vrow, gl, ld, vn);
  // a single-component run's mean and the prior's bounds stay in registers
  // across the steps (up to 8 dimensions per lane); otherwise each step
  // reads them again
  constexpr bool kHold = KC == 1 && DPL <= 8;
  float hm[kHold ? DPL : 1], hpa[kHold ? DPL : 1], hpb[kHold ? DPL : 1];
  if constexpr (kHold) {
#pragma unroll
    for (int i = 0; i < DPL; ++i) hm[i] = hpa[i] = hpb[i] = 0.0f;
    if (has) {
      if (K > 0) ldg_lane<DPL>(f + R.o_mu, gl, ld, hm);
      ldg_lane<DPL>(f + R.o_a, gl, ld, hpa);
      ldg_lane<DPL>(f + R.o_b, gl, ld, hpb);
    }
  }
  uint32_t nU = (uint32_t)__ldg(wrow), nH = nonflat ? (uint32_t)__ldg(wrow + 1) : 0u;
  uint32_t nS = wlane ? (uint32_t)__ldg(wrow + 3 + gl) : 0u;
  for (int s = 0; s < P; ++s) {
    float v[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) v[i] = vn[i];
    const uint32_t wU = nU, wH = nH, wS = nS;
    if (s + 1 < P) {
      const int* wn = wrow + (long long)(s + 1) * kStepWords;
      if (has) ldg_lane<DPL>(vrow + (long long)(s + 1) * ld, gl, ld, vn);
      nU = (uint32_t)__ldg(wn);
      if (nonflat) nH = (uint32_t)__ldg(wn + 1);
      if (wlane) nS = (uint32_t)__ldg(wn + 3 + gl);
    }
    // word nz + r of the step: drawn ahead for r < kStepWords, else now
    const int* ws = wrow + (long long)s * kStepWords;
    auto step_word = [&](uint32_t r) -> uint32_t {
      if (r < (uint32_t)kStepWords) return (uint32_t)__ldg(ws + r);
      const uint32_t wi = nz + r;
      return pick(draw_block(R, iter, (uint32_t)j, (uint32_t)s, wi >> 2), wi & 3u);
    };

    // coefficients of the step's line, reduced over the group
    float Cv = 0.0f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) Cv = fmaf(v[i], v[i], Cv);
    Cv = gsum<G>(Cv, kAll);
    float Dc[KC], Ec[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      Dc[c] = INFINITY;
      Ec[c] = 0.0f;
    }
    if (K > 0) {
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int cr = c < K ? c : K - 1;  // rows past K repeat the last one, then read as infinitely far
        float m[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) m[i] = 0.0f;
        if constexpr (kHold) {
#pragma unroll
          for (int i = 0; i < DPL; ++i) m[i] = hm[i];
        } else {
          if (has) ldg_lane<DPL>(f + R.o_mu + (long long)cr * ld, gl, ld, m);
        }
        float dq = 0.0f, de = 0.0f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
          const float e = x[i] - m[i];
          dq = fmaf(e, e, dq);
          de = fmaf(e, v[i], de);
        }
        dq = gsum<G>(dq, kAll);
        Ec[c] = gsum<G>(de, kAll);
        Dc[c] = c < K ? dq : INFINITY;
      }
    }
    // support and prior terms of the slice test; a run has either a box
    // prior (q0, q1 = t_lo, t_hi) or a Gaussian one (q0..q2 = P0..P2, q3 =
    // the slice height), so the two share registers
    float q0, q1, q2 = 0.0f, q3 = 0.0f;
    // the prior's per-dimension a (lower bound / mean) and b (upper bound / sd)
    float pa[DPL], pb[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) pa[i] = pb[i] = 0.0f;
    if constexpr (kHold) {
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        pa[i] = hpa[i];
        pb[i] = hpb[i];
      }
    } else {
      if (has) {
        ldg_lane<DPL>(f + R.o_a, gl, ld, pa);
        ldg_lane<DPL>(f + R.o_b, gl, ld, pb);
      }
    }
    if (box) {
      float t_lo = -INFINITY, t_hi = INFINITY;
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        // a <= x + t v <= b per dimension: [ta, tb] for v > 0, [tb, ta] for
        // v < 0, so the smaller end bounds t below and the larger above
        // (no lane branches); v = 0 with x strictly inside gives the
        // infinite ends of the reciprocal and leaves t free
        const float ai = pa[i] - x[i], bi = pb[i] - x[i];
        const float rv = __fdividef(1.0f, v[i]);
        const float ta = ai * rv, tb = bi * rv;
        t_lo = own[i] ? fmaxf(t_lo, fminf(ta, tb)) : t_lo;
        t_hi = own[i] ? fminf(t_hi, fmaxf(ta, tb)) : t_hi;
      }
      q0 = gmax<G>(t_lo, kAll);
      q1 = -gmax<G>(-t_hi, kAll);
    } else {
      float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f;
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        if (own[i]) {
          const float ib = 1.0f / pb[i];
          const float u = (x[i] - pa[i]) * ib, q = v[i] * ib;
          P0 = fmaf(u, u, P0);
          P1 = fmaf(u, q, P1);
          P2 = fmaf(q, q, P2);
        }
      }
      P0 = gsum<G>(P0, kAll);
      P1 = gsum<G>(P1, kAll);
      P2 = gsum<G>(P2, kAll);
      // HRSS: slice height log Pi(x) + ln u (word nz + 1); RW: the Metropolis
      // threshold log Pi(x) + ln u with u = word nz
      const float uh = u24(rw ? wU : wH);
      q3 = fmaf(-0.5f, P0, pconst) + logf(uh);
      q0 = P0;
      q1 = P1;
      q2 = P2;
    }
    float x0 = 0.0f, v0 = 0.0f;  // coordinate 0 for the fault likelihood
    if (lk == kLikFault) {
      x0 = __shfl_sync(kAll, x[0], 0, G);
      v0 = __shfl_sync(kAll, v[0], 0, G);
    }
    // one slice test at x + t v: support, prior slice height, then
    // logL > logL* (Sec. 3.1: E < E_batch).  A NaN likelihood reads as -inf
    // and is flagged (only where support and prior pass); nothing is counted
    // here.  No early exit: every lane evaluates, so a warp never splits.
    auto probe = [&](float t, float& ll, bool& isn) -> bool {
      bool ok = true;
      if (box) ok = t >= q0 && t <= q1;
      if (nonflat) {
        const float lp = fmaf(-0.5f, fmaf(t, fmaf(t, q2, 2.0f * q1), q0), pconst);
        ok = lp > q3;
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
        if (lk == kLikFault && fmaf(t, v0, x0) < R.fault_param)
          ll = (R.fault_mode == 1) ? __int_as_float(0x7fc00000) : INFINITY;
      }
      const bool nan_ll = isnan(ll);
      ll = nan_ll ? -INFINITY : ll;
      isn = ok && nan_ll;
      return ok && ll > lstar;
    };
    if (lk == kLikRastrigin) {
      // The Rastrigin mixture (App. F.3) is not affine along the line: every
      // test sums cos(2 pi y_i) over the group's dimensions (the Gaussian part
      // comes from the line coefficients), so the tests run one at a time.
      auto test = [&](float t, float& ll, bool& isn) -> bool {
        if (gl == 0) ++ran;
        if (box && !(t >= q0 && t <= q1)) return false;
        if (nonflat) {
          const float lp = fmaf(-0.5f, fmaf(t, fmaf(t, q2, 2.0f * q1), q0), R.prior_const);
          if (!(lp > q3)) return false;
        }
        float cs = 0.0f;
#pragma unroll
        for (int i = 0; i < DPL; ++i)
          if (own[i]) cs += cospif(2.0f * fmaf(t, v[i], x[i]));
        cs = gsum<G>(cs, mask);
        const float lf = -0.5f * fmaf(t, fmaf(t, Cv, 2.0f * Ec[0]), Dc[0]);
        const float lg = fmaf(10.0f, cs, -10.0f * (float)d);
        const float a1 = R.ras_la + lf, a2 = R.ras_l1a + lg;
        const float hi = fmaxf(a1, a2), lo = fminf(a1, a2);
        ll = (hi == -INFINITY) ? -INFINITY : hi + log1pf(expf(lo - hi));
        if (isnan(ll)) {
          ll = -INFINITY;
          isn = true;
        }
        return ll > lstar;
      };
      if (R.kernel == kKernelRw) {
        bool isn = false;
        float ll = 0.0f;
        const bool in = test(R.rw_scale, ll, isn);
        if (isn) ++nanc;
        if (in) {
#pragma unroll
          for (int i = 0; i < DPL; ++i) x[i] = fmaf(R.rw_scale, v[i], x[i]);
          lx = ll;
          ++acc;
        }
        continue;
      }
      const float tl0 = -w * u24(wU);
      float ends[2] = {tl0, tl0 + w};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float delta = q ? w : -w;
        float t = ends[q];
        int n = 0;
        for (; n < kStepOutCap; ++n) {
          bool isn = false;
          float ll = 0.0f;
          const bool in = test(t, ll, isn);
          if (isn) ++nanc;
          if (!in) break;
          t += delta;
        }
        ends[q] = t;
        exps += n;
        if (n == kStepOutCap) ++capo;
      }
      float tl = ends[0], tr = ends[1];
      bool ok = false;
      for (int r = 0; r < kShrinkCap; ++r) {
        const float t = fmaf(u24(step_word(3u + (uint32_t)r)), tr - tl, tl);
        ++shr;
        bool isn = false;
        float ll = 0.0f;
        const bool in = test(t, ll, isn);
        if (isn) ++nanc;
        if (in) {
#pragma unroll
          for (int i = 0; i < DPL; ++i) x[i] = fmaf(t, v[i], x[i]);
          lx = ll;
          ok = true;
          break;
        }
        if (t < 0.0f) tl = t;
        else tr = t;
      }
      if (ok) ++acc;
      continue;
    }
    if (rw) {
      // constrained random walk: one proposal y = x + s (L z), the line point
      // t = s; accepted under the same support / prior / logL* test
      const float ts = rws;
      bool isn = false;
      float ll = 0.0f;
      const bool in = probe(ts, ll, isn);
      if (gl == 0) ++ran;  // the group's lanes test the same point: one test
      if (isn) ++nanc;
      if (in) {
#pragma unroll
        for (int i = 0; i < DPL; ++i) x[i] = fmaf(ts, v[i], x[i]);
        lx = ll;
        ++acc;
      }
      continue;
    }
    // Stepping out: an end moves by repeated FP32 steps of +-w while the
    // slice test at it passes, at most kStepOutCap tests per side; index
    // kStepOutCap of a side is a stop that is never tested (the cap).  The
    // ends visited do not depend on the outcomes, so with G >= 2 the group
    // tests both sides at once: lanes [0, H) the left and [H, G) the right,
    // H = G/2 consecutive ends of each per round.  The first failing end of
    // a side is where the one-at-a-time procedure stops, and the counters are
    // those of that procedure.
    const float U = u24(wU);
    const float tl0 = -w * U;
    float ends[2] = {tl0, tl0 + w};
    if constexpr (G >= 2) {
      constexpr int H = G / 2;
      constexpr unsigned kHalf = (H == 32) ? 0xffffffffu : ((1u << H) - 1u);
      const int side = gl >= H ? 1 : 0;
      const int hl = gl - side * H;
      const float delta = side ? w : -w;
      float base[2] = {ends[0], ends[1]};  // the end at index b0 of each side
      int stop[2] = {-1, -1};
      // rounds until every group of the warp has stopped both sides; a group
      // that has stops testing (its lanes evaluate but count nothing)
      for (int b0 = 0; __any_sync(kAll, stop[0] < 0 || stop[1] < 0); b0 += H) {
        ++rounds;
        active += (stop[0] < 0 || stop[1] < 0) ? 1 : 0;
        const int idx = b0 + hl;
        const bool mine = (side ? stop[1] : stop[0]) < 0 && idx < kStepOutCap;
        float t = side ? base[1] : base[0];
#pragma unroll
        for (int i = 0; i < H - 1; ++i)
          if (i < hl) t += delta;
        bool isn = false;
        float ll = 0.0f;
        const bool pin = probe(t, ll, isn);
        ran += mine;
        const bool mine_open = (side ? stop[1] : stop[0]) < 0;
        const bool halt = mine_open && (idx >= kStepOutCap || !pin);
        const unsigned hb = (__ballot_sync(kAll, halt) >> gshift) & (G == 32 ? 0xffffffffu : (1u << G) - 1u);
        const unsigned nb = (__ballot_sync(kAll, mine && isn) >> gshift) & (G == 32 ? 0xffffffffu : (1u << G) - 1u);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const unsigned hq = (hb >> (q * H)) & kHalf, nq = (nb >> (q * H)) & kHalf;
          const int fq = __ffs(hq) - 1;
          // the first halting end of side q, else its last end this round
          const float tq = __shfl_sync(kAll, t, q * H + (hq ? fq : H - 1), G);
          const bool open_q = stop[q] < 0;
          nanc += open_q ? __popc(hq ? (nq & ((2u << fq) - 1u)) : nq) : 0;
          ends[q] = (open_q && hq) ? tq : ends[q];
          base[q] = (open_q && !hq) ? tq + (q ? w : -w) : base[q];
          stop[q] = (open_q && hq) ? b0 + fq : stop[q];
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        exps += stop[q];
        if (stop[q] == kStepOutCap) ++capo;
      }
    } else {
      // one lane: the left side, then the right
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float delta = q ? w : -w;
        float t = ends[q];
        int n = 0;
        for (; n < kStepOutCap; ++n) {
          bool isn = false;
          float ll = 0.0f;
          const bool in = probe(t, ll, isn);
          ++ran;
          if (isn) ++nanc;
          if (!in) break;
          t += delta;
        }
        ends[q] = t;
        exps += n;
        if (n == kStepOutCap) ++capo;
      }
    }
    float tl = ends[0], tr = ends[1];
    // Shrinkage, at most kShrinkCap proposals, then a null move.  Proposal r
    // is t_r = tl_r + u_r (tr_r - tl_r) and a rejection moves the end on
    // t_r's side to t_r, so the brackets of the proposals that follow
    // rejections are known before any test: each round lanes [0, S) of the
    // group form S consecutive proposals (a short scan over the shared u's)
    // and test them at once; the first inside the slice is the sequential
    // result.  S = min(G, 4): most steps accept their first or second
    // proposal, and the scan's length is the round's cost.  Rounds run until
    // every group of the warp has accepted or used the cap; a group that has
    // accepted evaluates but counts and changes nothing.
    constexpr int S = G < 4 ? G : 4;
    static_assert(S <= kStepWords - 3 && kShrinkCap % S == 0, "first-round proposals are drawn ahead");
    bool ok = false;
    float tacc = 0.0f, llacc = 0.0f;
    constexpr unsigned kGroupBits = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    for (int b0 = 0; b0 < kShrinkCap && __any_sync(kAll, !ok); b0 += S) {
      ++rounds;
      active += ok ? 0 : 1;
      const int idx = b0 + gl;
      const bool mine = !ok && gl < S && idx < kShrinkCap;
      uint32_t wr;
      if (b0 == 0) {
        wr = wS;  // the first round's proposals were drawn ahead
      } else {
        // drawn ahead below word kStepWords, else from the counter; both
        // formed by every lane, so the warp does not split
        const uint32_t r = 3u + (uint32_t)idx, wi = nz + r;
        const uint32_t wp = pick(draw_block(R, iter, (uint32_t)j, (uint32_t)s, wi >> 2), wi & 3u);
        const uint32_t wl = (uint32_t)__ldg(ws + min(r, (uint32_t)kStepWords - 1u));
        wr = r < (uint32_t)kStepWords ? wl : wp;
      }
      const float u = u24(wr);
      float lo = tl, hi = tr, t = 0.0f;
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const float ui = __shfl_sync(kAll, u, i, G);
        const float ti = fmaf(ui, hi - lo, lo);
        if (i == gl) t = ti;
        if (ti < 0.0f) lo = ti;
        else hi = ti;
      }
      bool isn = false;
      float ll = 0.0f;
      const bool pin = probe(t, ll, isn);
      ran += mine;
      const unsigned inb = (__ballot_sync(kAll, mine && pin) >> gshift) & kGroupBits;
      const unsigned nanb = (__ballot_sync(kAll, mine && isn) >> gshift) & kGroupBits;
      const int f = inb ? __ffs(inb) - 1 : 0;
      const float tf = __shfl_sync(kAll, t, f, G);
      const float lf = __shfl_sync(kAll, ll, f, G);
      // a group still shrinking takes this round's outcome (by selects)
      const int nvalid = min(S, kShrinkCap - b0);
      shr += ok ? 0 : (inb ? f + 1 : nvalid);
      nanc += ok ? 0 : __popc(inb ? (nanb & ((1u << f) - 1u)) : nanb);
      tacc = (!ok && inb) ? tf : tacc;
      llacc = (!ok && inb) ? lf : llacc;
      tl = ok ? tl : lo;
      tr = ok ? tr : hi;
      ok = ok || inb != 0;
    }
    if (ok) {
#pragma unroll
      for (int i = 0; i < DPL; ++i) x[i] = fmaf(tacc, v[i], x[i]);
      lx = llacc;
    }
    if (ok) ++acc;
  }
  // group-parallel rounds test ends and proposals past the first decisive
  // one; those extra tests are counted apart from the logical evaluations
  {
    int tot = ran;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) tot += __shfl_xor_sync(kAll, tot, o, G);
    ran = tot;
  }
  const int nul = R.p - acc;
  const int evals = (R.kernel == kKernelRw) ? R.p : exps + 2 * R.p - capo + shr;
  // (iv) replace dead slot j, born at logL*
  const int slot = D.i[R.o_dead + j];
  if (live && has) store_lane<DPL>(D.f + R.o_x + (long long)slot * ld, gl, ld, x);
  if (live && gl == 0) {
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
    if (ran > evals) atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->spec_evals), (unsigned long long)(ran - evals));
    if (rounds) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->rounds), (unsigned long long)rounds);
      atomicAdd(reinterpret_cast<unsigned long long*>(&Sw->active_rounds), (unsigned long long)active);
    }
  }
}

// resident blocks per SM the register budget is tuned for
constexpr int sweep_min_blocks(int dpl) { return dpl <= 2 ? 20 : dpl == 4 ? 18 : dpl == 8 ? 12 : 12; }

template <int G, int DPL, int KC>
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
    const bool live = j < wi.c1;
    sweep_chain<G, DPL, KC>(D, D.desc[wi.run], S, live ? j : wi.c0, gl, mask, live);
    __syncwarp();
  }
}

template <int KC>
cudaError_t launch_sweep_kc(int cfg, const Dev& D, const WorkItem* items, int n, int* queue, int grid,
                            cudaStream_t s) {
  switch (cfg) {
#define X(id, g, p) case id: k_sweep<g, p, KC><<<grid, kSweepThreads, 0, s>>>(D, items, n, queue); break;
    NSS_CFGS(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KC>
int sweep_blocks_per_sm_kc(int cfg) {
  int nb = 0;
  switch (cfg) {
#define X(id, g, p) case id: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<g, p, KC>, kSweepThreads, 0); break;
    NSS_CFGS(X)
#undef X
    default: break;
  }
  return nb > 0 ? nb : 1;
}

}  // namespace nss
