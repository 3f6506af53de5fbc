// nss_logreg.cu -- Bayesian logistic regression likelihood inside the HRSS
// sweep (Sec. 4.2 workloads; the sweep of Sec. 3.2 / App. B.4), for sm_103a.
//
// logL(x) = sum_n [y_n z_n - softplus(z_n)],  z = X x,  X the N x d design.
//
// Along an HRSS line x + t v the logits are affine in t:
//   z(t) = X x + t X v,
// so each step needs one product X v per chain (and X x once per chain per
// outer iteration for the parent), and every slice evaluation of that step is
// N fused multiply-adds and N softplus terms.  The products of all chains are
// one batched contraction Z = X [u_1 ... u_k], computed on the 5th-generation
// tensor cores: tcgen05.mma kind::f16 with BF16 operands and FP32
// accumulation in tensor memory, operands staged by TMA.  X holds bfloat16
// values exactly (the data set is bf16-exact); each FP32 vector u is split
// into three bfloat16 parts u = u_hi + u_mid + u_lo (|u - sum| <= 2^-24 |u|),
// so the contraction reproduces FP32 products.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"
#include "nss_tc.cuh"

namespace nss {

// ---------------------------------------------------------------------------
// Tensor-core contraction  out[c][r] = sum_p sum_k X[r][k] * U_p[c][k]
//   X   : bf16 [rows_pad][128]          (tensor map mapX, box 64 x 128)
//   U   : bf16 [3][cols_pad][128]       (tensor map mapU, box 64 x 128)
//   out : fp32 [cols][ldo]              (tensor map mapO, extents n_rows x
//                                        n_cols, box 128 rows x 32 columns)
// Persistent, warp-specialised: block b owns the 128-column tile b mod nct
// and the row tiles b / nct, b / nct + G / nct, ... (G blocks, a multiple of
// nct).  Warp 4 issues the TMA loads: the block's three U parts once, then
// each row tile's X into one of two stages; warp 5 issues the 24 MMAs of a
// tile (K = 128 in 8 steps x 3 bf16 parts) into one of two 128-column TMEM
// accumulators; warps 0-3 read an accumulator back (tcgen05.ld) 32 columns at
// a time, transpose them through one of two shared-memory staging buffers
// (chain-major, the output's layout) and thread 0 writes each 128 x 32 piece
// with one TMA store, while the next tile's loads and products proceed.
// Scalar stores from the epilogue threads had cost ~4 us per tile (the
// launch's bound); the TMA store writes whole lines.  Stages and
// accumulators are handed over by mbarriers (transaction counts for the
// loads, tcgen05.commit for the products, 128 arrivals for the drained
// accumulator), the staging buffers by bulk-group waits and a named barrier
// of the four epilogue warps; every mbarrier wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kTile = 128;
constexpr uint32_t kChunkBytes = 128u * 64u * 2u;   // 128 rows x 64 bf16
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr int kLogitsThreads = 192;                 // warps 0-3 epilogue, 4 loads, 5 products
constexpr uint32_t kStageBytes = 32u * 128u * 4u;  // 32 columns x 128 rows fp32
// U: 3 parts x 2 chunks; X: 2 stages x 2 chunks; two output staging buffers
constexpr int kLogitsSmem = 10 * kChunkBytes + 2 * kStageBytes + 1024;

__global__ void __launch_bounds__(kLogitsThreads, 1) k_logits(const __grid_constant__ CUtensorMap mapX,
                                                               const __grid_constant__ CUtensorMap mapU,
                                                               const __grid_constant__ CUtensorMap mapO, int cols_pad,
                                                               int n_rows, int n_cols, int* __restrict__ err,
                                                               const int* __restrict__ skip,
                                                               const float* __restrict__ zref) {
  if (skip && *skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* B = base;                      // [3 parts][2 chunks]
  uint8_t* A = base + 6 * kChunkBytes;    // [2 stages][2 chunks]
  __shared__ __align__(8) uint64_t bfull, afull[2], aempty[2], dfull[2], dempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nct = (n_cols + kTile - 1) / kTile, nrt = (n_rows + kTile - 1) / kTile;
  const int per = gridDim.x / nct;        // blocks per column tile
  const int ct = blockIdx.x % nct, rt0 = blockIdx.x / nct;
  const int col0 = ct * kTile;
  const int ntiles = rt0 < nrt ? (nrt - rt0 + per - 1) / per : 0;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bfull, 1);
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&afull[s], 1);
      tc::mbar_init(&aempty[s], 1);
      tc::mbar_init(&dfull[s], 1);
      tc::mbar_init(&dempty[s], 128);
    }
    failed = 0;
    tc::fence_mbar_init();
  }
  if (warp == 5) {
    tc::tmem_alloc(&tmem_base, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 4) {
    if (lane == 0 && ntiles > 0) {
      tc::mbar_arrive_expect_tx(&bfull, 6 * kChunkBytes);
      for (int p = 0; p < 3; ++p)
        for (int c = 0; c < 2; ++c)
          tc::tma_load_2d(B + (p * 2 + c) * kChunkBytes, &mapU, &bfull, c * 64, p * cols_pad + col0);
      for (int i = 0; i < ntiles; ++i) {
        const int s = i & 1;
        if (i >= 2 && !tc::mbar_wait(&aempty[s], ((i >> 1) - 1) & 1, kMaxPolls)) {
          atomicExch(err, 1);
          failed = 1;
          break;
        }
        const int row0 = (rt0 + i * per) * kTile;
        tc::mbar_arrive_expect_tx(&afull[s], 2 * kChunkBytes);
        for (int c = 0; c < 2; ++c) tc::tma_load_2d(A + (s * 2 + c) * kChunkBytes, &mapX, &afull[s], c * 64, row0);
      }
    }
  } else if (warp == 5) {
    if (lane == 0 && ntiles > 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kTile, kTile);
      bool ok = tc::mbar_wait(&bfull, 0, kMaxPolls);
      for (int i = 0; i < ntiles && ok; ++i) {
        const int s = i & 1;
        ok = tc::mbar_wait(&afull[s], (i >> 1) & 1, kMaxPolls);
        if (ok && i >= 2) ok = tc::mbar_wait(&dempty[s], ((i >> 1) - 1) & 1, kMaxPolls);
        if (!ok) break;
        tc::fence_after_sync();
        uint32_t acc = 0;
        for (int c = 0; c < 2; ++c)
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(A + (s * 2 + c) * kChunkBytes) + kk * 32);
              const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(B + (p * 2 + c) * kChunkBytes) + kk * 32);
              tc::mma_bf16(tmem + (uint32_t)(s * kTile), ad, bd, idesc, acc);
              acc = 1;
            }
        tc::mma_commit(&aempty[s]);
        tc::mma_commit(&dfull[s]);
      }
      if (!ok) {
        atomicExch(err, 2);
        failed = 1;
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of the tile);
    // staging buffer b holds a piece as [32 columns][128 rows]
    float* stage = reinterpret_cast<float*>(base + 10 * kChunkBytes);
    const int lr = warp * 32 + lane;
    int piece = 0;
    for (int i = 0; i < ntiles; ++i) {
      const int s = i & 1;
      // the four warps agree on the outcome, so they leave together and no
      // named barrier below waits for a warp that has gone
      const bool ok = tc::named_bar_and(1, 128, tc::mbar_wait(&dfull[s], (i >> 1) & 1, kMaxPolls));
      if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 3);
        break;
      }
      tc::fence_after_sync();
      const int row0 = (rt0 + i * per) * kTile;
      const int r = row0 + lr;
      const float z0 = (zref && r < n_rows) ? zref[r] : 0.0f;
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc, ++piece) {
        float v[32];
        tc::tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(s * kTile + cc * 32), v);
        float* buf = stage + (piece & 1) * (32 * 128);
        // the store issued from this buffer two pieces ago has read it
        if (threadIdx.x == 0) tc::bulk_wait_read<1>();
        tc::named_bar_sync(1, 128);
#pragma unroll
        for (int q = 0; q < 32; ++q) buf[q * 128 + lr] = v[q] + z0;
        tc::fence_proxy_async_smem();
        tc::named_bar_sync(1, 128);
        if (threadIdx.x == 0) {
          tc::tma_store_2d(&mapO, buf, row0, col0 + cc * 32);
          tc::bulk_commit();
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&dempty[s]);
    }
    // every store complete before the block ends (and its shared memory goes)
    if (threadIdx.x == 0) tc::bulk_wait<0>();
  }
  // let any load or product still in flight land before shared and tensor
  // memory go away (after a wait that ran out; bounded)
  __syncthreads();
  if (failed && threadIdx.x == 0) {
    tc::mbar_wait(&bfull, 0, kMaxPolls);
    for (int s = 0; s < 2; ++s) tc::mbar_wait(&afull[s], 0, kMaxPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 5) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// FP32 -> three bfloat16 parts: h = bf16(u), m = bf16(u - h), l = bf16(u - h - m)
// (each difference is exact in FP32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split3(float u, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(u);
  const float r1 = u - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ void write_parts(__nv_bfloat16* parts, long long part_stride, int row, int t,
                                            float u) {
  __nv_bfloat16 h, m, l;
  split3(u, h, m, l);
  parts[static_cast<long long>(row) * 128 + t] = h;
  parts[part_stride + static_cast<long long>(row) * 128 + t] = m;
  parts[2 * part_stride + static_cast<long long>(row) * 128 + t] = l;
}

// ---------------------------------------------------------------------------
// Chain start of an outer iteration: copy each chain's parent into its
// working position, clear its counters, and split the positions for the
// contraction X x_parent.  Block j = chain j, thread t = dimension t.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lr_parents(Dev D, LRArgs A, int run) {
  const RunDesc& R = D.desc[run];
  if (D.st[run].done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const int parent = D.i[R.o_parent + j];
  const float x = (t < R.d) ? D.f[R.o_x + static_cast<long long>(parent) * R.dpad + t] : 0.0f;
  A.xc[static_cast<long long>(j) * 128 + t] = x;
  write_parts(A.parts, A.part_stride, j, t, (t < R.d) ? x - A.center[t] : 0.0f);
  if (t == 0) A.lc[j] = D.f[R.o_logL + parent];
  if (t < 6) D.i[R.o_stats + t * R.k + j] = 0;
}

// The initial live set: split every live point for the contraction X x.
__global__ void __launch_bounds__(128) k_lr_live_parts(Dev D, LRArgs A, int run) {
  const RunDesc& R = D.desc[run];
  const int s = blockIdx.x, t = threadIdx.x;
  if (s >= R.m) return;
  const float x = (t < R.d) ? D.f[R.o_x + static_cast<long long>(s) * R.dpad + t] : 0.0f;
  write_parts(A.parts, A.part_stride, s, t, (t < R.d) ? x - A.center[t] : 0.0f);
}

// Centre of the contraction: the live-set mean mu (FP64 sums), and the
// reference logits X mu (FP64 dot products), so that the tensor cores only
// contract the small offsets x - mu.
__global__ void __launch_bounds__(128) k_lr_center(Dev D, LRArgs A, int run) {
  const RunDesc& R = D.desc[run];
  if (D.st[run].done) return;
  const int t = threadIdx.x;
  double s = 0.0;
  if (t < R.d)
    for (int i = 0; i < R.m; ++i) s += (double)D.f[R.o_x + static_cast<long long>(i) * R.dpad + t];
  A.center[t] = (t < R.d) ? static_cast<float>(s / R.m) : 0.0f;
}

__global__ void __launch_bounds__(256) k_lr_zref(Dev D, LRArgs A, int run) {
  const RunDesc& R = D.desc[run];
  if (D.st[run].done) return;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= R.n_data) return;
  const __nv_bfloat16* xr = A.Xb + static_cast<long long>(n) * 128;
  double s = 0.0;
  for (int i = 0; i < R.d; ++i) s += (double)__bfloat162float(xr[i]) * (double)A.center[i];
  A.zref[n] = static_cast<float>(s);
}

// ---------------------------------------------------------------------------
// Per-chain block reductions over the N logits (512 threads, thread t owns
// elements n = t + 512 i).
// ---------------------------------------------------------------------------
constexpr int kLRThreads = 512;

__device__ __forceinline__ float2 block_sum2(float a, float b, float2* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) red[wid] = make_float2(a, b);
  __syncthreads();
  if (wid == 0) {
    float2 v = (lane < (kLRThreads >> 5)) ? red[lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) red[32] = v;
  }
  __syncthreads();
  const float2 r = red[32];
  __syncthreads();
  return r;
}

// y z - softplus(z), softplus(z) = max(z, 0) + log(1 + e^-|z|)
__device__ __forceinline__ float bern_logit(float z, bool y) {
  const float sp = fmaxf(z, 0.0f) + __logf(1.0f + __expf(-fabsf(z)));
  return (y ? z : 0.0f) - sp;
}

// logL of rows of a logits matrix (the initial live set)
template <int EMAX>
__global__ void __launch_bounds__(kLRThreads) k_lr_rowll(Dev D, LRArgs A, int run) {
  __shared__ float2 red[33];
  const RunDesc& R = D.desc[run];
  const int s = blockIdx.x, t = threadIdx.x;
  if (s >= R.m) return;
  const uint32_t yb = A.ybits[t];
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    const int n = t + kLRThreads * i;
    if (n < R.n_data) acc += bern_logit(A.zx[static_cast<long long>(s) * A.ldz + n], (yb >> i) & 1u);
  }
  const float2 tot = block_sum2(acc, 0.0f, red);
  if (t == 0) {
    const float ll = isnan(tot.x) ? -INFINITY : tot.x;
    D.f[R.o_logL + s] = ll;
    D.f[R.o_birth + s] = -INFINITY;
  }
}

// ---------------------------------------------------------------------------
// Direction of HRSS step s for every chain: z ~ N(0, I) from words
// [0, 2 ceil(d/2)) of counter (iteration, chain, s, .), d~ = L z,
// v = d~/|z| (or d~/|d~|).  Block j = chain j, thread t = dimension t.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lr_dir(Dev D, LRArgs A, int run, int step) {
  __shared__ float zs[128];
  __shared__ float red[4];
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  if (S.done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const uint32_t iter = static_cast<uint32_t>(S.iter);
  float z = 0.0f;
  if (t < R.d) {
    const uint4 w = draw_block(R, iter, static_cast<uint32_t>(j), static_cast<uint32_t>(step),
                               static_cast<uint32_t>(t >> 2));
    float a, b;
    if (t & 2) box_muller(w.z, w.w, a, b);
    else box_muller(w.x, w.y, a, b);
    z = (t & 1) ? b : a;
  }
  zs[t] = z;
  float zz = z * z;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
  if ((t & 31) == 0) red[t >> 5] = zz;
  __syncthreads();
  zz = red[0] + red[1] + red[2] + red[3];
  float dt = 0.0f;
  if (t < R.d) {
    const float* Lr = D.f + R.o_L + static_cast<long long>(t) * R.dpad;
    for (int b = 0; b <= t; ++b) dt = fmaf(Lr[b], zs[b], dt);
  }
  float inrm;
  if (R.dir_norm == 0) {
    inrm = rsqrtf(zz);
  } else {
    __syncthreads();
    float dd = dt * dt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
    if ((t & 31) == 0) red[t >> 5] = dd;
    __syncthreads();
    inrm = rsqrtf(red[0] + red[1] + red[2] + red[3]);
  }
  const float v = (t < R.d) ? dt * inrm : 0.0f;
  A.vdir[static_cast<long long>(j) * 128 + t] = v;
  write_parts(A.parts, A.part_stride, j, t, v);
}

// ---------------------------------------------------------------------------
// HRSS step s of every chain along its line, with the logits affine in t.
// Block j = chain j (512 threads).  Slice test: prior slice height under the
// N(a, b^2) prior, then logL > logL* (strict).  Words: U at nz, height at
// nz+1, shrinkage r at nz+3+r, nz = 2 ceil(d/2) (the same layout as every
// other likelihood).
// ---------------------------------------------------------------------------
template <int EMAX>
__global__ void __launch_bounds__(kLRThreads, 2) k_lr_slice(Dev D, LRArgs A, int run, int step) {
  __shared__ float2 red[33];
  const RunDesc& R = D.desc[run];
  RunState* S = D.st + run;
  if (S->done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const uint32_t iter = static_cast<uint32_t>(S->iter);
  const float lstar = S->logLstar;
  const int N = R.n_data, d = R.d;
  float zx[EMAX], zv[EMAX];
  const long long rowz = static_cast<long long>(j) * A.ldz;
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    const int n = t + kLRThreads * i;
    zx[i] = (n < N) ? A.zx[rowz + n] : 0.0f;
    zv[i] = (n < N) ? A.zv[rowz + n] : 0.0f;
  }
  const uint32_t yb = A.ybits[t];
  const bool own = t < d;
  float xt = own ? A.xc[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float vt = own ? A.vdir[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float at = own ? D.f[R.o_a + t] : 0.0f;
  const float ibt = own ? 1.0f / D.f[R.o_b + t] : 0.0f;
  float lx = A.lc[j];

  const uint32_t nz = 2u * static_cast<uint32_t>((d + 1) >> 1);
  uint32_t cblk = 0xFFFFFFFFu;
  uint4 cw = make_uint4(0, 0, 0, 0);
  auto word = [&](uint32_t wi) {
    if ((wi >> 2) != cblk) {
      cblk = wi >> 2;
      cw = draw_block(R, iter, static_cast<uint32_t>(j), static_cast<uint32_t>(step), cblk);
    }
    return pick(cw, wi & 3u);
  };
  // prior slice height: log Pi(x) + ln u
  float ux = own ? (xt - at) * ibt : 0.0f;
  const float2 px = block_sum2(-0.5f * ux * ux, 0.0f, red);
  const float height = px.x + R.prior_const + logf(u24(word(nz + 1u)));

  int evals = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
  auto in_slice = [&](float tt, float& ll) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < EMAX; ++i) {
      const int n = t + kLRThreads * i;
      if (n < N) acc += bern_logit(fmaf(tt, zv[i], zx[i]), (yb >> i) & 1u);
    }
    const float yt = fmaf(tt, vt, xt);
    const float u = own ? (yt - at) * ibt : 0.0f;
    const float2 tot = block_sum2(acc, -0.5f * u * u, red);
    ++evals;
    ll = tot.x;
    if (isnan(ll)) {
      ll = -INFINITY;
      ++nanc;
    }
    const float lp = tot.y + R.prior_const;
    return (lp > height) && (ll > lstar);
  };

  const float w = R.w;
  const float U = u24(word(nz));
  float tl = -w * U, tr = tl + w, lly;
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
  float tacc = 0.0f;
  for (int r = 0; r < kShrinkCap; ++r) {
    const float u = u24(word(nz + 3u + static_cast<uint32_t>(r)));
    const float tt = fmaf(u, tr - tl, tl);
    ++shr;
    if (in_slice(tt, lly)) {
      ok = true;
      tacc = tt;
      lx = lly;
      break;
    }
    if (tt < 0.0f) tl = tt;
    else tr = tt;
  }
  if (ok) {
#pragma unroll
    for (int i = 0; i < EMAX; ++i) {
      const int n = t + kLRThreads * i;
      if (n < N) A.zx[rowz + n] = fmaf(tacc, zv[i], zx[i]);
    }
    if (own) A.xc[static_cast<long long>(j) * 128 + t] = fmaf(tacc, vt, xt);
  }
  if (t == 0) {
    A.lc[j] = lx;
    int* st = D.i + R.o_stats;
    st[j] += evals;
    st[R.k + j] += ok ? 1 : 0;
    st[2 * R.k + j] += ok ? 0 : 1;
    st[3 * R.k + j] += exps;
    st[4 * R.k + j] += shr;
    st[5 * R.k + j] += capo;
    atomicAdd(reinterpret_cast<unsigned long long*>(&S->evals), static_cast<unsigned long long>(evals));
    if (!ok) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nulls), 1ull);
    if (capo) atomicAdd(reinterpret_cast<unsigned long long*>(&S->cap_out), static_cast<unsigned long long>(capo));
    if (nanc) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nan_evals), static_cast<unsigned long long>(nanc));
  }
}

// (iv) replace dead slot j with chain j's final point, born at logL*
__global__ void __launch_bounds__(128) k_lr_replace(Dev D, LRArgs A, int run) {
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  if (S.done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const int slot = D.i[R.o_dead + j];
  if (t < R.dpad) D.f[R.o_x + static_cast<long long>(slot) * R.dpad + t] = (t < R.d) ? A.xc[static_cast<long long>(j) * 128 + t] : 0.0f;
  if (t == 0) {
    D.f[R.o_logL + slot] = A.lc[j];
    D.f[R.o_birth + slot] = S.logLstar;
  }
}

// ---------------------------------------------------------------------------
// The plain path's logistic HRSS step (direct evaluation, the comparator of
// the line-affine form above): the k chains advance in lockstep evaluation
// rounds; each round every chain still testing proposes its next slice test
// (the next stepping-out end or shrinkage proposal of the sequential
// algorithm), the logits of all k candidate points are one tensor-core GEMM
// (k_logits over their bf16 parts), and each chain's block reduces its
// Bernoulli sum and takes the transition.  Same words and counters as
// k_lr_slice.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lr_direct_init(Dev D, LRArgs A, LRDirect* st, int run, int step) {
  __shared__ float red[4];
  const RunDesc& R = D.desc[run];
  const RunState& S = D.st[run];
  if (S.done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const uint32_t iter = static_cast<uint32_t>(S.iter);
  const bool own = t < R.d;
  const float xt = own ? A.xc[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float ux = own ? (xt - D.f[R.o_a + t]) * (1.0f / D.f[R.o_b + t]) : 0.0f;
  float v = -0.5f * ux * ux;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    const uint32_t nz = 2u * static_cast<uint32_t>((R.d + 1) >> 1);
    const uint4 b0 = draw_block(R, iter, (uint32_t)j, (uint32_t)step, nz >> 2);
    const uint32_t wU = pick(b0, nz & 3u);
    const uint32_t wi = nz + 1u;
    const uint32_t wH = ((wi >> 2) == (nz >> 2)) ? pick(b0, wi & 3u)
                                                 : pick(draw_block(R, iter, (uint32_t)j, (uint32_t)step, wi >> 2), wi & 3u);
    LRDirect c{};
    c.height = (red[0] + red[1] + red[2] + red[3]) + R.prior_const + logf(u24(wH));
    c.tl = -R.w * u24(wU);
    c.tr = c.tl + R.w;
    c.t = c.tl;
    c.phase = 0;
    st[j] = c;
  }
}

// bf16 parts of the candidate point y = x + t v, centred (phase 3: unchanged)
__global__ void __launch_bounds__(128) k_lr_direct_cand(Dev D, LRArgs A, const LRDirect* st, int run) {
  const RunDesc& R = D.desc[run];
  if (D.st[run].done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  const LRDirect c = st[j];
  if (c.phase == 3) return;
  const bool own = t < R.d;
  const float xt = own ? A.xc[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float vt = own ? A.vdir[static_cast<long long>(j) * 128 + t] : 0.0f;
  write_parts(A.parts, A.part_stride, j, t, own ? fmaf(c.t, vt, xt) - A.center[t] : 0.0f);
}

template <int EMAX>
__global__ void __launch_bounds__(kLRThreads) k_lr_direct_eval(Dev D, LRArgs A, LRDirect* st, int run, int step,
                                                               int* active) {
  __shared__ float2 red[33];
  __shared__ int accepted;
  const RunDesc& R = D.desc[run];
  RunState* S = D.st + run;
  if (S->done) return;
  const int j = blockIdx.x, t = threadIdx.x;
  if (j >= R.k) return;
  LRDirect c = st[j];
  if (c.phase == 3) return;  // the same for the whole block
  const int N = R.n_data, d = R.d;
  const uint32_t yb = A.ybits[t];
  const long long rowz = static_cast<long long>(j) * A.ldz;
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < EMAX; ++i) {
    const int n = t + kLRThreads * i;
    if (n < N) acc += bern_logit(A.zx[rowz + n], (yb >> i) & 1u);
  }
  const bool own = t < d;
  const float xt = own ? A.xc[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float vt = own ? A.vdir[static_cast<long long>(j) * 128 + t] : 0.0f;
  const float yt = fmaf(c.t, vt, xt);
  const float u = own ? (yt - D.f[R.o_a + t]) * (1.0f / D.f[R.o_b + t]) : 0.0f;
  const float2 tot = block_sum2(acc, -0.5f * u * u, red);
  if (t == 0) {
    const bool nan = isnan(tot.x);
    const float ll = nan ? -INFINITY : tot.x;
    const bool in = (tot.y + R.prior_const > c.height) && (ll > S->logLstar);
    const uint32_t iter = static_cast<uint32_t>(S->iter);
    const uint32_t nz = 2u * static_cast<uint32_t>((d + 1) >> 1);
    auto shrink = [&](int r) {
      const uint32_t wi = nz + 3u + static_cast<uint32_t>(r);
      const float uu = u24(pick(draw_block(R, iter, (uint32_t)j, (uint32_t)step, wi >> 2), wi & 3u));
      return fmaf(uu, c.tr - c.tl, c.tl);
    };
    ++c.evals;
    c.nanc += nan ? 1 : 0;
    int acc_now = 0;
    if (c.phase == 0 || c.phase == 1) {
      const bool left = c.phase == 0;
      if (in) {
        if (left) c.tl -= R.w;
        else c.tr += R.w;
        ++c.e;
        ++c.exps;
      }
      const bool stop = !in || c.e == kStepOutCap;
      if (in && c.e == kStepOutCap) ++c.capo;
      if (!stop) {
        c.t = left ? c.tl : c.tr;
      } else if (left) {
        c.phase = 1;
        c.e = 0;
        c.t = c.tr;
      } else {
        c.phase = 2;
        c.r = 0;
        c.t = shrink(0);
      }
    } else {
      ++c.shr;
      if (in) {
        acc_now = 1;
        ++c.acc;
        A.lc[j] = ll;
        c.phase = 3;
      } else {
        if (c.t < 0.0f) c.tl = c.t;
        else c.tr = c.t;
        ++c.r;
        if (c.r == kShrinkCap) c.phase = 3;
        else c.t = shrink(c.r);
      }
    }
    if (c.phase == 3) {
      int* sts = D.i + R.o_stats;
      sts[j] += c.evals;
      sts[R.k + j] += acc_now;
      sts[2 * R.k + j] += 1 - acc_now;
      sts[3 * R.k + j] += c.exps;
      sts[4 * R.k + j] += c.shr;
      sts[5 * R.k + j] += c.capo;
      atomicAdd(reinterpret_cast<unsigned long long*>(&S->evals), static_cast<unsigned long long>(c.evals));
      if (!acc_now) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nulls), 1ull);
      if (c.capo) atomicAdd(reinterpret_cast<unsigned long long*>(&S->cap_out), static_cast<unsigned long long>(c.capo));
      if (c.nanc) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nan_evals), static_cast<unsigned long long>(c.nanc));
    } else {
      atomicAdd(active, 1);
    }
    accepted = acc_now;
    st[j] = c;
  }
  __syncthreads();
  if (accepted && own) A.xc[static_cast<long long>(j) * 128 + t] = yt;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// bf16 matrix [rows][128] in global memory, box 64 columns x 128 rows, 128-byte swizzle
bool make_map_bf16(CUtensorMap* map, void* base, unsigned long long rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {128, rows};
  const cuuint64_t strides[1] = {128 * 2};
  const cuuint32_t box[2] = {64, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

cudaError_t setup_logits_attributes() {
  return cudaFuncSetAttribute(k_logits, cudaFuncAttributeMaxDynamicSharedMemorySize, kLogitsSmem);
}

// fp32 [n_cols][ld] output written by TMA stores of 128 rows x 32 columns
// (rows past n_rows and columns past n_cols are not written)
static bool make_map_out(CUtensorMap* map, float* base, long long ld, int n_rows, int n_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (ld * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n_rows, (cuuint64_t)n_cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {128, 32};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// out: fp32 [n_cols][ldo], written by TMA stores, so `out` must be 16-byte
// aligned and ldo a multiple of 4 (else cudaErrorInvalidValue, nothing launched)
cudaError_t launch_logits(const CUtensorMap& mapX, const CUtensorMap& mapU, int rows_pad, int cols_pad, float* out,
                          long long ldo, int n_rows, int n_cols, int* err, const int* skip, const float* zref,
                          cudaStream_t s) {
  if (n_cols < 1 || n_rows < 1 || n_rows > rows_pad || ldo < n_rows) return cudaErrorInvalidValue;
  CUtensorMap mapO;
  if (!make_map_out(&mapO, out, ldo, n_rows, n_cols)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one block per SM, a whole number of blocks per column tile
  const int nct = (n_cols + kTile - 1) / kTile, nrt = (n_rows + kTile - 1) / kTile;
  const int per = std::max(1, std::min(nrt, std::max(1, sms) / nct));
  k_logits<<<nct * per, kLogitsThreads, kLogitsSmem, s>>>(mapX, mapU, mapO, cols_pad, n_rows, n_cols, err, skip, zref);
  return cudaGetLastError();
}

cudaError_t launch_lr_parents(const Dev& D, const LRArgs& A, int run, int k, cudaStream_t s) {
  k_lr_parents<<<k, 128, 0, s>>>(D, A, run);
  return cudaGetLastError();
}
cudaError_t launch_lr_center(const Dev& D, const LRArgs& A, int run, int n_data, cudaStream_t s) {
  k_lr_center<<<1, 128, 0, s>>>(D, A, run);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_lr_zref<<<(n_data + 255) / 256, 256, 0, s>>>(D, A, run);
  return cudaGetLastError();
}

cudaError_t launch_lr_live_parts(const Dev& D, const LRArgs& A, int run, int m, cudaStream_t s) {
  k_lr_live_parts<<<m, 128, 0, s>>>(D, A, run);
  return cudaGetLastError();
}
cudaError_t launch_lr_rowll(const Dev& D, const LRArgs& A, int run, int m, int emax, cudaStream_t s) {
  if (emax <= 4) k_lr_rowll<4><<<m, kLRThreads, 0, s>>>(D, A, run);
  else if (emax <= 20) k_lr_rowll<20><<<m, kLRThreads, 0, s>>>(D, A, run);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t launch_lr_dir(const Dev& D, const LRArgs& A, int run, int k, int step, cudaStream_t s) {
  k_lr_dir<<<k, 128, 0, s>>>(D, A, run, step);
  return cudaGetLastError();
}
cudaError_t launch_lr_slice(const Dev& D, const LRArgs& A, int run, int k, int step, int emax, cudaStream_t s) {
  if (emax <= 4) k_lr_slice<4><<<k, kLRThreads, 0, s>>>(D, A, run, step);
  else if (emax <= 20) k_lr_slice<20><<<k, kLRThreads, 0, s>>>(D, A, run, step);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t launch_lr_direct_init(const Dev& D, const LRArgs& A, LRDirect* st, int run, int k, int step,
                                  cudaStream_t s) {
  k_lr_direct_init<<<k, 128, 0, s>>>(D, A, st, run, step);
  return cudaGetLastError();
}
cudaError_t launch_lr_direct_cand(const Dev& D, const LRArgs& A, const LRDirect* st, int run, int k, cudaStream_t s) {
  k_lr_direct_cand<<<k, 128, 0, s>>>(D, A, st, run);
  return cudaGetLastError();
}
cudaError_t launch_lr_direct_eval(const Dev& D, const LRArgs& A, LRDirect* st, int run, int k, int step, int emax,
                                  int* active, cudaStream_t s) {
  if (emax <= 4) k_lr_direct_eval<4><<<k, kLRThreads, 0, s>>>(D, A, st, run, step, active);
  else if (emax <= 20) k_lr_direct_eval<20><<<k, kLRThreads, 0, s>>>(D, A, st, run, step, active);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t launch_lr_replace(const Dev& D, const LRArgs& A, int run, int k, cudaStream_t s) {
  k_lr_replace<<<k, 128, 0, s>>>(D, A, run);
  return cudaGetLastError();
}

// Self-test of the bounded wait: an mbarrier whose phase never completes
// (nothing arrives on it) makes mbar_wait give up after max_polls polls; the
// kernel reports that (2) instead of spinning, and returns.
__global__ void k_wait_selftest(int* out, uint32_t max_polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  const bool done = tc::mbar_wait(&bar, 0, max_polls);
  if (threadIdx.x == 0) out[0] = done ? 1 : 2;
}

cudaError_t launch_wait_selftest(int* out, uint32_t max_polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(out, max_polls);
  return cudaGetLastError();
}

}  // namespace nss
