// nss_gp_tc.cu -- the GP hyperparameter likelihood of the HRSS sweep with the
// kernel-matrix factorisation on the 5th-generation tensor cores (the GP
// workloads of Sec. 4.3: the time of a GP evaluation is its Cholesky
// factorisation), for sm_103a.
//
// theta = (ln l, ln a, ln s); for data (t_i, y_i), i < n <= 256,
//   K_ij = a^2 exp(-(t_i - t_j)^2 / (2 l^2)) + s^2 [i == j],
//   log p(y | theta) = -1/2 |alpha|^2 - sum_i ln L_ii - n/2 ln 2 pi,
//   K = L L^T, alpha = L^-1 y.
//
// One block of 256 threads per SM holds one candidate's matrix at a time,
// padded to np = 32 ceil(n / 32) rows with an identity block, in tensor
// memory: row i in TMEM lane i mod 128, columns (i div 128) * 256 + j, so
// the two 128-row halves fill all 512 columns.  Thread i owns row i.  The
// factorisation is right-looking in panels of 32 columns:
//   - the panel's columns of rows >= j0 come from TMEM (tcgen05.ld);
//   - the 32 x 32 diagonal block is factored in the registers of the warp
//     that owns its rows, one column per step with shuffles (pivot
//     reciprocal square roots from rsqrtf, each L_jj as pivot x
//     rsqrt(pivot)), and its factor goes to shared memory;
//   - each row below solves its panel entries against that factor, and the
//     diagonal block's rows give the panel's part of alpha by forward
//     substitution; the rows below subtract it from their part of y;
//   - the trailing matrix takes D -= L21 L21^T on the tensor cores:
//     tcgen05.mma kind::tf32 (M = 128 per half, N = the trailing columns,
//     K = 32 in four instructions), accumulating into TMEM in FP32.  L21
//     is split into two TF32 parts hi + lo and the product is formed as
//     hi hi^T + hi lo^T + lo hi^T (the 3xTF32 scheme: each product to about
//     2^-21 relative, near an FP32 product), with the instruction's
//     negate-A flag making each product a subtraction.  The panel is staged
//     in shared memory as K-major rows of 32 FP32 words (128 B) in the
//     128-byte swizzled layout.
// ln det and |alpha|^2 accumulate in FP64.  A non-positive or non-finite
// FP32 pivot makes logL = -inf (counted with the NaN evaluations).  Every
// wait on the tensor core is bounded; a wait that runs out sets the error
// flag and the kernel frees its tensor memory and returns.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"
#include "nss_tc.cuh"

namespace nss {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcMaxN = 256;
constexpr int kTcCols = 512;                               // TMEM columns: two 128-row halves of 256
constexpr uint32_t kTcMaxPolls = 1u << 22;
constexpr uint32_t kTcPartBytes = kTcMaxN * 32 * 4;        // 256 rows x 32 FP32 words
// dynamic shared memory: the panel's two parts plus alignment slack (a single
// block fits per SM, as it must: it takes all of TMEM)
constexpr int kTcDynSmem = 2 * kTcPartBytes + 1024;

struct TcShared {
  float LT[32][32];   // the diagonal block's factor transposed (column cc in LT[cc]), 16-byte rows
  float inv[32];      // reciprocals of its diagonal
  float alpha[32];    // the panel's part of alpha
  float t[kTcMaxN], y[kTcMaxN];
  double ldet, qa;
  uint64_t bar;       // MMA completion
  uint32_t tmem;
  uint32_t phase;     // completed phases of `bar`
};

// logL of theta; every thread of the block calls it and gets the same value.
// Returns false (for every thread) when a tensor-core wait ran out.
// Panel buffers: phi / plo the TF32 parts of L21 (consecutive, kTcPartBytes
// each).
__device__ bool gp_loglik_tc(TcShared& sh, uint8_t* phi, int n, int np, const float th[3], float& out, int* err) {
  uint8_t* plo = phi + kTcPartBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t trow = sh.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((tid >> 7) * 256);
  const bool row_ok = tid < np;  // warp-uniform: np is a multiple of 32
  const float ell = expf(th[0]), amp = expf(th[1]), sn = expf(th[2]);
  const float a2 = amp * amp, s2 = sn * sn, c = -0.5f / (ell * ell);
  // lower part of row tid of K (chunks 0 .. warp) into TMEM; padded rows
  // and columns form an identity block
  if (row_ok) {
    const float ti = tid < n ? sh.t[tid] : 0.0f;
#pragma unroll 1
    for (int q = 0; q <= warp; ++q) {
      float v[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int j = 32 * q + e;
        if (tid < n && j < n) {
          const float dt = ti - sh.t[j];
          v[e] = a2 * expf(c * dt * dt) + (j == tid ? s2 : 0.0f);
        } else {
          v[e] = (j == tid) ? 1.0f : 0.0f;
        }
      }
      tc::tmem_st32(trow + (uint32_t)(32 * q), v);
    }
  }
  float r = (tid < n) ? sh.y[tid] : 0.0f;  // this row's part of y, less the solved panels
  if (tid == 0) {
    sh.ldet = 0.0;
    sh.qa = 0.0;
  }
  tc::fence_before_sync();
  __syncthreads();
  const int npan = np >> 5;
  bool waiting = false;
#pragma unroll 1
  for (int p = 0; p < npan; ++p) {
    const int j0 = 32 * p;
    if (waiting) {
      const bool okw = tc::mbar_wait(&sh.bar, sh.phase & 1u, kTcMaxPolls);
      waiting = false;
      if (!__syncthreads_and(okw ? 1 : 0)) {
        if (tid == 0) atomicExch(err, 3);
        return false;
      }
      if (tid == 0) sh.phase += 1;
      tc::fence_after_sync();
    }
    float a[32];
    if (warp >= p && row_ok) tc::tmem_ld32(trow + (uint32_t)j0, a);
    bool bad = false;
    if (warp == p) {
      // the diagonal block in this warp's registers: lane l holds row j0 + l
      // (a[e] = entry (j0 + l, j0 + e)).  Column c takes its pivot from lane
      // c, turns the lanes' entries of column c into factor entries (zeros
      // above the diagonal) and subtracts their outer product from the later
      // columns; the forward substitution of the block's part of alpha rides
      // along.  The panel's |alpha|^2 and log-diagonal terms are summed over
      // the warp in FP64 afterwards.
      float mine = 0.0f, myinv = 0.0f, mydiag = 1.0f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float piv = __shfl_sync(0xffffffffu, a[c], c);
        bad = bad || !(piv > 0.0f) || !isfinite(piv);  // the same in every lane
        const float rc = rsqrtf(piv);
        const float lcc = piv * rc;
        a[c] = lane > c ? a[c] * rc : (lane == c ? lcc : 0.0f);
        const float ac = __shfl_sync(0xffffffffu, r, c) * rc;
        if (lane > c) r = fmaf(-a[c], ac, r);
        if (lane == c) {
          mine = ac;
          myinv = rc;
          mydiag = lcc;
        }
#pragma unroll
        for (int q = c + 1; q < 32; ++q) a[q] = fmaf(-a[c], __shfl_sync(0xffffffffu, a[c], q), a[q]);
      }
      sh.alpha[lane] = mine;
      sh.inv[lane] = myinv;
#pragma unroll
      for (int c = 0; c < 32; ++c) sh.LT[c][lane] = a[c];
      double qa = (double)mine * (double)mine, ld = (double)logf(mydiag);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        qa += __shfl_xor_sync(0xffffffffu, qa, o);
        ld += __shfl_xor_sync(0xffffffffu, ld, o);
      }
      if (lane == 0) {
        sh.qa += qa;
        sh.ldet += ld;
      }
    }
    if (__syncthreads_or(bad ? 1 : 0)) {
      out = -INFINITY;
      return true;
    }
    if (warp > p && row_ok) {
      // rows below: their panel entries x = a L^-T (L the block's factor), column by column
      // (column cc of the factor read as 16-byte broadcasts)
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) {
        a[cc] *= sh.inv[cc];
#pragma unroll
        for (int b = (cc + 1) >> 2; b < 8; ++b) {
          const float4 l = *reinterpret_cast<const float4*>(&sh.LT[cc][4 * b]);
          if (4 * b > cc) a[4 * b] = fmaf(-a[cc], l.x, a[4 * b]);
          if (4 * b + 1 > cc) a[4 * b + 1] = fmaf(-a[cc], l.y, a[4 * b + 1]);
          if (4 * b + 2 > cc) a[4 * b + 2] = fmaf(-a[cc], l.z, a[4 * b + 2]);
          if (4 * b + 3 > cc) a[4 * b + 3] = fmaf(-a[cc], l.w, a[4 * b + 3]);
        }
      }
    }
    __syncthreads();
    const bool below = warp > p && row_ok;
    if (below) {
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) r = fmaf(-a[cc], sh.alpha[cc], r);
    }
    const int jt = j0 + 32;
    if (jt < np) {
      // the panel's rows below the block as TF32 parts (zeros elsewhere),
      // K-major 128-byte rows, 16-byte chunk q of row i at chunk q ^ (i & 7)
      const int ro = tid * 128;
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        float hv[4], lv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float x = below ? a[4 * c4 + e] : 0.0f;
          hv[e] = tc::to_tf32(x);
          lv[e] = tc::to_tf32(x - hv[e]);
        }
        const int pc = ro + (c4 ^ (tid & 7)) * 16;
        *reinterpret_cast<float4*>(phi + pc) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4*>(plo + pc) = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t ah = tc::smem_u32(phi), al = tc::smem_u32(plo);
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
          // rows of half hh are 128 hh .. 128 hh + 127; of their trailing
          // columns only those up to the half's last row are ever read
          const int cend = min(np, 128 * (hh + 1));
          const int N = cend - jt;
          if (128 * hh >= np || N <= 0) continue;
          const uint32_t idesc = tc::idesc_tf32_f32(128, N, true);  // D += (-A) B^T
          const uint32_t dcol = sh.tmem + (uint32_t)(hh * 256 + jt);
#pragma unroll
          for (int part = 0; part < 3; ++part) {
            const uint32_t A = (part == 2 ? al : ah) + (uint32_t)(hh * 128 * 128);
            const uint32_t B = (part == 1 ? al : ah) + (uint32_t)(jt * 128);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_tf32(dcol, tc::desc_kmajor_sw128(A + kk * 32), tc::desc_kmajor_sw128(B + kk * 32), idesc, 1u);
          }
        }
        tc::mma_commit(&sh.bar);
      }
      waiting = true;
    }
  }
  __syncthreads();
  const double ll = -0.5 * sh.qa - sh.ldet - 0.5 * (double)n * 1.8378770664093454836;
  out = (float)ll;
  __syncthreads();
  return true;
}

__device__ void tc_setup(TcShared& sh, const float* __restrict__ t, const float* __restrict__ y, int n) {
  const int tid = threadIdx.x;
  for (int i = tid; i < kTcMaxN; i += blockDim.x) {
    sh.t[i] = i < n ? t[i] : 0.0f;
    sh.y[i] = i < n ? y[i] : 0.0f;
  }
  if (tid == 0) {
    tc::mbar_init(&sh.bar, 1);
    tc::fence_mbar_init();
    sh.phase = 0;
  }
  if (tid < 32) {
    tc::tmem_alloc(&sh.tmem, kTcCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__device__ void tc_teardown(TcShared& sh) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(sh.tmem, kTcCols);
}

__device__ uint8_t* tc_panels(uint8_t* raw) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
}

// p HRSS steps of chains blockIdx.x, blockIdx.x + gridDim.x, ... of run
// `run`, each followed by the replacement of its dead slot.
__global__ void __launch_bounds__(kTcThreads, 1) k_gp_sweep_tc(Dev D, GPArgs A, int run, int* err) {
  extern __shared__ uint8_t gp_raw[];
  __shared__ TcShared sh;
  const RunDesc& R = D.desc[run];
  RunState* S = D.st + run;
  if (S->done) return;
  const int n = R.n_data, np = (n + 31) & ~31;
  tc_setup(sh, A.t, A.y, n);
  uint8_t* phi = tc_panels(gp_raw);
  const uint32_t iter = (uint32_t)S->iter;
  const float lstar = S->logLstar;
  float a[3], b[3], Lm[3][3];
  for (int i = 0; i < 3; ++i) {
    a[i] = D.f[R.o_a + i];
    b[i] = D.f[R.o_b + i];
  }
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) Lm[r][q] = D.f[R.o_L + r * R.dpad + q];
  const float w = R.w;
  const uint32_t nz = 4u;  // 2 ceil(3/2)
  bool alive = true;
#pragma unroll 1
  for (int j = blockIdx.x; j < R.k && alive; j += gridDim.x) {
    const int parent = D.i[R.o_parent + j];
    float x[3];
    for (int i = 0; i < 3; ++i) x[i] = D.f[R.o_x + (long long)parent * R.dpad + i];
    float lx = D.f[R.o_logL + parent];
    int evals = 0, acc = 0, nul = 0, exps = 0, shr = 0, capo = 0, nanc = 0;
#pragma unroll 1
    for (int s = 0; s < R.p && alive; ++s) {
      const uint4 w0 = draw_block(R, iter, (uint32_t)j, (uint32_t)s, 0u);
      const uint4 w1 = draw_block(R, iter, (uint32_t)j, (uint32_t)s, 1u);
      float z[4];
      box_muller(w0.x, w0.y, z[0], z[1]);
      box_muller(w0.z, w0.w, z[2], z[3]);
      const float zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
      float v[3];
      for (int r = 0; r < 3; ++r) v[r] = Lm[r][0] * z[0] + Lm[r][1] * z[1] + Lm[r][2] * z[2];
      const float inrm = (R.dir_norm == 0) ? rsqrtf(zz) : rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int r = 0; r < 3; ++r) v[r] *= inrm;
      uint32_t cblk = 1u;
      uint4 cw = w1;
      auto word = [&](uint32_t wi) {
        if ((wi >> 2) != cblk) {
          cblk = wi >> 2;
          cw = draw_block(R, iter, (uint32_t)j, (uint32_t)s, cblk);
        }
        return pick(cw, wi & 3u);
      };
      // one slice test; false with alive cleared if the tensor core stalled
      auto in_slice = [&](float t, float& ll) {
        float y[3];
        bool in = true;
        for (int r = 0; r < 3; ++r) {
          y[r] = fmaf(t, v[r], x[r]);
          if (!(y[r] >= a[r] && y[r] <= b[r])) in = false;
        }
        ++evals;
        if (!in) return false;
        if (!gp_loglik_tc(sh, phi, n, np, y, ll, err)) {
          alive = false;
          return false;
        }
        if (isnan(ll) || ll == -INFINITY) {  // FP32 breakdown of K (or NaN): outside every slice
          ++nanc;
          ll = -INFINITY;
        }
        return ll > lstar;
      };
      const float U = u24(word(nz));
      float tl = -w * U, tr = tl + w, lly = 0.0f;
      // stepping out to the left (stage 0), to the right (stage 1), then
      // shrinkage (stage 2), through one evaluation site so that the
      // factorisation is inlined once
      bool ok = false;
      int stage = 0, q = 0;
#pragma unroll 1
      while (alive) {
        float t;
        if (stage < 2) {
          if (q >= kStepOutCap) {
            ++capo;
            ++stage;
            q = 0;
            continue;
          }
          t = stage == 0 ? tl : tr;
        } else {
          if (q >= kShrinkCap) break;
          t = fmaf(u24(word(nz + 3u + (uint32_t)q)), tr - tl, tl);
          ++shr;
        }
        const bool in = in_slice(t, lly);
        if (!alive) break;
        ++q;
        if (stage < 2) {
          if (!in) {
            ++stage;
            q = 0;
            continue;
          }
          if (stage == 0) tl -= w;
          else tr += w;
          ++exps;
        } else if (in) {
          for (int e = 0; e < 3; ++e) x[e] = fmaf(t, v[e], x[e]);
          lx = lly;
          ok = true;
          break;
        } else if (t < 0.0f) {
          tl = t;
        } else {
          tr = t;
        }
      }
      if (ok) ++acc;
      else ++nul;
    }
    if (!alive) break;
    const int slot = D.i[R.o_dead + j];
    if (threadIdx.x < R.dpad)
      D.f[R.o_x + (long long)slot * R.dpad + threadIdx.x] = (threadIdx.x < 3) ? x[threadIdx.x] : 0.0f;
    if (threadIdx.x == 0) {
      D.f[R.o_logL + slot] = lx;
      D.f[R.o_birth + slot] = lstar;
      int* st = D.i + R.o_stats;
      st[j] = evals;
      st[R.k + j] = acc;
      st[2 * R.k + j] = nul;
      st[3 * R.k + j] = exps;
      st[4 * R.k + j] = shr;
      st[5 * R.k + j] = capo;
      atomicAdd(reinterpret_cast<unsigned long long*>(&S->evals), (unsigned long long)evals);
      if (nul) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nulls), (unsigned long long)nul);
      if (capo) atomicAdd(reinterpret_cast<unsigned long long*>(&S->cap_out), (unsigned long long)capo);
      if (nanc) atomicAdd(reinterpret_cast<unsigned long long*>(&S->nan_evals), (unsigned long long)nanc);
    }
  }
  tc_teardown(sh);
}

// logL of m parameter points theta [m][3] (the factorisation alone)
__global__ void __launch_bounds__(kTcThreads, 1) k_gp_loglik_tc(const float* __restrict__ t, const float* __restrict__ y,
                                                                 int n, const float* __restrict__ theta, int m,
                                                                 float* __restrict__ out, int* err) {
  extern __shared__ uint8_t gp_raw[];
  __shared__ TcShared sh;
  const int np = (n + 31) & ~31;
  tc_setup(sh, t, y, n);
  uint8_t* phi = tc_panels(gp_raw);
#pragma unroll 1
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    const float th[3] = {theta[3 * i], theta[3 * i + 1], theta[3 * i + 2]};
    float ll = 0.0f;
    if (!gp_loglik_tc(sh, phi, n, np, th, ll, err)) break;
    if (threadIdx.x == 0) out[i] = ll;
  }
  tc_teardown(sh);
}

}  // namespace

cudaError_t setup_gp_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_gp_sweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcDynSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gp_loglik_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcDynSmem);
}

cudaError_t launch_gp_sweep_tc(const Dev& D, const GPArgs& A, int run, int k, int n, int num_sms, int* err,
                               cudaStream_t s) {
  if (n < 1 || n > kTcMaxN) return cudaErrorInvalidValue;
  const int grid = std::max(1, std::min(k, num_sms));
  k_gp_sweep_tc<<<grid, kTcThreads, kTcDynSmem, s>>>(D, A, run, err);
  return cudaGetLastError();
}

cudaError_t launch_gp_loglik_tc(const float* t, const float* y, int n, const float* theta, int m, float* out,
                                int num_sms, int* err, cudaStream_t s) {
  if (n < 1 || n > kTcMaxN || m < 1) return cudaErrorInvalidValue;
  const int grid = std::max(1, std::min(m, num_sms));
  k_gp_loglik_tc<<<grid, kTcThreads, kTcDynSmem, s>>>(t, y, n, theta, m, out, err);
  return cudaGetLastError();
}

}  // namespace nss
