// nss_gp.cu -- Gaussian-process hyperparameter likelihood inside the HRSS
// sweep (the GP workloads of Sec. 4.3; the sweep of Sec. 3.2 / App. B.4),
// for sm_103a.
//
// theta = (ln l, ln a, ln s); for data (t_i, y_i), i < n,
//   K_ij = a^2 exp(-(t_i - t_j)^2 / (2 l^2)) + s^2 [i == j],
//   log p(y | theta) = -1/2 y^T K^-1 y - sum_i ln L_ii - n/2 ln 2 pi,  K = L L^T.
// Here: the SIMT evaluation used for the initial live set and the noise-scale
// gradient, one block of 1024 threads per parameter point (the sweep's
// evaluations use the tensor-core factorisation of nss_gp_tc.cu).  An
// evaluation fills the bordered matrix [[K, .], [y^T, .]]
// (n + 1 rows, packed lower triangle in shared memory, FP32) and factors it
// by right-looking column steps; the last row then holds alpha = L^-1 y, so
// y^T K^-1 y = |alpha|^2.  ln det and |alpha|^2 are accumulated in FP64.  A
// non-positive pivot (FP32 breakdown of an ill-conditioned K) makes the
// candidate's logL = -inf; it is counted with the NaN evaluations.
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {

constexpr int kGPThreads = 1024;
constexpr int kGPMaxN = 256;
constexpr int kGPPanel = 8;  // columns per factorisation panel

__device__ __forceinline__ int pidx(int i, int j) { return (i * (i + 1)) / 2 + j; }

struct GPShared {
  float inv;
  int ok;
  double red[32];
};

// logL of theta for the run's data; every thread of the block calls it and
// gets the same value.  P: packed (n+1) x (n+1) lower triangle.
__device__ float gp_loglik(const float* __restrict__ tt, const float* __restrict__ yy, int n, const float th[3],
                           float* P, GPShared& sh) {
  const int T = blockDim.x, tid = threadIdx.x;
  const float ell = expf(th[0]), amp = expf(th[1]), sn = expf(th[2]);
  const float a2 = amp * amp, s2 = sn * sn, c = -0.5f / (ell * ell);
  const int N = n + 1;
  // fill: warp w takes rows w, w + 32, ...; its lanes the row's entries
  {
    const int lane = tid & 31, wid = tid >> 5, nw = T >> 5;
    for (int i = wid; i < N; i += nw) {
      const int bi = (i * (i + 1)) / 2;
      const float ti = i < n ? tt[i] : 0.0f;
      for (int j = lane; j <= i; j += 32) {
        float v;
        if (i < n) {
          const float dt = ti - tt[j];
          v = a2 * expf(c * dt * dt) + (i == j ? s2 : 0.0f);
        } else {
          v = (j < n) ? yy[j] : 0.0f;
        }
        P[bi + j] = v;
      }
    }
  }
  if (tid == 0) sh.ok = 1;
  __syncthreads();
  // Right-looking factorisation in panels of kGPPanel columns, with the same
  // operations in the same order as column-by-column steps (so the same
  // bits): column j's pivot l = sqrt(A_jj), the entries below it scaled by
  // 1/l, and every later entry A_ik -= L_ij L_kj applied in increasing j.
  // Per panel: warp 0 factors the diagonal block; each row below solves its
  // panel entries (its updates from the panel's earlier columns, then the
  // scale); the trailing entries take the panel's columns in order.  Three
  // block barriers per panel instead of three per column.
  // L_i,j0.. of the rows below the block; row stride kGPPanel + 4 floats so
  // that a quarter-warp's 16-byte loads of 8 different rows hit distinct banks
  constexpr int kPS = kGPPanel + 4;
  __shared__ __align__(16) float panel[(kGPMaxN + 1) * kPS];
  __shared__ float pinv[kGPPanel];
  double ldet = 0.0;
  for (int j0 = 0; j0 < n; j0 += kGPPanel) {
    const int jb = min(kGPPanel, n - j0);
    if (tid < 32) {
      // the diagonal block in registers: lane r < jb holds row j0 + r;
      // column c's entries are broadcast by shuffles
      const int lane = tid;
      float a[kGPPanel];
#pragma unroll
      for (int q = 0; q < kGPPanel; ++q) a[q] = (lane < jb && q <= lane) ? P[pidx(j0 + lane, j0 + q)] : 0.0f;
#pragma unroll
      for (int c = 0; c < kGPPanel; ++c) {
        if (c < jb) {
          const float d = __shfl_sync(0xffffffffu, a[c], c);
          const bool good = d > 0.0f && isfinite(d);
          const float l = sqrtf(good ? d : 1.0f);
          const float inv = 1.0f / l;
          if (lane == 0) {
            pinv[c] = inv;
            if (!good) sh.ok = 0;
            ldet += (double)logf(l);
          }
          if (!good) break;  // the pivot is the same in every lane
          if (lane == c) a[c] = l;
          else if (lane > c && lane < jb) a[c] *= inv;
#pragma unroll
          for (int q = c + 1; q < kGPPanel; ++q) {
            const float lqc = __shfl_sync(0xffffffffu, a[c], q);
            if (q <= lane && lane < jb) a[q] = fmaf(-a[c], lqc, a[q]);
          }
        }
      }
      if (lane < jb) {
#pragma unroll
        for (int q = 0; q < kGPPanel; ++q)
          if (q <= lane) P[pidx(j0 + lane, j0 + q)] = a[q];
      }
      __syncwarp();
    }
    __syncthreads();
    if (!sh.ok) break;
    // rows below the block: their panel entries
    const int r0 = j0 + jb;
    for (int i = r0 + tid; i < N; i += T) {
      const int bi = pidx(i, j0);
      float li[kGPPanel];
#pragma unroll
      for (int c = 0; c < kGPPanel; ++c) {
        if (c < jb) {
          float a = P[bi + c];
#pragma unroll
          for (int q = 0; q < c; ++q) a = fmaf(-li[q], P[pidx(j0 + c, j0 + q)], a);
          a *= pinv[c];
          li[c] = a;
          P[bi + c] = a;
        } else {
          li[c] = 0.0f;
        }
      }
      float4* pr = reinterpret_cast<float4*>(panel + (size_t)i * kPS);
#pragma unroll
      for (int c4 = 0; c4 < kGPPanel / 4; ++c4)
        pr[c4] = make_float4(li[4 * c4], li[4 * c4 + 1], li[4 * c4 + 2], li[4 * c4 + 3]);
    }
    __syncthreads();
    // trailing entries: warp w takes rows r0 + w, r0 + w + 32, ...; lanes
    // the columns k in [r0, min(i, n - 1)]
    {
      const int lane = tid & 31, wid = tid >> 5, nw = T >> 5;
      for (int i = r0 + wid; i < N; i += nw) {
        const float4* pi4 = reinterpret_cast<const float4*>(panel + (size_t)i * kPS);
        float li[kGPPanel];
#pragma unroll
        for (int c4 = 0; c4 < kGPPanel / 4; ++c4) {
          const float4 t4 = pi4[c4];
          li[4 * c4] = t4.x; li[4 * c4 + 1] = t4.y; li[4 * c4 + 2] = t4.z; li[4 * c4 + 3] = t4.w;
        }
        const int kmax = min(i, n - 1), bi = (i * (i + 1)) / 2;
        for (int k = r0 + lane; k <= kmax; k += 32) {
          const float4* pk4 = reinterpret_cast<const float4*>(panel + (size_t)k * kPS);
          float lk[kGPPanel];
#pragma unroll
          for (int c4 = 0; c4 < kGPPanel / 4; ++c4) {
            const float4 t4 = pk4[c4];
            lk[4 * c4] = t4.x; lk[4 * c4 + 1] = t4.y; lk[4 * c4 + 2] = t4.z; lk[4 * c4 + 3] = t4.w;
          }
          float acc = P[bi + k];
#pragma unroll
          for (int c = 0; c < kGPPanel; ++c)
            if (c < jb) acc = fmaf(-li[c], lk[c], acc);
          P[bi + k] = acc;
        }
      }
    }
    __syncthreads();
  }
  const int ok = sh.ok;
  __syncthreads();
  if (!ok) return -INFINITY;
  // |alpha|^2 from the last row, FP64 accumulation
  double q = 0.0;
  for (int j = tid; j < n; j += T) {
    const double a = (double)P[pidx(n, j)];
    q += a * a;
  }
  q = block_sum_d(q, sh.red);
  if (tid == 0) sh.red[31] = ldet;
  __syncthreads();
  const double ld = sh.red[31];
  __syncthreads();
  const double ll = -0.5 * q - ld - 0.5 * (double)n * 1.8378770664093454836;
  return (float)ll;
}

// Initial live set: logL of every prior draw (block per slot).
__global__ void __launch_bounds__(kGPThreads) k_gp_init(Dev D, GPArgs A, int run) {
  extern __shared__ float P[];
  __shared__ GPShared sh;
  const RunDesc& R = D.desc[run];
  const int s = blockIdx.x;
  if (s >= R.m) return;
  float th[3];
  for (int i = 0; i < 3; ++i) th[i] = D.f[R.o_x + (long long)s * R.dpad + i];
  float ll = gp_loglik(A.t, A.y, R.n_data, th, P, sh);
  if (isnan(ll)) ll = -INFINITY;
  if (threadIdx.x == 0) D.f[R.o_logL + s] = ll;
}

// Fisher-identity term of a fixed noise multiplier s (K = a^2 k + (s sigma_n)^2 I)
// at s = 1 for the listed dead points: d/ds log p(y | theta) = sigma_n^2
// (|K^-1 y|^2 - tr K^-1).  One block per point: the bordered factorisation
// of gp_loglik leaves L and alpha = L^-1 y in shared memory; warp 0 solves
// L^T beta = alpha (beta = K^-1 y); every warp solves L z = e_j for columns
// j = warp, warp + 32, ... (tr K^-1 = sum_j |z_j|^2).  Sums in FP64.
__global__ void __launch_bounds__(kGPThreads) k_gp_noise_grad(Dev D, GPArgs A, int run, const int* __restrict__ idx,
                                                              int n_idx, double* __restrict__ coef) {
  extern __shared__ float P[];
  __shared__ GPShared sh;
  __shared__ double wsum[32];
  const RunDesc& R = D.desc[run];
  const int b = blockIdx.x;
  if (b >= n_idx) return;
  const long long i = idx[b];
  const int n = R.n_data;
  float th[3];
  for (int q = 0; q < 3; ++q) th[q] = D.f[R.o_dx + i * R.dpad + q];
  const float ll = gp_loglik(A.t, A.y, n, th, P, sh);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* zbuf = P + (n + 1) * (n + 2) / 2 + wid * n;   // [32][n]
  float* beta = P + (n + 1) * (n + 2) / 2 + 32 * n;    // [n]
  if (!(ll > -INFINITY)) {
    if (threadIdx.x == 0) coef[i] = 0.0;
    return;
  }
  double part = 0.0;  // lane 0 of each warp: its columns' sum of squares (warp 0 also |beta|^2)
  if (wid == 0) {
    for (int r = n - 1; r >= 0; --r) {
      float acc = 0.0f;
      for (int k = r + 1 + lane; k < n; k += 32) acc = fmaf(P[pidx(k, r)], beta[k], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) {
        const float br = (P[pidx(n, r)] - acc) / P[pidx(r, r)];
        beta[r] = br;
        part += (double)br * (double)br;
      }
      __syncwarp();
    }
  }
  for (int j = wid; j < n; j += 32) {
    for (int r = j; r < n; ++r) {
      float acc = 0.0f;
      for (int k = j + lane; k < r; k += 32) acc = fmaf(P[pidx(r, k)], zbuf[k], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) {
        const float zr = ((r == j ? 1.0f : 0.0f) - acc) / P[pidx(r, r)];
        zbuf[r] = zr;
        part -= (double)zr * (double)zr;
      }
      __syncwarp();
    }
  }
  if (lane == 0) wsum[wid] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += wsum[q];
    const double s2n = exp(2.0 * (double)th[2]);
    coef[i] = exp(D.dd[R.o_lw + i]) * s2n * t;
  }
}

size_t gp_smem_bytes(int n) { return sizeof(float) * (size_t)((n + 1) * (n + 2) / 2); }
size_t gp_grad_smem_bytes(int n) { return gp_smem_bytes(n) + sizeof(float) * (size_t)(33 * n); }

cudaError_t setup_gp_attributes() {
  const int bytes = (int)gp_smem_bytes(kGPMaxN);
  cudaError_t e = cudaFuncSetAttribute(k_gp_init, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gp_noise_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gp_grad_smem_bytes(kGPMaxN));
}

cudaError_t launch_gp_noise_grad(const Dev& D, const GPArgs& A, int run, const int* idx, int n_idx, int n,
                                 double* coef, cudaStream_t s) {
  if (n_idx <= 0) return cudaSuccess;
  k_gp_noise_grad<<<n_idx, kGPThreads, gp_grad_smem_bytes(n), s>>>(D, A, run, idx, n_idx, coef);
  return cudaGetLastError();
}

cudaError_t launch_gp_init(const Dev& D, const GPArgs& A, int run, int m, int n, cudaStream_t s) {
  k_gp_init<<<m, kGPThreads, gp_smem_bytes(n), s>>>(D, A, run);
  return cudaGetLastError();
}


}  // namespace nss
