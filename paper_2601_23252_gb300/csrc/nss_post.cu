// nss_post.cu -- posterior expectations over a finished run's dead points:
// the posterior mean and the Fisher-identity gradients of log Z, for sm_103a.
//
// For Z(theta) = int L(x; theta) Pi(x; theta) dx,
//   d log Z / d theta = E_post[ d/dtheta log L(x; theta) + d/dtheta log Pi(x; theta) ],
// and the posterior expectation of any f is estimated with the dead points'
// normalised weights (App. D.2): sum_i w_i f(x_i), w_i = exp(log_w_i).
// Pass 1 forms one FP64 coefficient per dead point (and component); pass 2
// sums them in a fixed order, so the result does not depend on scheduling.
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {
namespace {

constexpr int kPostMaxComp = 8;

// one thread per dead point: coef[i] (scalar kinds) or coef[i*K + c] (means)
__global__ void k_post_point(PostArgs A, double* __restrict__ coef) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const double w = exp(A.lw[i]);
  const float* x = A.x + i * A.ld;
  if (A.kind == kPostMean) {
    coef[i] = w;
    return;
  }
  if (A.kind == kPostPriorLogPrec) {
    double s = 0.0;
    for (int a = 0; a < A.d; ++a) {
      const double u = ((double)x[a] - (double)A.pa[a]) / (double)A.pb[a];
      s += u * u;
    }
    coef[i] = w * (0.5 * A.d - 0.5 * s);
    return;
  }
  // Gaussian / equal-weight mixture: squared distances and responsibilities
  double q[kPostMaxComp];
  double qmin = INFINITY;
  for (int c = 0; c < A.K; ++c) {
    const float* mu = A.mu + (long long)c * A.ld;
    double s = 0.0;
    for (int a = 0; a < A.d; ++a) {
      const double e = (double)x[a] - (double)mu[a];
      s += e * e;
    }
    q[c] = s;
    qmin = fmin(qmin, s);
  }
  const double s2 = A.sigma * A.sigma;
  double r[kPostMaxComp], rs = 0.0;
  for (int c = 0; c < A.K; ++c) {
    r[c] = exp(-(q[c] - qmin) / (2.0 * s2));
    rs += r[c];
  }
  if (A.kind == kPostLikSigma) {
    double e = 0.0;
    for (int c = 0; c < A.K; ++c) e += r[c] * q[c];
    e /= rs;
    coef[i] = w * (e / (s2 * A.sigma) - (double)A.d / A.sigma);
  } else {  // means: r_c / sigma^2, times (x - mu_c) in pass 2
    for (int c = 0; c < A.K; ++c) coef[i * A.K + c] = w * (r[c] / rs) / s2;
  }
}

// pass 2, scalar kinds: one block, thread t sums entries t, t + T, ... then a
// fixed-order block reduction
__global__ void k_post_sum(const double* __restrict__ coef, long long n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += coef[i];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) out[0] = s;
}

// pass 2, vector kinds: block c; thread (part, a) sums dimension a over dead
// points part, part + P, ...; parts reduced in order in shared memory
__global__ void k_post_vec(PostArgs A, const double* __restrict__ coef, double* __restrict__ out) {
  extern __shared__ double acc[];  // [blockDim]
  const int c = blockIdx.x;
  const int a = threadIdx.x % A.ld, part = threadIdx.x / A.ld;
  const int P = blockDim.x / A.ld;
  const bool mean = A.kind == kPostMean;
  double s = 0.0;
  if (part < P && a < A.d) {
    const double mu = mean ? 0.0 : (double)A.mu[(long long)c * A.ld + a];
    for (long long i = part; i < A.n; i += P) {
      const double cf = mean ? coef[i] : coef[i * A.K + c];
      s += cf * ((double)A.x[i * A.ld + a] - mu);
    }
  }
  acc[threadIdx.x] = s;
  __syncthreads();
  if (part == 0 && a < A.d) {
    double t = 0.0;
    for (int q = 0; q < P; ++q) t += acc[q * A.ld + a];
    out[(long long)c * A.d + a] = t;
  }
}

__global__ void k_scale_logL(const float* __restrict__ logL, float beta, long long n, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = logL[i] > -INFINITY ? beta * logL[i] : -INFINITY;  // beta > 0; -inf and NaN keep weight 0
}

__global__ void k_sq_weights(const double* __restrict__ lw, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = exp(2.0 * lw[i]);
}

}  // namespace

cudaError_t launch_scale_logL(const float* logL, float beta, long long n, float* out, cudaStream_t s) {
  k_scale_logL<<<256, 256, 0, s>>>(logL, beta, n, out);
  return cudaGetLastError();
}

cudaError_t launch_sq_weights(const double* lw, long long n, double* out, cudaStream_t s) {
  k_sq_weights<<<256, 256, 0, s>>>(lw, n, out);
  return cudaGetLastError();
}

cudaError_t launch_post(const PostArgs& A, double* coef, double* out, cudaStream_t s) {
  if (A.n <= 0) return cudaErrorInvalidValue;
  k_post_point<<<(int)((A.n + 255) / 256), 256, 0, s>>>(A, coef);
  if (A.kind == kPostLikMu || A.kind == kPostMean) {
    const int nb = A.kind == kPostMean ? 1 : A.K;
    const int T = (256 / A.ld) * A.ld;
    k_post_vec<<<nb, T, sizeof(double) * T, s>>>(A, coef, out);
  } else {
    k_post_sum<<<1, 1024, 0, s>>>(coef, A.n, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_post_sum(const double* coef, long long n, double* out, cudaStream_t s) {
  k_post_sum<<<1, 1024, 0, s>>>(coef, n, out);
  return cudaGetLastError();
}

}  // namespace nss
