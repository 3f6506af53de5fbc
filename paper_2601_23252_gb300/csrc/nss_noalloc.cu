// nss_noalloc.cu -- the post-hoc volume simulation with fixed, preallocated
// scratch, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// evidence of a finished run: a service whose framework allocator already
// owns (and caches) the device memory, or latency-bound code that has a
// no-allocation rule after start-up because cudaMalloc/cudaFree synchronise
// the device and can stall every stream.  nss_volume_sim_static gives them
// the same simulation as nss_run/nss_finalise, on device buffers they pass
// in, with its per-tile partial sums kept in one file-scope __device__ array
// instead of memory allocated per call.
//
// That array is shared by every call in the process and keeps the previous
// call's contents; each call writes every entry it later reads, so nothing
// has to start at zero.  Two calls whose kernels overlap on the GPU (for
// example on two streams) race on it; the caller must order them.
#include <cmath>

#include "../../include/nss.h"
#include "nss_device.cuh"

namespace nss {
namespace {

constexpr int kStaticMaxSim = 128;            // trajectories R
constexpr int kStaticMaxTiles = 512;          // 512 x 1024 = 524288 dead points
constexpr int kStaticMaxDead = kStaticMaxTiles * kVolTile;
constexpr size_t kStaticSlab = (size_t)kStaticMaxSim * kStaticMaxTiles;
constexpr size_t kStaticDoubles = 4 * kStaticSlab + 8;   // tsum, toff, tmax, tacc, misc

// Held by every GPU that loads this library until the process exits (2 MiB).
static __device__ __align__(256) double g_vol_scratch[kStaticDoubles];

struct StaticVol {
  const float* logL;
  const int* nlive;
  long long n;
  int R, nt;
  uint32_t k0, k1;
  double *tsum, *toff, *tmax, *tacc, *misc;
};

__global__ void k_svol_tilesum(StaticVol V) {
  const int tile = blockIdx.x, r = threadIdx.x;
  if (r >= V.R) return;
  const long long i0 = (long long)tile * kVolTile, i1 = min(i0 + kVolTile, V.n);
  double s = 0.0;
  uint4 blk;
  long long bi = -1;
  for (long long i = i0; i < i1; ++i) s += (double)vol_term_f(V.k0, V.k1, r, i, V.nlive[i], blk, bi);
  V.tsum[(size_t)r * V.nt + tile] = s;
}

__global__ void k_svol_scan(StaticVol V) {
  const int r = threadIdx.x;
  if (r >= V.R) return;
  double acc = 0.0;
  for (int q = 0; q < V.nt; ++q) {
    const size_t o = (size_t)r * V.nt + q;
    V.toff[o] = acc;
    acc += V.tsum[o];
  }
}

// the same tile-relative scheme as k_vol_weights (nss_kernels.cu)
__global__ void k_svol_weights(StaticVol V, double* __restrict__ lw) {
  extern __shared__ float shf[];  // [blockDim][32]
  __shared__ double red[32];
  __shared__ double part_s[32 * 32];
  const int tile = blockIdx.x, r = threadIdx.x;
  const long long n = V.n;
  const long long i0 = (long long)tile * kVolTile, i1 = min(i0 + kVolTile, n);
  const bool act = r < V.R;
  float lm = -INFINITY;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) lm = fmaxf(lm, V.logL[i]);
  lm = (float)block_max_d((double)lm, red);
  const double start = act ? V.toff[(size_t)r * V.nt + tile] : 0.0;
  const double start_mean = block_sum_d(start, red) / (double)V.R;
  uint4 blk;
  long long bi = -1;
  float off = 0.0f, comp = 0.0f;
  float tcur = act ? vol_term_f(V.k0, V.k1, r, i0, V.nlive[i0], blk, bi) : 0.0f;
  double Sacc = 0.0;
  const float ln2f = 0.693147182f;
  for (long long c0 = i0; c0 < i1; c0 += 32) {
    const int cn = (int)min((long long)32, i1 - c0);
    if (act) {
      for (int q = 0; q < cn; ++q) {
        const long long i = c0 + q;
        const float tnxt = (i + 1 < n) ? vol_term_f(V.k0, V.k1, r, i + 1, V.nlive[i + 1], blk, bi) : -INFINITY;
        const float rel = off + (logf(-expm1f(tcur + tnxt)) - ln2f);
        const float li = V.logL[i];
        if (li > -INFINITY) Sacc += (double)expf((li - lm) + rel);
        shf[r * 32 + q] = rel;
        const float y = tcur - comp, tt = off + y;
        comp = (tt - off) - y;
        off = tt;
        tcur = tnxt;
      }
    }
    __syncthreads();
    {
      const int pt = threadIdx.x & 31, part = threadIdx.x >> 5, P = blockDim.x >> 5;
      double sp = 0.0;
      if (pt < cn)
        for (int q = part; q < V.R; q += P) sp += (double)shf[q * 32 + pt];
      part_s[part * 32 + pt] = sp;
      __syncthreads();
      if (threadIdx.x < cn) {
        double tot = 0.0;
        for (int q = 0; q < P; ++q) tot += part_s[q * 32 + threadIdx.x];
        lw[c0 + threadIdx.x] = (double)V.logL[c0 + threadIdx.x] + (start_mean + tot / (double)V.R);
      }
    }
    __syncthreads();
  }
  if (act) {
    V.tmax[(size_t)r * V.nt + tile] = (lm > -INFINITY && Sacc > 0.0) ? (double)lm + start : -INFINITY;
    V.tacc[(size_t)r * V.nt + tile] = Sacc;
  }
}

__global__ void k_svol_final(StaticVol V, const double* __restrict__ lw, double* __restrict__ stats) {
  __shared__ double red[32];
  __shared__ double lz[kStaticMaxSim];
  for (int r = threadIdx.x; r < V.R; r += blockDim.x) {
    double M = -INFINITY;
    for (int q = 0; q < V.nt; ++q) M = fmax(M, V.tmax[(size_t)r * V.nt + q]);
    double s = 0.0;
    for (int q = 0; q < V.nt; ++q) {
      const size_t o = (size_t)r * V.nt + q;
      if (V.tmax[o] > -INFINITY) s += V.tacc[o] * exp(V.tmax[o] - M);
    }
    lz[r] = M + log(s);
  }
  __syncthreads();
  double mean = 0.0;
  for (int r = threadIdx.x; r < V.R; r += blockDim.x) mean += lz[r];
  mean = block_sum_d(mean, red) / V.R;
  double var = 0.0;
  for (int r = threadIdx.x; r < V.R; r += blockDim.x) var += (lz[r] - mean) * (lz[r] - mean);
  var = block_sum_d(var, red) / (V.R > 1 ? V.R - 1 : 1);
  double mx = -INFINITY;
  for (long long i = threadIdx.x; i < V.n; i += blockDim.x) mx = fmax(mx, lw[i]);
  mx = block_max_d(mx, red);
  double s = 0.0;
  for (long long i = threadIdx.x; i < V.n; i += blockDim.x) s += (double)expf((float)(lw[i] - mx));
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    stats[0] = mean;
    stats[1] = sqrt(var);
    V.misc[0] = mx + log(s);
  }
}

__global__ void k_svol_norm(StaticVol V, double* __restrict__ lw) {
  const double c = V.misc[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V.n; i += (long long)gridDim.x * blockDim.x)
    lw[i] -= c;
}

// Device address of the scratch array for the current device, looked up on
// every call (cheap), so a device context that was reset or re-created since
// an earlier call never gets a stale address.  The first lookup on a device
// loads the array's module there, so make the first call on each device
// before any stream capture.
cudaError_t scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_vol_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace nss

extern "C" nss_status nss_volume_sim_static(const float* logL, const int* nlive, long long n, int n_sim,
                                            uint64_t seed, uint32_t run_id, double* log_w, double* logZ_stats,
                                            void* cuda_stream) {
  using namespace nss;
  if (!logL || !nlive || !log_w || !logZ_stats) return NSS_ERR_ARG;
  if (n < 1 || n > kStaticMaxDead) return NSS_ERR_ARG;
  if (n_sim < 2 || n_sim > kStaticMaxSim) return NSS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return NSS_ERR_CUDA;
  StaticVol V;
  V.logL = logL;
  V.nlive = nlive;
  V.n = n;
  V.R = n_sim;
  V.nt = (int)((n + kVolTile - 1) / kVolTile);
  V.k0 = (uint32_t)seed;
  V.k1 = (uint32_t)(seed >> 32) ^ run_id;
  V.tsum = scratch;
  V.toff = scratch + kStaticSlab;
  V.tmax = scratch + 2 * kStaticSlab;
  V.tacc = scratch + 3 * kStaticSlab;
  V.misc = scratch + 4 * kStaticSlab;
  const int bt = (n_sim + 31) / 32 * 32;
  k_svol_tilesum<<<V.nt, bt, 0, s>>>(V);
  k_svol_scan<<<1, bt, 0, s>>>(V);
  k_svol_weights<<<V.nt, bt, (size_t)bt * 32 * sizeof(float), s>>>(V, log_w);
  k_svol_final<<<1, 256, 0, s>>>(V, log_w, logZ_stats);
  k_svol_norm<<<64, 256, 0, s>>>(V, log_w);
  e = cudaGetLastError();
  return e == cudaSuccess ? NSS_OK : NSS_ERR_CUDA;
}
