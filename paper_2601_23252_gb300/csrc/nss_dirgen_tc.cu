// nss_dirgen_tc.cu -- the whitened directions of an outer iteration's HRSS
// steps (Sec. 3.2, direction metric) with the whitening product on the
// 5th-generation tensor cores, for sm_103a.
//
// Every step of every chain of a run draws z ~ N(0, I_d) from its own Philox
// counter (iteration, chain, step, .) and needs d~ = L z with the run's
// metric factor L: over the k x p steps of the iteration that is the dense
// product Z L^T of a [k p x d] matrix of normals with the [d x d] factor.
// One block of 256 threads takes tiles of 128 steps (rows q = chain * p +
// step of the run's direction store); row r of a tile belongs to threads r
// and r + 128, each of which draws half of the row's Philox blocks:
//   - the two threads draw the row's normals (Box-Muller pairs of the row's
//     counter stream, as in the CUDA-core kernel; the row's blocks alternate
//     between them, and the step's first scalar words are split so that the
//     two threads' loads are closest) and write them to shared memory as two
//     TF32 parts hi + lo in the K-major 128-byte swizzled layout;
//   - the block stages L (rows n < N, zero above the diagonal and past d) in
//     the same layout, also split hi + lo;
//   - one thread issues tcgen05.mma kind::tf32 (M = 128, N = 32 KC, K = 8)
//     for hi hi^T + hi lo^T + lo hi^T, accumulating d~ in tensor memory in
//     FP32 (the 3xTF32 scheme: each product to about 2^-21 relative);
//   - each thread reads its half of the row's columns back (tcgen05.ld, TMEM
//     lane r), and the row is scaled to v = d~ / |z| (unit Mahalanobis
//     length) or d~ / |d~| and stored.
// KC = 1 serves d <= 32, KC = 2 serves d <= 64.  The block caches the run,
// rows and done flag of its next work items in shared memory, so items of
// finished runs cost no global load each.  The MMA wait is bounded: a wait
// that runs out sets the error flag, and the block frees its tensor memory
// and returns.
#include <algorithm>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"
#include "nss_tc.cuh"

namespace nss {
namespace {

constexpr int kDtThreads = 256;
constexpr int kDtCache = 256;      // work items cached per pass
constexpr uint32_t kDtMaxPolls = 1u << 22;
constexpr int kDtErr = 4;          // error code of a wait that ran out

template <int KC>
struct DirTc {
  static constexpr int N = 32 * KC;       // MMA N and tensor-memory columns
  static constexpr int kA = 128 * 128;    // bytes of one K-chunk (32 TF32 columns) of 128 rows
  static constexpr int kB = N * 128;      // bytes of one K-chunk of N rows
  static constexpr int kSmem = 2 * KC * kA + 2 * KC * kB + 1024;  // + alignment slack
};

__device__ __forceinline__ void split_tf32(const float4 x, float4& hi, float4& lo) {
  hi = make_float4(tc::to_tf32(x.x), tc::to_tf32(x.y), tc::to_tf32(x.z), tc::to_tf32(x.w));
  lo = make_float4(tc::to_tf32(x.x - hi.x), tc::to_tf32(x.y - hi.y), tc::to_tf32(x.z - hi.z),
                   tc::to_tf32(x.w - hi.w));
}

// byte offset of 16-byte chunk c4 (0..7) of row r in a 128-byte-row swizzled tile
__device__ __forceinline__ int sw128(int r, int c4) { return r * 128 + ((c4 ^ (r & 7)) << 4); }

// Words nz .. nz + 11 of the step's counter stream (U, slice height,
// reserved, the first nine shrinkage proposals), as the CUDA-core kernel
// writes them; this thread draws the Philox blocks q in [q0, q1) of the
// three or four that hold them.
__device__ __forceinline__ void step_words_tc(uint32_t k0, uint32_t k1, int d, int p, uint32_t iter, int j, int s,
                                              int q0, int q1, int* __restrict__ wout) {
  const uint32_t nz = 2u * (uint32_t)((d + 1) >> 1);
  const int b0 = (int)(nz >> 2), off = (int)(nz & 3u);
  int* o = wout + ((long long)j * p + s) * kStepWords;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < q0 || q >= q1 || (q == 3 && off == 0)) continue;
    const uint4 blk = philox4x32_10(make_uint4(iter, (uint32_t)j, (uint32_t)s, (uint32_t)(b0 + q)), k0, k1);
    const uint32_t w[4] = {blk.x, blk.y, blk.z, blk.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = 4 * q + e - off;
      if (idx >= 0 && idx < kStepWords) o[idx] = (int)w[e];
    }
  }
}

// items: {run, q0, q1, -} tiles of at most 128 rows of one run
template <int KC>
__global__ void __launch_bounds__(kDtThreads) k_dirgen_tc(Dev D, const WorkItem* __restrict__ items, int n_items,
                                                           int* err) {
  using T = DirTc<KC>;
  constexpr int kHalfB = 4 * KC;             // Philox blocks (4 normals each) per half row
  constexpr int kHalfC = 16 * KC;            // columns per half row
  extern __shared__ uint8_t dt_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int4 cache[kDtCache];           // run, q0, q1, done
  __shared__ float part[2][128];             // per half row: sum of z^2, then of d~^2
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dt_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Ahi = base;
  uint8_t* Alo = base + KC * T::kA;
  uint8_t* Bhi = base + 2 * KC * T::kA;
  uint8_t* Blo = Bhi + KC * T::kB;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & 127, h = tid >> 7;     // row of the tile, half of the row
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, (uint32_t)T::N);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  // warp w reads TMEM lanes 32 (w mod 4) .. + 31, its half's columns
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * kHalfC);
  uint32_t phase = 0;
  bool alive = true;
  const int G = gridDim.x;
#pragma unroll 1
  for (int first = blockIdx.x; first < n_items && alive; first += kDtCache * G) {
    {
      const int it = first + tid * G;
      int4 e = make_int4(0, 0, 0, 1);
      if (tid < kDtCache && it < n_items) {
        const WorkItem wi = items[it];
        e = make_int4(wi.run, wi.c0, wi.c1, D.st[wi.run].done);
      }
      if (tid < kDtCache) cache[tid] = e;
    }
    __syncthreads();
#pragma unroll 1
    for (int ci = 0; ci < kDtCache && alive; ++ci) {
      const int4 e = cache[ci];
      if (e.w) continue;  // a finished run, or past the list (the same for the whole block)
      // the run's fields in registers, loaded once per tile
      const RunDesc& R = D.desc[e.x];
      const int d = R.d, ld = R.dpad, p = R.p;
      const uint32_t k0 = R.key0, k1 = R.key1;
      const long long o_V = R.o_V, o_wd = R.o_wd;
      const bool unit_l = R.kernel == kKernelRw, mahal = R.dir_norm == 0;
      const uint32_t iter = (uint32_t)D.st[e.x].iter;
      // the factor L, rows n < N (zero above the diagonal and past d): this
      // thread's granules are loaded now and staged after the normals
      const float* __restrict__ Lg = D.f + R.o_L;
      constexpr int kLG = T::N * 8 * KC / kDtThreads;  // float4 granules per thread
      float4 lg[kLG];
#pragma unroll
      for (int u = 0; u < kLG; ++u) {
        const int g = tid + u * kDtThreads;
        const int n = g / (8 * KC), gc = g - n * (8 * KC), col = 32 * (gc >> 3) + 4 * (gc & 7);
        lg[u] = (n < d && col <= n) ? *reinterpret_cast<const float4*>(Lg + (long long)n * ld + col)  // ld % 4 == 0
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      // this thread's half of row r of Z: the row's Philox blocks of normals
      // alternate between the two halves (block b to half b mod 2), and the
      // three or four blocks of step words go to the halves so that their
      // loads (a normals block ~8 units, a step-word block ~5) are closest
      const int q = e.y + r;
      const bool valid = q < e.z;
      const int j = valid ? q / p : 0, s = valid ? q - j * p : 0;
      const int nbt = (d + 3) >> 2, nsw = (((d + 1) >> 1) & 1) ? 4 : 3;
      int n1 = 0, best = 1 << 30;
#pragma unroll 1
      for (int c = 0; c <= nsw; ++c) {
        const int cost = max(8 * (nbt >> 1) + 5 * c, 8 * ((nbt + 1) >> 1) + 5 * (nsw - c));
        if (cost < best) {
          best = cost;
          n1 = c;
        }
      }
      float zz = 0.0f;
#pragma unroll 4
      for (int bb = 0; bb < kHalfB; ++bb) {
        const int b = 2 * bb + h;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid && 4 * b < d) {
          const uint4 w = philox4x32_10(make_uint4(iter, (uint32_t)j, (uint32_t)s, (uint32_t)b), k0, k1);
          box_muller_dir(w.x, w.y, z.x, z.y);
          box_muller_dir(w.z, w.w, z.z, z.w);
          if (4 * b + 1 >= d) z.y = 0.f;
          if (4 * b + 2 >= d) z.z = 0.f;
          if (4 * b + 3 >= d) z.w = 0.f;
        }
        zz = fmaf(z.x, z.x, zz);
        zz = fmaf(z.y, z.y, zz);
        zz = fmaf(z.z, z.z, zz);
        zz = fmaf(z.w, z.w, zz);
        float4 hi, lo;
        split_tf32(z, hi, lo);
        const int c = b >> 3, c4 = b & 7;
        *reinterpret_cast<float4*>(Ahi + c * T::kA + sw128(r, c4)) = hi;
        *reinterpret_cast<float4*>(Alo + c * T::kA + sw128(r, c4)) = lo;
      }
      part[h][r] = zz;
#pragma unroll
      for (int u = 0; u < kLG; ++u) {
        const int g = tid + u * kDtThreads;
        const int n = g / (8 * KC), gc = g - n * (8 * KC), c = gc >> 3, c4 = gc & 7, col = 32 * c + 4 * c4;
        float4 l = lg[u];
        if (col + 1 > n) l.y = 0.f;
        if (col + 2 > n) l.z = 0.f;
        if (col + 3 > n) l.w = 0.f;
        float4 hi, lo;
        split_tf32(l, hi, lo);
        *reinterpret_cast<float4*>(Bhi + c * T::kB + sw128(n, c4)) = hi;
        *reinterpret_cast<float4*>(Blo + c * T::kB + sw128(n, c4)) = lo;
      }
      if (valid) step_words_tc(k0, k1, d, p, iter, j, s, h ? 0 : n1, h ? n1 : 4, D.i + o_wd);
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      const float zsum = part[0][r] + part[1][r];
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_tf32_f32(128, T::N, false);
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          const uint32_t ah = tc::smem_u32(Ahi + c * T::kA), al = tc::smem_u32(Alo + c * T::kA);
          const uint32_t bh = tc::smem_u32(Bhi + c * T::kB), bl = tc::smem_u32(Blo + c * T::kB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = (uint32_t)(kk * 32);
            tc::mma_tf32(tmem, tc::desc_kmajor_sw128(ah + o), tc::desc_kmajor_sw128(bh + o), idesc,
                         (c | kk) != 0 ? 1u : 0u);
            tc::mma_tf32(tmem, tc::desc_kmajor_sw128(ah + o), tc::desc_kmajor_sw128(bl + o), idesc, 1u);
            tc::mma_tf32(tmem, tc::desc_kmajor_sw128(al + o), tc::desc_kmajor_sw128(bh + o), idesc, 1u);
          }
        }
        tc::mma_commit(&bar);
      }
      // one warp polls the barrier; the others wait at the block barrier
      // without taking issue slots from the co-resident block
      bool ok = true;
      if (warp == 0) ok = tc::mbar_wait(&bar, phase & 1u, kDtMaxPolls);
      ++phase;
      if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) {
          atomicExch(err, kDtErr);
          // one more bounded wait for the products still in flight, then give up
          tc::mbar_wait(&bar, (phase - 1) & 1u, kDtMaxPolls);
        }
        alive = false;
        break;
      }
      tc::fence_after_sync();
      float v[kHalfC];
      if constexpr (KC == 1) {
        tc::tmem_ld16(trow, v);
      } else {
        tc::tmem_ld32(trow, v);
      }
      float dd = 0.0f;
#pragma unroll
      for (int i = 0; i < kHalfC; ++i) dd = fmaf(v[i], v[i], dd);
      part[h][r] = dd;  // every thread read its z sum before the MMA wait
      __syncthreads();
      if (valid) {
        const float nrm = mahal ? zsum : part[0][r] + part[1][r];
        const float inrm = unit_l ? 1.0f : rsqrtf(nrm);  // RW: L z itself
        float4* out = reinterpret_cast<float4*>(D.f + o_V + (long long)q * ld + h * kHalfC);
#pragma unroll
        for (int b = 0; b < kHalfC / 4; ++b)
          if (h * kHalfC + 4 * b < ld)
            out[b] = make_float4(v[4 * b] * inrm, v[4 * b + 1] * inrm, v[4 * b + 2] * inrm, v[4 * b + 3] * inrm);
      }
      // the next tile overwrites shared memory and tensor memory only after
      // every thread's reads of this one
      tc::fence_before_sync();
      __syncthreads();
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)T::N);
}

}  // namespace

cudaError_t setup_dirgen_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_dirgen_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, DirTc<1>::kSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dirgen_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, DirTc<2>::kSmem);
  // the whole unified L1 / shared array as shared memory: the blocks resident
  // per SM are set by their shared-memory footprint
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dirgen_tc<1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dirgen_tc<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

// Blocks resident per SM: the shared-memory footprint (dynamic + static +
// the 1 KB the driver reserves per block) against the SM's shared memory,
// and the registers of a 256-thread block against the SM's 64 K.
int dirgen_tc_blocks_per_sm(int kc) {
  int dev = 0, smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  const cudaError_t e = kc == 1 ? cudaFuncGetAttributes(&fa, k_dirgen_tc<1>) : cudaFuncGetAttributes(&fa, k_dirgen_tc<2>);
  if (e != cudaSuccess || smem <= 0) return 1;
  const int dyn = kc == 1 ? DirTc<1>::kSmem : DirTc<2>::kSmem;
  const int by_smem = smem / (dyn + (int)fa.sharedSizeBytes + 1024);
  const int by_regs = 65536 / (std::max(fa.numRegs, 1) * kDtThreads);
  return std::max(1, std::min(by_smem, by_regs));
}

cudaError_t launch_dirgen_tc(int kc, const Dev& D, const WorkItem* items, int n, int grid, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  grid = std::max(1, std::min(grid, n));
  switch (kc) {
    case 1: k_dirgen_tc<1><<<grid, kDtThreads, DirTc<1>::kSmem, s>>>(D, items, n, err); break;
    case 2: k_dirgen_tc<2><<<grid, kDtThreads, DirTc<2>::kSmem, s>>>(D, items, n, err); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace nss
