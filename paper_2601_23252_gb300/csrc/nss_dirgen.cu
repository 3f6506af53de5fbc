// nss_dirgen.cu -- the directions of every HRSS step of an outer iteration,
// drawn ahead of the sweep (Sec. 3.2, direction metric), for sm_103a.
//
// A direction depends on the run's metric factor L and on its own Philox
// counter (iteration, chain, step, .), never on the chain's position, so all
// k x p of them are independent work.  One thread makes one direction:
//   z_i ~ N(0, 1) from Box-Muller pair i/2 of words [0, 2 ceil(d/2)),
//   d~ = L z (L lower triangular), v = d~ / |z| (unit Mahalanobis length)
//   or d~ / |d~| (unit Euclidean length),
// and writes v to V[chain][step][0, dpad), with the step's first scalar
// words (step_words) beside it.  The 32 threads of a warp are 32
// chains of one run at one step, so every read of L (staged in shared memory
// per block) is a broadcast.  Rows of d~ are formed from the last to the first so that d~_r
// can overwrite z_r (row r reads z_c for c <= r only): z and d~ share one
// array, in registers for d <= 32 and in shared memory above.
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {
namespace {

constexpr int kDirThreads = 128;
constexpr int kDirStepsPerBlock = 8;  // steps of one item per block, 2 per warp

// Philox block of counter (c0, c1, c2, blk) under the run's key (k0, k1),
// the key held in registers by the caller
__device__ __forceinline__ uint4 philox4x32_10_at(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t blk) {
  return philox4x32_10(make_uint4(c0, c1, c2, blk), k0, k1);
}

// Words nz .. nz + 11 of step s's counter stream (nz = 2 ceil(d/2)): the
// bracket offset U, the prior slice height, the reserved word and the first
// nine shrinkage proposals, which the sweep reads instead of drawing them.
__device__ __forceinline__ void step_words(const RunDesc& R, uint32_t iter, int j, int s, int* __restrict__ wout) {
  const uint32_t nz = 2u * (uint32_t)((R.d + 1) >> 1);
  const int b0 = (int)(nz >> 2), off = (int)(nz & 3u);  // off is 0 or 2 (nz is even)
  int* o = wout + ((long long)j * R.p + s) * kStepWords;
  const uint32_t k0 = R.key0, k1 = R.key1;
  // one Philox block per pass (a rolled loop keeps the kernel's code small)
#pragma unroll 1
  for (int q = 0; q < 3 + (off != 0); ++q) {
    const uint4 blk = philox4x32_10_at(k0, k1, iter, (uint32_t)j, (uint32_t)s, (uint32_t)(b0 + q));
    const uint32_t w[4] = {blk.x, blk.y, blk.z, blk.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = 4 * q + e - off;
      if (idx >= 0 && idx < kStepWords) o[idx] = (int)w[e];
    }
  }
}

// floats per thread of the normals' staging rows: d <= 32 stages float4
// rows (stride DMAX + 4: a quarter-warp's 16-byte accesses hit distinct
// banks), d > 32 keeps z and d~ there (odd stride)
template <int DMAX>
__host__ __device__ constexpr int dirgen_zrow() {
  return DMAX > 32 ? DMAX + 1 : DMAX + 4;
}

template <int DMAX>
__device__ __forceinline__ void one_direction(const RunDesc& R, const float* __restrict__ Ls, float* zsh,
                                              uint32_t iter, int j, int s, float* __restrict__ vout) {
  constexpr bool kShared = DMAX > 32;
  constexpr int kReg = kShared ? 1 : DMAX;
  const int d = R.d, ld = R.dpad;
  const uint32_t k0 = R.key0, k1 = R.key1;
  float4* out = reinterpret_cast<float4*>(vout + ((long long)j * R.p + s) * ld);
  float zz = 0.0f, dd = 0.0f;
  if constexpr (!kShared) {
    // the normals, one Philox block (two Box-Muller pairs) per pass of a
    // rolled loop through this thread's row of shared memory, then into
    // registers
    float4* zs4 = reinterpret_cast<float4*>(zsh);
#pragma unroll 1
    for (int q = 0; 4 * q < d; ++q) {
      float a0, a1, a2, a3;
      const uint4 w = philox4x32_10_at(k0, k1, iter, (uint32_t)j, (uint32_t)s, (uint32_t)q);
      box_muller_dir(w.x, w.y, a0, a1);
      box_muller_dir(w.z, w.w, a2, a3);
      zs4[q] = make_float4(a0, a1, a2, a3);
    }
    float z[kReg];
#pragma unroll
    for (int q = 0; q < kReg / 4; ++q) {
      const float4 t = (4 * q < d) ? zs4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      z[4 * q] = t.x; z[4 * q + 1] = t.y; z[4 * q + 2] = t.z; z[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int i = 0; i < kReg; ++i) {
      if (i >= d) z[i] = 0.0f;
      zz = fmaf(z[i], z[i], zz);
    }
    const float4* L4 = reinterpret_cast<const float4*>(Ls);
    const int ld4 = ld >> 2;
#pragma unroll
    for (int r = kReg - 1; r >= 0; --r) {
      if (r < d) {
        const float4* row = L4 + r * ld4;
        float acc = 0.0f;
#pragma unroll
        for (int b = 0; b < r / 4; ++b) {
          const float4 l = row[b];
          acc = fmaf(l.x, z[4 * b], fmaf(l.y, z[4 * b + 1], fmaf(l.z, z[4 * b + 2], fmaf(l.w, z[4 * b + 3], acc))));
        }
        // the diagonal block: columns 4(r/4) .. r only (later ones already hold d~)
        const float4 l = row[r / 4];
        const int b = r / 4, e = r % 4;
        float t = 0.0f;
        if (e >= 3) t = fmaf(l.w, z[4 * b + 3], t);
        if (e >= 2) t = fmaf(l.z, z[4 * b + 2], t);
        if (e >= 1) t = fmaf(l.y, z[4 * b + 1], t);
        t = fmaf(l.x, z[4 * b], t);
        z[r] = acc + t;
      }
    }
#pragma unroll
    for (int i = 0; i < kReg; ++i) dd = fmaf(z[i], z[i], dd);
    const float inrm = R.kernel == kKernelRw ? 1.0f : rsqrtf(R.dir_norm == 0 ? zz : dd);  // RW: L z itself
#pragma unroll
    for (int b = 0; b < kReg / 4; ++b)
      if (4 * b < ld) out[b] = make_float4(z[4 * b] * inrm, z[4 * b + 1] * inrm, z[4 * b + 2] * inrm, z[4 * b + 3] * inrm);
  } else {
    float* z = zsh;
    for (int q = 0; 4 * q < ld; ++q) {
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
      if (4 * q < d) {
        const uint4 w = philox4x32_10_at(k0, k1, iter, (uint32_t)j, (uint32_t)s, (uint32_t)q);
        box_muller_dir(w.x, w.y, a0, a1);
        box_muller_dir(w.z, w.w, a2, a3);
      }
      const float t4[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float zi = (4 * q + e < d) ? t4[e] : 0.0f;
        z[4 * q + e] = zi;
        zz = fmaf(zi, zi, zz);
      }
    }
    for (int r = d - 1; r >= 0; --r) {
      const float4* row = reinterpret_cast<const float4*>(Ls + r * ld);
      float acc = 0.0f;
      const int nb = r / 4;
      for (int b = 0; b < nb; ++b) {
        const float4 l = row[b];
        acc = fmaf(l.x, z[4 * b], fmaf(l.y, z[4 * b + 1], fmaf(l.z, z[4 * b + 2], fmaf(l.w, z[4 * b + 3], acc))));
      }
      const float* lr = Ls + r * ld;
      float t = 0.0f;
      for (int c = r; c >= 4 * nb; --c) t = fmaf(lr[c], z[c], t);
      z[r] = acc + t;
      dd = fmaf(z[r], z[r], dd);
    }
    const float inrm = R.kernel == kKernelRw ? 1.0f : rsqrtf(R.dir_norm == 0 ? zz : dd);  // RW: L z itself
    for (int b = 0; 4 * b < ld; ++b)
      out[b] = make_float4(z[4 * b] * inrm, z[4 * b + 1] * inrm, z[4 * b + 2] * inrm, z[4 * b + 3] * inrm);
  }
}

// block (item, step chunk): the run's factor L is staged in shared memory
// once; warp w makes the directions of steps chunk*8 + w and + 4 for the
// item's 32 chains (one per lane).  Short blocks keep the launch's last
// partial wave short (measured: 16 steps per block left a long tail).
template <int DMAX>
__global__ void __launch_bounds__(kDirThreads) k_dirgen(Dev D, const WorkItem* __restrict__ items, int n_items) {
  extern __shared__ __align__(16) float dsm[];  // L [ld][ld], then z [kDirThreads][zrow]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const WorkItem wi = items[it];
  const RunDesc& R = D.desc[wi.run];
  const RunState& S = D.st[wi.run];
  const int s0 = blockIdx.y * kDirStepsPerBlock;
  if (S.done || s0 >= R.p) return;
  const int ld = R.dpad;
  const float4* Lg = reinterpret_cast<const float4*>(D.f + R.o_L);
  float4* L4 = reinterpret_cast<float4*>(dsm);
  for (int t = threadIdx.x; t < (ld * ld) >> 2; t += kDirThreads) L4[t] = Lg[t];
  __syncthreads();
  const int j = wi.c0 + lane;
  if (j >= wi.c1) return;
  const uint32_t iter = (uint32_t)S.iter;
  float* zsh = dsm + DMAX * DMAX + threadIdx.x * dirgen_zrow<DMAX>();
  const int s1 = min(R.p, s0 + kDirStepsPerBlock);
  for (int s = s0 + wid; s < s1; s += kDirThreads / 32) {
    one_direction<DMAX>(R, dsm, zsh, iter, j, s, D.f + R.o_V);
    step_words(R, iter, j, s, D.i + R.o_wd);
  }
}

template <int DMAX>
size_t dirgen_smem() {
  return sizeof(float) * ((size_t)DMAX * DMAX + (size_t)kDirThreads * dirgen_zrow<DMAX>());
}

}  // namespace

int dirgen_class(int d) {
  if (d <= 8) return 8;
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  if (d <= 64) return 64;
  return 128;
}

cudaError_t setup_dirgen_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_dirgen<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dirgen_smem<64>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dirgen<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dirgen_smem<128>());
}

cudaError_t launch_dirgen(int dclass, const Dev& D, const WorkItem* items, int n, int max_p, cudaStream_t s) {
  const dim3 grid(n, (max_p + kDirStepsPerBlock - 1) / kDirStepsPerBlock);
  switch (dclass) {
    case 8: k_dirgen<8><<<grid, kDirThreads, dirgen_smem<8>(), s>>>(D, items, n); break;
    case 16: k_dirgen<16><<<grid, kDirThreads, dirgen_smem<16>(), s>>>(D, items, n); break;
    case 32: k_dirgen<32><<<grid, kDirThreads, dirgen_smem<32>(), s>>>(D, items, n); break;
    case 64: k_dirgen<64><<<grid, kDirThreads, dirgen_smem<64>(), s>>>(D, items, n); break;
    case 128: k_dirgen<128><<<grid, kDirThreads, dirgen_smem<128>(), s>>>(D, items, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace nss
