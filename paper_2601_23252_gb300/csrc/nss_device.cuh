// nss_device.cuh -- device helpers shared by the Nested Slice Sampling kernels:
// the counter-based generator, uniform and normal maps, group and block
// reductions, and sort keys.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "nss_internal.h"

namespace nss {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64-bit products with the published multipliers; the key is bumped by
// the published Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each product as one 32 x 32 -> 64-bit multiply (both halves at once)
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 draw_block(const RunDesc& R, uint32_t c0, uint32_t c1, uint32_t c2,
                                            uint32_t blk) {
  return philox4x32_10(make_uint4(c0, c1, c2, blk), R.key0, R.key1);
}

__device__ __forceinline__ uint32_t pick(const uint4& b, uint32_t lane) {
  return lane == 0 ? b.x : lane == 1 ? b.y : lane == 2 ? b.z : b.w;
}

// u = (2*(w >> 9) + 1) * 2^-24: an odd multiple of 2^-24 in (0, 1), exact in FP32.
// Formed without an integer-to-float conversion: the bits (w >> 9) as the
// mantissa of 1.m in [1, 2), minus (1 - 2^-24); the difference
// m 2^-23 + 2^-24 is exactly representable, so the subtraction is exact.
__device__ __forceinline__ float u24(uint32_t w) {
  return __uint_as_float((w >> 9) | 0x3F800000u) - 0x1.fffffep-1f;
}

// 52-bit uniform (2*x + 1) * 2^-53 from two words, exact in FP64.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const unsigned long long x = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
  return (2.0 * (double)x + 1.0) * 0x1p-53;
}

// The same uniform rounded to FP32 ((float)u53(a, b)), without FP64
// arithmetic: the 53-bit odd integer 2x + 1 converted with round-to-nearest,
// then an exact scaling by 2^-53.
__device__ __forceinline__ float u53f(uint32_t a, uint32_t b) {
  const unsigned long long x = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
  return __ull2float_rn(2ull * x + 1ull) * 0x1p-53f;
}

// Volume-simulation term of death i on trajectory r (App. D.2):
// log(u_{r,i}) / n_i in FP32, u from counter (r, i/2, TAG_VOLSIM, 0); `blk`
// caches the Philox block of the pair (i even, i odd) under key id `bi`.
__device__ __forceinline__ float vol_term_f(uint32_t k0, uint32_t k1, int r, long long i, int n, uint4& blk,
                                            long long& bi) {
  if ((i >> 1) != bi) {
    bi = i >> 1;
    blk = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)bi, kTagVolsim, 0u), k0, k1);
  }
  const float u = (i & 1) ? u53f(blk.z, blk.w) : u53f(blk.x, blk.y);
  return logf(u) / (float)n;
}

// Box-Muller: r = sqrt(-2 ln u1), angle 2 pi u2.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float r = sqrtf(-2.0f * logf(u24(a)));
  float s, c;
  sincospif(2.0f * u24(b), &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Box-Muller for the step directions: the same radius, and the angle taken
// as pi + 2 pi (u2 - 1/2), so the hardware sine and cosine see the centred
// argument in [-pi, pi] (absolute error about 2^-21 there, against the
// rounding of 2 pi (u2 - 1/2) itself, ~2^-22): cos 2 pi u2 = -cos of it,
// sin 2 pi u2 = -sin of it.
__device__ __forceinline__ void box_muller_dir(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float r = sqrtf(-2.0f * logf(u24(a)));
  float s, c;
  __sincosf(6.28318530717958648f * (u24(b) - 0.5f), &s, &c);
  z0 = -r * c;
  z1 = -r * s;
}

// ---- reductions within a chain group of G lanes (butterfly: every lane of
// the group ends with the bitwise-identical total) ----
template <int G>
__device__ __forceinline__ float gsum(float v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
  return v;
}

template <int G>
__device__ __forceinline__ float gmax(float v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
  return v;
}

// ballot of a group of G lanes, as bits 0..G-1 (bit i: group lane i)
template <int G>
__device__ __forceinline__ unsigned gballot(bool p, unsigned mask) {
  const unsigned b = __ballot_sync(mask, p) & mask;
  return G == 32 ? b : b >> (__ffs(mask) - 1);
}

// ---- block reductions (fixed order: deterministic) ----
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// scratch: >= 32 doubles of shared memory; every thread of the block calls.
__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum_d(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  const double r = scratch[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max_d(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max_d(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : -INFINITY;
  if (wid == 0) t = warp_max_d(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  const double r = scratch[0];
  __syncthreads();
  return r;
}

// exclusive prefix sum of one int per thread; returns the prefix, *total the sum
__device__ __forceinline__ int block_exscan_i(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  __syncthreads();
  if (lane == 31) scratch[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int s = (lane < nw) ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += n;
    }
    scratch[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int base = wid > 0 ? scratch[wid - 1] : 0;
  *total = scratch[nw - 1];
  __syncthreads();
  return base + inc - v;
}

// Sort key ordering (logL ascending, slot ascending); -0 is folded into +0.
__device__ __forceinline__ unsigned long long sort_key(float f, int slot) {
  f = f + 0.0f;
  uint32_t u = __float_as_uint(f);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (uint32_t)slot;
}

// Bitonic sort of n (power of two) keys in shared memory by the whole block.
__device__ __forceinline__ void bitonic_sort(unsigned long long* keys, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = keys[lo], b = keys[hi];
        if ((a > b) == up) {
          keys[lo] = b;
          keys[hi] = a;
        }
      }
    }
  }
  __syncthreads();
}

// Bitonic sort of n (power of two, n <= blockDim.x, blockDim.x a multiple of
// 32) keys in shared memory, one key per thread in a register: stages whose
// partner lies in the same warp (stride < 32) exchange by shuffles, the
// others through shared memory.  Threads i >= n sort a block of padding keys
// of their own.  Same result as bitonic_sort.
__device__ __forceinline__ void bitonic_sort_reg(unsigned long long* keys, int n) {
  const int i = threadIdx.x;
  unsigned long long a = (i < n) ? keys[i] : ~0ull;
  for (int size = 2; size <= n; size <<= 1) {
    const bool up = (i & size) == 0;
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      unsigned long long b;
      if (stride >= 32) {
        __syncthreads();
        if (i < n) keys[i] = a;
        __syncthreads();
        b = (i < n) ? keys[i ^ stride] : a;
      } else {
        b = __shfl_xor_sync(0xffffffffu, a, stride);
      }
      const bool lower = (i & stride) == 0;
      const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
      a = (lower == up) ? lo : hi;
    }
  }
  __syncthreads();
  if (i < n) keys[i] = a;
  __syncthreads();
}

__device__ __forceinline__ double logaddexp_d(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = fmax(a, b);
  return m + log1p(exp(-fabs(a - b)));
}

}  // namespace nss
