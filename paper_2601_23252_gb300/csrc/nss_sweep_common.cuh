// nss_sweep_common.cuh -- device helpers shared by the initial prior draw and
// the HRSS sweep kernels (lane slices of a point row, counter-stream words of
// one step) and the table of sweep configurations.
#pragma once
#include <cfloat>
#include <cmath>

#include "nss_device.cuh"
#include "nss_kernels.h"

namespace nss {

// ---- lane-slice loads and stores of a point row ---------------------------
// Lane gl owns entries [gl*DPL, gl*DPL + DPL) of a row of ld floats (ld a
// multiple of 4).  For DPL >= 8 the lane's range can run past ld (d = 20 with
// 8 entries per lane): each float4 is guarded, and entries past ld read as 0
// and are never written.
template <int DPL>
__device__ __forceinline__ void load_lane(const float* __restrict__ row, int gl, int ld, float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      const float4 t = (DPL == 4 || 4 * b < ld) ? reinterpret_cast<const float4*>(row)[b]
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
    }
  } else if constexpr (DPL == 2) {
    const float2 t = reinterpret_cast<const float2*>(row)[gl];
    x[0] = t.x; x[1] = t.y;
  } else {
    x[0] = row[gl];
  }
}

template <int DPL>
__device__ __forceinline__ void ldg_lane(const float* __restrict__ row, int gl, int ld, float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      const float4 t = (DPL == 4 || 4 * b < ld) ? __ldg(reinterpret_cast<const float4*>(row) + b)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
    }
  } else if constexpr (DPL == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(row) + gl);
    x[0] = t.x; x[1] = t.y;
  } else {
    x[0] = __ldg(row + gl);
  }
}

template <int DPL>
__device__ __forceinline__ void store_lane(float* row, int gl, int ld, const float (&x)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const int b = gl * (DPL / 4) + q;
      if (DPL == 4 || 4 * b < ld)
        reinterpret_cast<float4*>(row)[b] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
  } else if constexpr (DPL == 2) {
    reinterpret_cast<float2*>(row)[gl] = make_float2(x[0], x[1]);
  } else {
    row[gl] = x[0];
  }
}

// Standard normals of the lane's dimensions from words [0, 2 ceil(d/2)) of the
// counter stream (c0, c1, c2): dimension i uses Box-Muller pair i/2.
template <int DPL>
__device__ __forceinline__ void lane_normals(const RunDesc& R, uint32_t c0, uint32_t c1, uint32_t c2,
                                             int gl, float (&z)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl * (DPL / 4) + q));
      box_muller(w.x, w.y, z[4 * q], z[4 * q + 1]);
      box_muller(w.z, w.w, z[4 * q + 2], z[4 * q + 3]);
    }
  } else if constexpr (DPL == 2) {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl >> 1));
    if (gl & 1) box_muller(w.z, w.w, z[0], z[1]);
    else box_muller(w.x, w.y, z[0], z[1]);
  } else {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl >> 2));
    float a, b;
    if (gl & 2) box_muller(w.z, w.w, a, b);
    else box_muller(w.x, w.y, a, b);
    z[0] = (gl & 1) ? b : a;
  }
}

// Uniforms of the lane's dimensions, word i for dimension i.
template <int DPL>
__device__ __forceinline__ void lane_uniform_words(const RunDesc& R, uint32_t c0, uint32_t c1, uint32_t c2,
                                                   int gl, uint32_t (&u)[DPL]) {
  if constexpr (DPL >= 4) {
#pragma unroll
    for (int q = 0; q < DPL / 4; ++q) {
      const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)(gl * (DPL / 4) + q));
      u[4 * q] = w.x; u[4 * q + 1] = w.y; u[4 * q + 2] = w.z; u[4 * q + 3] = w.w;
    }
  } else {
    const uint4 w = draw_block(R, c0, c1, c2, (uint32_t)((gl * DPL) >> 2));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    const int o = (gl * DPL) & 3;
#pragma unroll
    for (int i = 0; i < DPL; ++i) u[i] = ws[o + i];
  }
}

// The words of one HRSS step: group lane b computes Philox block b of the
// step's counter stream (iteration, chain, step, b) once; a word w < 4G is
// then read from lane w/4 by a shuffle, a later word (a shrinkage proposal
// past the first 4G - nz - 3) is drawn on demand.
template <int G>
struct StepWords {
  uint4 mine;       // block base + gl of the step's counter stream
  uint32_t base;
  uint32_t cblk;    // one-block cache for words past the shared range
  uint4 cw;
  __device__ __forceinline__ void draw(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step, int gl,
                                       uint32_t base_) {
    base = base_;
    mine = draw_block(R, iter, chain, step, base + (uint32_t)gl);
    cblk = 0xFFFFFFFFu;
  }
  // word wi, uniform over the group
  __device__ __forceinline__ uint32_t word(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step,
                                           uint32_t wi, unsigned mask) {
    const uint32_t b = wi >> 2;
    if (b >= base && b - base < (uint32_t)G) return __shfl_sync(mask, pick(mine, wi & 3u), (int)(b - base), G);
    if (b != cblk) {
      cw = draw_block(R, iter, chain, step, b);
      cblk = b;
    }
    return pick(cw, wi & 3u);
  }
  // word wi, one per lane (consecutive lanes ask for consecutive words)
  __device__ __forceinline__ uint32_t lane_word(const RunDesc& R, uint32_t iter, uint32_t chain, uint32_t step,
                                                uint32_t wi, unsigned mask) const {
    const uint32_t src = (wi >> 2) - base;
    const bool shared = src < (uint32_t)G;
    const int sl = shared ? (int)src : 0;
    const uint4 blk = make_uint4(__shfl_sync(mask, mine.x, sl, G), __shfl_sync(mask, mine.y, sl, G),
                                 __shfl_sync(mask, mine.z, sl, G), __shfl_sync(mask, mine.w, sl, G));
    if (shared) return pick(blk, wi & 3u);
    return pick(draw_block(R, iter, chain, step, wi >> 2), wi & 3u);
  }
  // all four words of block b (base <= b < base + G), for lane-specific picks
  __device__ __forceinline__ uint4 block(int b, unsigned mask) const {
    return make_uint4(__shfl_sync(mask, mine.x, b, G), __shfl_sync(mask, mine.y, b, G),
                      __shfl_sync(mask, mine.z, b, G), __shfl_sync(mask, mine.w, b, G));
  }
};

// threads per block of the grouped sweep kernels
constexpr int kSweepThreads = 32;   // one warp per block: resident warps per SM set by registers alone

// ---- configuration table ----------------------------------------------------
// grouped configurations (id, G lanes per chain, DPL dimensions per lane)
#define NSS_CFGS(X) \
  X(0, 1, 4) X(1, 2, 4) X(2, 4, 4) X(3, 8, 4) X(4, 16, 4) X(5, 32, 4) \
  X(6, 2, 2) X(7, 4, 2) X(8, 8, 2) X(9, 16, 2) X(10, 32, 2) \
  X(11, 4, 1) X(12, 8, 1) X(13, 16, 1) X(14, 32, 1) \
  X(15, 2, 8) X(16, 4, 8) X(17, 8, 8) X(18, 16, 8) \
  X(19, 2, 16) X(20, 4, 16) X(21, 8, 16)

// configurations kLaneCfg0..24: one chain per lane (nss_sweep_lane.cu), d <= 8, 16, 32
inline int lane_dmax(int cfg) { return cfg == 22 ? 8 : cfg == 23 ? 16 : 32; }


}  // namespace nss
