// Table-gradient scatter of the backward kernels with runs merged: a pair of
// lanes takes one level of consecutive samples (consecutive along a ray, so
// often in the same cell, most at the coarse levels), sums their corner
// contributions in registers and sends one set of reductions per run of
// samples in the same cell.
#pragma once

#include "nerfxl_field.cuh"
#include "nerfxl_tc.cuh"

namespace nerfxl {

// The half of a run's corner contributions with corner x offset h (0: x0,
// 1: x0 + 1): two lanes of one warp take the two halves of the same rows, so
// that each sends one 8-byte reduction per (y, z) corner and the two lanes'
// reductions of an x-pair go out in the same instruction. The memory system
// takes one request per 32-byte sector that an instruction touches, not one
// per lane: an x-pair whose entries share a sector (one aligned group of four
// 8-byte entries: dense, unless the first entry is the last of its group;
// hashed with the x prime 1, unless x = 3 mod 4; three x-pairs in four) costs
// one request instead of the two of a 16-byte plus an 8-byte reduction from
// one lane. The corner weight is wx (wy wz), the trilinear weight of the
// forward's gather (same arithmetic).
__device__ __forceinline__ void accumulate_half(const float f[3], int h, float g0, float g1, float acc[8]) {
  const float wx = h ? f[0] : 1.0f - f[0];
  const float wy[2] = {1.0f - f[1], f[1]}, wz[2] = {1.0f - f[2], f[2]};
#pragma unroll
  for (int e = 0; e < 4; ++e) {  // (y, z) corner e = y | z << 1
    const float w = wx * (wy[e & 1] * wz[e >> 1]);
    acc[2 * e] = fmaf(w, g0, acc[2 * e]);
    acc[2 * e + 1] = fmaf(w, g1, acc[2 * e + 1]);
  }
}

template <bool kDense>
__device__ __forceinline__ void scatter_half_ix(const LevelParams& lp, float2* __restrict__ gl, int l, uint32_t x,
                                                int cy, int cz, const float acc[8]) {
  const LevelIndex<kDense> ix(lp, l, cy, cz);
  const uint64_t pol = tc::policy_evict_last();
#pragma unroll
  for (int e = 0; e < 4; ++e) tc::red_add_v2(gl + ix(x, e), make_float2(acc[2 * e], acc[2 * e + 1]), pol);
}

// kUniform: the level is the same across the warp, so the dense / hashed
// choice is a uniform branch; otherwise both index forms are formed and
// selected per corner (no divergence).
template <bool kUniform>
__device__ __forceinline__ void scatter_half(const LevelParams& lp, float2* __restrict__ gtab, int l, int h, int cx,
                                             int cy, int cz, const float acc[8]) {
  float2* gl = gtab + lp.off[l];
  const uint32_t x = (uint32_t)(cx + h);
  const bool dense = (lp.dense_mask >> l) & 1u;
  if (kUniform) {
    if (dense) scatter_half_ix<true>(lp, gl, l, x, cy, cz, acc);
    else scatter_half_ix<false>(lp, gl, l, x, cy, cz, acc);
  } else {
    const LevelIndex<true> dix(lp, l, cy, cz);
    const LevelIndex<false> hix(lp, l, cy, cz);
    const uint64_t pol = tc::policy_evict_last();
#pragma unroll
    for (int e = 0; e < 4; ++e)
      tc::red_add_v2(gl + (dense ? dix(x, e) : hix(x, e)), make_float2(acc[2 * e], acc[2 * e + 1]), pol);
  }
}

// One level of n consecutive rows of a tile, x-half h of the corners (the
// partner lane, which takes the other half of the same rows, runs the same
// cells in step): row i has region coordinates u(i), feature gradients
// (g0, g1) = g(i) of this level, and takes part when bit i of vmask is set;
// equal cells of successive taking-part rows form a run. The row loop is
// unrolled by two only (u(i) and g(i) read their row where it is, in shared
// memory), so the code holds two reduction sites: in a warp-specialized
// kernel the other warps' code runs beside this on the same SM, and a fully
// unrolled scatter's size showed as instruction-fetch stalls.
template <int N, bool kUniform, typename U, typename G>
__device__ __forceinline__ void scatter_runs_half(const LevelParams& lp, float2* __restrict__ gtab, int l, int h,
                                                  uint32_t vmask, U&& u, G&& g) {
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
  int cx = -1, cy = 0, cz = 0;
  const int n = lp.N[l];
#pragma unroll 2
  for (int i = 0; i < N; ++i) {
    if (!((vmask >> i) & 1u)) continue;
    float ui[3];
    u(i, ui);
    const float2 gi = g(i);
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(ui[ax], n, c[ax], f[ax]);
    if (cx >= 0 && (c[0] != cx || c[1] != cy || c[2] != cz)) {
      scatter_half<kUniform>(lp, gtab, l, h, cx, cy, cz, acc);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
    }
    cx = c[0];
    cy = c[1];
    cz = c[2];
    accumulate_half(f, h, gi.x, gi.y, acc);
  }
  if (cx >= 0) scatter_half<kUniform>(lp, gtab, l, h, cx, cy, cz, acc);
}

}  // namespace nerfxl
