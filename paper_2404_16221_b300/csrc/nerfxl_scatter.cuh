// Table-gradient scatter of the backward kernels with runs merged: a thread
// that takes one level of consecutive samples (consecutive along a ray, so
// often in the same cell, most at the coarse levels) sums their corner
// contributions in registers and sends one set of reductions per run of
// samples in the same cell.
#pragma once

#include "nerfxl_field.cuh"
#include "nerfxl_tc.cuh"

namespace nerfxl {

// Corner contributions of one sample at one level into acc (corner c = x | y << 1 |
// z << 2, two features each): the trilinear weights of the cell fractions f
// (the cells and weights of the forward's gather, same arithmetic) times the
// sample's two feature gradients.
__device__ __forceinline__ void accumulate_corners(const float f[3], float g0, float g1, float acc[16]) {
  const float wx[2] = {1.0f - f[0], f[0]}, wy[2] = {1.0f - f[1], f[1]}, wz[2] = {1.0f - f[2], f[2]};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = wx[c & 1] * (wy[(c >> 1) & 1] * wz[c >> 2]);
    acc[2 * c] = fmaf(w, g0, acc[2 * c]);
    acc[2 * c + 1] = fmaf(w, g1, acc[2 * c + 1]);
  }
}

// The summed corner contributions of a run of samples in cell (cx, cy, cz) of
// level l into the region's FP32 gradient table. The corners of an x-pair
// (x, x+1) go out as one 16-byte reduction on the aligned entry pair holding
// the first corner (zero in the other half unless the second corner is that
// pair's other entry) plus, when it is not, one 8-byte reduction; both index
// forms are formed and selected per corner (measured faster here than
// branching per level).
__device__ __forceinline__ void scatter_cell(const LevelParams& lp, float2* __restrict__ gtab, int l, int cx, int cy,
                                             int cz, const float acc[16]) {
  float2* gl = gtab + lp.off[l];
  const bool dense = (lp.dense_mask >> l) & 1u;
  const LevelIndex<true> dix(lp, l, cy, cz);
  const LevelIndex<false> hix(lp, l, cy, cz);
  const uint32_t x0 = (uint32_t)cx;
  const uint64_t pol = tc::policy_evict_last();
#pragma unroll
  for (int e = 0; e < 4; ++e) {  // (y, z) corner e = y | z << 1
    const uint32_t i0 = dense ? dix(x0, e) : hix(x0, e);
    const uint32_t i1 = dense ? i0 + 1u : hix(x0 + 1u, e);
    const int c0 = ((e & 1) << 1) | ((e >> 1) << 2);  // corner (x0, y, z); (x0 + 1, y, z) is c0 | 1
    const float a0 = acc[2 * c0], a1 = acc[2 * c0 + 1], b0 = acc[2 * c0 + 2], b1 = acc[2 * c0 + 3];
    const bool pair = (i0 ^ i1) == 1u;
    const bool odd = i0 & 1u;
    const float p0 = pair ? b0 : 0.0f, p1 = pair ? b1 : 0.0f;
    tc::red_add_v4(reinterpret_cast<float4*>(gl + (i0 & ~1u)),
                   odd ? make_float4(p0, p1, a0, a1) : make_float4(a0, a1, p0, p1), pol);
    if (!pair) tc::red_add_v2(gl + i1, make_float2(b0, b1), pol);
  }
}

// One level of n consecutive rows of a tile: row i has region coordinates
// u(i), feature gradients (g0, g1) = g(i) of this level, and takes part when
// bit i of vmask is set. Equal cells of successive taking-part rows form a run.
template <int N, typename U, typename G>
__device__ __forceinline__ void scatter_runs(const LevelParams& lp, float2* __restrict__ gtab, int l, uint32_t vmask,
                                             U&& u, G&& g) {
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
  int cx = -1, cy = 0, cz = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!((vmask >> i) & 1u)) continue;
    float ui[3];
    u(i, ui);
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(ui[ax], lp.N[l], c[ax], f[ax]);
    if (cx >= 0 && (c[0] != cx || c[1] != cy || c[2] != cz)) {
      scatter_cell(lp, gtab, l, cx, cy, cz, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
    }
    cx = c[0];
    cy = c[1];
    cz = c[2];
    const float2 gi = g(i);
    accumulate_corners(f, gi.x, gi.y, acc);
  }
  if (cx >= 0) scatter_cell(lp, gtab, l, cx, cy, cz, acc);
}

// The half of a run's corner contributions with corner x offset h (0: x0,
// 1: x0 + 1): two lanes of one warp take the two halves of the same rows, so
// that each sends one 8-byte reduction per (y, z) corner and the two lanes'
// reductions of an x-pair go out in the same instruction. The memory system
// takes one request per 32-byte sector that an instruction touches, not one
// per lane: an x-pair whose entries share a sector (an aligned pair, or
// entries 4m+1 and 4m+2: three x-pairs in four, dense or hashed) costs one
// request instead of the two of a 16-byte plus an 8-byte reduction from one
// lane. Corner weights and sums as in accumulate_corners, so every
// contribution and every per-run sum is the same number as there.
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

// The level is uniform across the warp (both lanes of every pair take the
// same level), so the dense / hashed choice is a uniform branch.
__device__ __forceinline__ void scatter_half(const LevelParams& lp, float2* __restrict__ gtab, int l, int h, int cx,
                                             int cy, int cz, const float acc[8]) {
  float2* gl = gtab + lp.off[l];
  const uint32_t x = (uint32_t)(cx + h);
  if ((lp.dense_mask >> l) & 1u) scatter_half_ix<true>(lp, gl, l, x, cy, cz, acc);
  else scatter_half_ix<false>(lp, gl, l, x, cy, cz, acc);
}

// scatter_runs for the x-half h of the corners (the partner lane, which takes
// the other half of the same rows, runs the same cells in step).
template <int N, typename U, typename G>
__device__ __forceinline__ void scatter_runs_half(const LevelParams& lp, float2* __restrict__ gtab, int l, int h,
                                                  uint32_t vmask, U&& u, G&& g) {
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
  int cx = -1, cy = 0, cz = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!((vmask >> i) & 1u)) continue;
    float ui[3];
    u(i, ui);
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(ui[ax], lp.N[l], c[ax], f[ax]);
    if (cx >= 0 && (c[0] != cx || c[1] != cy || c[2] != cz)) {
      scatter_half(lp, gtab, l, h, cx, cy, cz, acc);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
    }
    cx = c[0];
    cy = c[1];
    cz = c[2];
    const float2 gi = g(i);
    accumulate_half(f, h, gi.x, gi.y, acc);
  }
  if (cx >= 0) scatter_half(lp, gtab, l, h, cx, cy, cz, acc);
}

// scatter_runs_half with the row loop rolled: u(i) and g(i) read their row
// where it is (shared memory), and the code holds one reduction site.
template <int N, typename U, typename G>
__device__ __forceinline__ void scatter_runs_half_rolled(const LevelParams& lp, float2* __restrict__ gtab, int l,
                                                         int h, uint32_t vmask, U&& u, G&& g) {
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
  int cx = -1, cy = 0, cz = 0;
  const int n = lp.N[l];
#pragma unroll 1
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
      scatter_half(lp, gtab, l, h, cx, cy, cz, acc);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
    }
    cx = c[0];
    cy = c[1];
    cz = c[2];
    accumulate_half(f, h, gi.x, gi.y, acc);
  }
  if (cx >= 0) scatter_half(lp, gtab, l, h, cx, cy, cz, acc);
}

}  // namespace nerfxl
