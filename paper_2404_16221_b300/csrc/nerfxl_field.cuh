// Per-sample field evaluation and chunk rendering shared by the forward,
// backward and debug kernels (FP32 plain path).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nerfxl_device.cuh"

namespace nerfxl {

// ---------------------------------------------------------------------------
// Field evaluation of one sample, FP32 plain path.

struct FieldPtrs {
  const float* boxes;
  const float* tables;  // [K][E][2]
  const float* mlp;     // [K][kMlpParams]
};

// Hash-grid encoding of one level (F = 2): the two features
// sum_corners w * table[l][idx][j].
__device__ __forceinline__ float2 encode_level_f32(const LevelParams& lp, const float2* __restrict__ table,
                                                   const float u[3], int l) {
  int c[3];
  float f[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
  float2 v[8];
  const float2* tl = table + lp.off[l];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    // x-neighbour pair: one aligned 16-byte load covers both corners when
    // their indices differ only in bit 0 (even x for hashed levels, even
    // index for dense ones); otherwise a second 8-byte load.
    const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
    const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
    const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
    const float4 q = __ldg(reinterpret_cast<const float4*>(tl + (i0 & ~1u)));
    const bool odd = i0 & 1u;
    v[e] = odd ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
    if ((i0 ^ i1) == 1u) v[e + 1] = odd ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
    else v[e + 1] = __ldg(tl + i1);
  }
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const float w = ((e & 1) ? f[0] : 1.0f - f[0]) * (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) *
                    (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
    s0 = fmaf(w, v[e].x, s0);
    s1 = fmaf(w, v[e].y, s1);
  }
  return make_float2(s0, s1);
}

// Hash-grid encoding (F = 2): feat[2l + j] = sum_corners w * table[l][idx][j].
__device__ __forceinline__ void encode_f32(const LevelParams& lp, const float2* __restrict__ table, const float u[3],
                                           float feat[kIn]) {
#pragma unroll
  for (int i = 0; i < kIn; ++i) feat[i] = 0.0f;
#pragma unroll
  for (int l = 0; l < kIn / 2; ++l) {
    if (l >= lp.L) break;
    const float2 v = encode_level_f32(lp, table, u, l);
    feat[2 * l] = v.x;
    feat[2 * l + 1] = v.y;
  }
}

// Corner indices of one level, set up once per cell and shared by its four
// x-pairs: corner (x, y + dy, z + dz) has index x + yz[dy + 2 dz] on a dense
// level and (x ^ yz[dy + 2 dz]) & mask on a hashed one.
template <bool kDense>
struct LevelIndex {
  uint32_t yz[4];
  uint32_t mask;
  __device__ LevelIndex(const LevelParams& lp, int l, int cy, int cz) {
    if (kDense) {
      const uint32_t side = (uint32_t)lp.N[l] + 1u;
      const uint32_t b = (uint32_t)cy * side + (uint32_t)cz * side * side;
      yz[0] = b;
      yz[1] = b + side;
      yz[2] = b + side * side;
      yz[3] = b + side + side * side;
    } else {
      const uint32_t hy0 = (uint32_t)cy * kHashPrime2, hy1 = hy0 + kHashPrime2;
      const uint32_t hz0 = (uint32_t)cz * kHashPrime3, hz1 = hz0 + kHashPrime3;
      yz[0] = hy0 ^ hz0;
      yz[1] = hy1 ^ hz0;
      yz[2] = hy0 ^ hz1;
      yz[3] = hy1 ^ hz1;
    }
    mask = lp.hash_mask;
  }
  __device__ uint32_t operator()(uint32_t x, int e) const { return kDense ? x + yz[e] : ((x ^ yz[e]) & mask); }
};

// Pair loads of the gather: the aligned entry pair holding a corner (first =
// the corner's own entry, second = the other entry of the pair), and one
// entry, as float2 features. The 16-bit form picks the 32-bit word before
// converting it.
template <typename TabT>
struct PairLoad;
template <>
struct PairLoad<float2> {
  using P = float4;
  __device__ static P pair(const float2* t, uint32_t i) { return __ldg(reinterpret_cast<const float4*>(t + (i & ~1u))); }
  __device__ static float2 first(const P& v, bool odd) { return odd ? make_float2(v.z, v.w) : make_float2(v.x, v.y); }
  __device__ static float2 second(const P& v, bool odd) { return odd ? make_float2(v.x, v.y) : make_float2(v.z, v.w); }
  __device__ static float2 one(const float2* t, uint32_t i) { return __ldg(t + i); }
};
template <>
struct PairLoad<__half2> {
  using P = uint2;
  __device__ static P pair(const __half2* t, uint32_t i) { return __ldg(reinterpret_cast<const uint2*>(t + (i & ~1u))); }
  __device__ static float2 cvt(uint32_t w) { return __half22float2(*reinterpret_cast<const __half2*>(&w)); }
  __device__ static float2 first(const P& v, bool odd) { return cvt(odd ? v.y : v.x); }
  __device__ static float2 second(const P& v, bool odd) { return cvt(odd ? v.x : v.y); }
  __device__ static float2 one(const __half2* t, uint32_t i) { return __half22float2(__ldg(t + i)); }
};

// One level's trilinear gather (F = 2) at cell c, fractions f.
template <bool kDense, typename TabT>
__device__ __forceinline__ float2 gather_level(const LevelParams& lp, const TabT* __restrict__ tl, int l, const int c[3],
                                               const float f[3]) {
  using LD = PairLoad<TabT>;
  const LevelIndex<kDense> ix(lp, l, c[1], c[2]);
  const uint32_t x0 = (uint32_t)c[0];
  const float wy[2] = {1.0f - f[1], f[1]}, wz[2] = {1.0f - f[2], f[2]};
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint32_t i0 = ix(x0, e), i1 = ix(x0 + 1u, e);
    const typename LD::P pv = LD::pair(tl, i0);
    const bool odd = i0 & 1u;
    const float2 v0 = LD::first(pv, odd);
    float2 v1;
    if ((i0 ^ i1) == 1u) v1 = LD::second(pv, odd);
    else v1 = LD::one(tl, i1);
    const float wyz = wy[e & 1] * wz[e >> 1];
    const float w0 = (1.0f - f[0]) * wyz, w1 = f[0] * wyz;
    s0 = fmaf(w0, v0.x, s0);
    s1 = fmaf(w0, v0.y, s1);
    s0 = fmaf(w1, v1.x, s0);
    s1 = fmaf(w1, v1.y, s1);
  }
  return make_float2(s0, s1);
}

// Gather of four consecutive levels l0..l0+3 (F = 2) of one sample: out[8]
// holds their features in level order; levels >= L give zeros.
template <typename TabT>
__device__ __forceinline__ void gather4(const LevelParams& lp, const TabT* __restrict__ table, const float u[3], int l0,
                                        float out[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l = l0 + q;
    float2 s = make_float2(0.0f, 0.0f);
    if (l < lp.L) {
      int c[3];
      float f[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
      const TabT* tl = table + lp.off[l];
      if ((lp.dense_mask >> l) & 1u) s = gather_level<true>(lp, tl, l, c, f);
      else s = gather_level<false>(lp, tl, l, c, f);
    }
    out[2 * q] = s.x;
    out[2 * q + 1] = s.y;
  }
}

// FP16 tables: per-corner index arithmetic, which schedules better than the
// per-cell form above for 4-byte entries.
template <>
__device__ __forceinline__ void gather4<__half2>(const LevelParams& lp, const __half2* __restrict__ table,
                                                 const float u[3], int l0, float out[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l = l0 + q;
    float s0 = 0.0f, s1 = 0.0f;
    if (l < lp.L) {
      int c[3];
      float f[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
      const __half2* tl = table + lp.off[l];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
        const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
        const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
        const uint2 qv = __ldg(reinterpret_cast<const uint2*>(tl + (i0 & ~1u)));
        const bool odd = i0 & 1u;
        const uint32_t a = odd ? qv.y : qv.x, b = odd ? qv.x : qv.y;
        const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&a));
        float2 v1;
        if ((i0 ^ i1) == 1u) v1 = __half22float2(*reinterpret_cast<const __half2*>(&b));
        else v1 = __half22float2(__ldg(tl + i1));
        const float wyz = (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) * (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
        const float w0 = (1.0f - f[0]) * wyz, w1 = f[0] * wyz;
        s0 = fmaf(w0, v0.x, s0);
        s1 = fmaf(w0, v0.y, s1);
        s0 = fmaf(w1, v1.x, s0);
        s1 = fmaf(w1, v1.y, s1);
      }
    }
    out[2 * q] = s0;
    out[2 * q + 1] = s1;
  }
}

// One level l < L of one sample, with exactly the arithmetic of one level of
// gather4 (the level-grouped gather computes the same features bit for bit).
template <typename TabT>
__device__ __forceinline__ float2 gather1(const LevelParams& lp, const TabT* __restrict__ table, const float u[3],
                                          int l) {
  int c[3];
  float f[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
  const TabT* tl = table + lp.off[l];
  if ((lp.dense_mask >> l) & 1u) return gather_level<true>(lp, tl, l, c, f);
  return gather_level<false>(lp, tl, l, c, f);
}

template <>
__device__ __forceinline__ float2 gather1<__half2>(const LevelParams& lp, const __half2* __restrict__ table,
                                                   const float u[3], int l) {
  float s0 = 0.0f, s1 = 0.0f;
  int c[3];
  float f[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
  const __half2* tl = table + lp.off[l];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
    const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
    const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
    const uint2 qv = __ldg(reinterpret_cast<const uint2*>(tl + (i0 & ~1u)));
    const bool odd = i0 & 1u;
    const uint32_t a = odd ? qv.y : qv.x, b = odd ? qv.x : qv.y;
    const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&a));
    float2 v1;
    if ((i0 ^ i1) == 1u) v1 = __half22float2(*reinterpret_cast<const __half2*>(&b));
    else v1 = __half22float2(__ldg(tl + i1));
    const float wyz = (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) * (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
    const float w0 = (1.0f - f[0]) * wyz, w1 = f[0] * wyz;
    s0 = fmaf(w0, v0.x, s0);
    s1 = fmaf(w0, v0.y, s1);
    s0 = fmaf(w1, v1.x, s0);
    s1 = fmaf(w1, v1.y, s1);
  }
  return make_float2(s0, s1);
}

// MLP with weights staged in shared memory as W1t [64][32] (row n holds
// column n of W1), W2t [64][64], W3 [64][4]. Layer 2 and 3 are fused per
// hidden unit so that only h1 stays live.
__device__ __forceinline__ void mlp_f32_smem(const float* __restrict__ s_w, const float feat[kIn], float out[kOut]) {
  const float4* W1t = reinterpret_cast<const float4*>(s_w);
  const float4* W2t = reinterpret_cast<const float4*>(s_w + kIn * kWidth);
  const float4* W3 = reinterpret_cast<const float4*>(s_w + kIn * kWidth + kWidth * kWidth);
  float h1[kWidth];
#pragma unroll
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
#pragma unroll
    for (int i4 = 0; i4 < kIn / 4; ++i4) {
      const float4 w = W1t[n * (kIn / 4) + i4];
      acc = fmaf(feat[4 * i4 + 0], w.x, acc);
      acc = fmaf(feat[4 * i4 + 1], w.y, acc);
      acc = fmaf(feat[4 * i4 + 2], w.z, acc);
      acc = fmaf(feat[4 * i4 + 3], w.w, acc);
    }
    h1[n] = fmaxf(acc, 0.0f);
  }
  float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f, o3 = 0.0f;
#pragma unroll 2
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
#pragma unroll
    for (int i4 = 0; i4 < kWidth / 4; ++i4) {
      const float4 w = W2t[n * (kWidth / 4) + i4];
      acc = fmaf(h1[4 * i4 + 0], w.x, acc);
      acc = fmaf(h1[4 * i4 + 1], w.y, acc);
      acc = fmaf(h1[4 * i4 + 2], w.z, acc);
      acc = fmaf(h1[4 * i4 + 3], w.w, acc);
    }
    const float h2 = fmaxf(acc, 0.0f);
    const float4 w3 = W3[n];
    o0 = fmaf(h2, w3.x, o0);
    o1 = fmaf(h2, w3.y, o1);
    o2 = fmaf(h2, w3.z, o2);
    o3 = fmaf(h2, w3.w, o3);
  }
  out[0] = o0;
  out[1] = o1;
  out[2] = o2;
  out[3] = o3;
}

// Stage region k's FP32 MLP block into shared memory (transposed layout).
__device__ __forceinline__ void load_mlp_f32(const float* __restrict__ blk, float* __restrict__ s_w) {
  for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;  // W1[row][col]
    s_w[col * kIn + row] = blk[i];
  }
  const float* W2 = blk + kIn * kWidth;
  float* s2 = s_w + kIn * kWidth;
  for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;
    s2[col * kWidth + row] = W2[i];
  }
  const float* W3 = W2 + kWidth * kWidth;
  float* s3 = s2 + kWidth * kWidth;
  for (int i = threadIdx.x; i < kWidth * kOut; i += blockDim.x) s3[i] = W3[i];
}

// Chunk partial: {tau, C[3], A, D', L, 0}; D' and L use t' = tbar - tn.
struct Partial {
  float tau, c0, c1, c2, A, D, L;
};

// Region-local volume rendering of one chunk by the `width` lanes holding it
// (Eq. 1-2 restricted to the chunk, transmittance restarting at 1; `lane` is
// the sample's index in the chunk, every lane of the warp calls this). If
// `keep` is given, the lane also stores the quantities its adjoint reuses:
// keep[0] = Tn (transmittance after the sample), keep[stride] = w,
// keep[2 stride] = sum_j w_j |tr - tr_j| over the chunk.
__device__ __forceinline__ Partial render_chunk(float sigma, const float rgb[3], float tr, float dl, int lane,
                                                float* keep = nullptr, int stride = 0, int width = 32) {
  const float tau = sigma * dl;
  const float incl = warp_inclusive_scan(tau, lane, width);
  const float excl = warp_exclusive_from_inclusive(incl, lane, width);
  const float T = expf(-excl);
  const float alpha = -expm1f(-tau);
  const float w = T * alpha;
  const float wt = w * tr;
  const float Wx = warp_exclusive_from_inclusive(warp_inclusive_scan(w, lane, width), lane, width);
  const float WTx = warp_exclusive_from_inclusive(warp_inclusive_scan(wt, lane, width), lane, width);
  const float l = 2.0f * w * (tr * Wx - WTx) + w * w * dl * (1.0f / 3.0f);
  if (keep) {
    const float W_gt = warp_suffix_scan(w, lane, width) - w;
    const float WT_gt = warp_suffix_scan(wt, lane, width) - wt;
    __stcs(keep, expf(-incl));
    __stcs(keep + stride, w);
    __stcs(keep + 2 * stride, (tr * Wx - WTx) + (WT_gt - tr * W_gt));
  }
  Partial p;
  p.tau = __shfl_sync(0xFFFFFFFFu, incl, width - 1, width);
  p.c0 = warp_sum(w * rgb[0], width);
  p.c1 = warp_sum(w * rgb[1], width);
  p.c2 = warp_sum(w * rgb[2], width);
  p.A = warp_sum(w, width);
  p.D = warp_sum(wt, width);
  p.L = warp_sum(l, width);
  return p;
}


// Hash-grid gather for FP16 tables: one 4-byte half2 per corner, 8-byte x-pairs.
__device__ __forceinline__ void encode_f16(const LevelParams& lp, const __half2* __restrict__ table, const float u[3],
                                           float feat[kIn]) {
#pragma unroll
  for (int i = 0; i < kIn; ++i) feat[i] = 0.0f;
#pragma unroll
  for (int l = 0; l < kIn / 2; ++l) {
    if (l >= lp.L) break;
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
    const __half2* tl = table + lp.off[l];
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
      const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
      const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(tl + (i0 & ~1u)));
      const bool odd = i0 & 1u;
      const uint32_t a = odd ? q.y : q.x, b = odd ? q.x : q.y;
      v[e] = __half22float2(*reinterpret_cast<const __half2*>(&a));
      if ((i0 ^ i1) == 1u) {
        v[e + 1] = __half22float2(*reinterpret_cast<const __half2*>(&b));
      } else {
        v[e + 1] = __half22float2(__ldg(tl + i1));
      }
    }
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float w = ((e & 1) ? f[0] : 1.0f - f[0]) * (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) *
                      (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
      s0 = fmaf(w, v[e].x, s0);
      s1 = fmaf(w, v[e].y, s1);
    }
    feat[2 * l] = s0;
    feat[2 * l + 1] = s1;
  }
}

template <bool kF16Table>
struct TableOf;
template <>
struct TableOf<false> {
  using T = float2;
  __device__ static void encode(const LevelParams& lp, const void* t, const float u[3], float feat[kIn]) {
    encode_f32(lp, static_cast<const float2*>(t), u, feat);
  }
};
template <>
struct TableOf<true> {
  using T = __half2;
  __device__ static void encode(const LevelParams& lp, const void* t, const float u[3], float feat[kIn]) {
    encode_f16(lp, static_cast<const __half2*>(t), u, feat);
  }
};

// Adjoint of the chunk-local render for the `width` lanes of one chunk
// (`lane`: index in the chunk). Inputs per lane: sigma, rgb, t' (tbar - tn),
// delta; chunk adjoints gtc, gC, gA, gD, gL. Returns dL/d(sigma), dL/d(rgb).
__device__ __forceinline__ void render_chunk_adjoint(float sigma, const float rgb[3], float tr, float dl, int lane,
                                                     float gtc, const float gC[3], float gA, float gD, float gL,
                                                     float& g_sigma, float g_rgb[3], int width = 32) {
  const float tau = sigma * dl;
  const float incl = warp_inclusive_scan(tau, lane, width);
  const float excl = warp_exclusive_from_inclusive(incl, lane, width);
  const float T = expf(-excl);
  const float Tn = expf(-incl);
  const float w = T * -expm1f(-tau);
  const float wt = w * tr;
  const float W_in = warp_inclusive_scan(w, lane, width);
  const float WT_in = warp_inclusive_scan(wt, lane, width);
  const float W_lt = warp_exclusive_from_inclusive(W_in, lane, width);
  const float WT_lt = warp_exclusive_from_inclusive(WT_in, lane, width);
  const float W_gt = warp_suffix_scan(w, lane, width) - w;
  const float WT_gt = warp_suffix_scan(wt, lane, width) - wt;
  // sum_j w_j |t_i - t_j| over the chunk
  const float pair = (tr * W_lt - WT_lt) + (WT_gt - tr * W_gt);
  const float gw = gC[0] * rgb[0] + gC[1] * rgb[1] + gC[2] * rgb[2] + gA + gD * tr +
                   gL * (2.0f * pair + (2.0f / 3.0f) * w * dl);
  const float gww = gw * w;
  const float later = warp_suffix_scan(gww, lane, width) - gww;  // sum_{j > i} g_w_j w_j
  const float g_tau = gtc + gw * Tn - later;
  g_sigma = g_tau * dl;
#pragma unroll
  for (int q = 0; q < 3; ++q) g_rgb[q] = w * gC[q];
}

// Adjoint of the chunk-local render from the forward's kept Tn, w and pair
// (see render_chunk): one suffix scan instead of the recomputed prefix sums.
__device__ __forceinline__ void render_chunk_adjoint_kept(float rgb_dot_gC, float tr, float dl, float Tn, float w,
                                                          float pair, int lane, float gtc, float gA, float gD, float gL,
                                                          float& g_tau, int width = 32) {
  const float gw = rgb_dot_gC + gA + gD * tr + gL * (2.0f * pair + (2.0f / 3.0f) * w * dl);
  const float gww = gw * w;
  const float later = warp_suffix_scan(gww, lane, width) - gww;  // sum_{j > i} g_w_j w_j
  g_tau = gtc + gw * Tn - later;
}

// Stage region k's 16-bit MLP block into shared memory as FP32 (same
// transposed layout as load_mlp_f32).
template <int kMlpType>  // 1 = bf16, 2 = fp16
__device__ __forceinline__ float mlp_elem(const void* blk, int i) {
  if (kMlpType == 1) return __bfloat162float(static_cast<const __nv_bfloat16*>(blk)[i]);
  if (kMlpType == 2) return __half2float(static_cast<const __half*>(blk)[i]);
  return static_cast<const float*>(blk)[i];
}

template <int kMlpType>
__device__ __forceinline__ void load_mlp_any(const void* blk, float* __restrict__ s_w) {
  for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;
    s_w[col * kIn + row] = mlp_elem<kMlpType>(blk, i);
  }
  float* s2 = s_w + kIn * kWidth;
  for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;
    s2[col * kWidth + row] = mlp_elem<kMlpType>(blk, kIn * kWidth + i);
  }
  float* s3 = s2 + kWidth * kWidth;
  for (int i = threadIdx.x; i < kWidth * kOut; i += blockDim.x) s3[i] = mlp_elem<kMlpType>(blk, kIn * kWidth + kWidth * kWidth + i);
}

// MLP reading the row-major block W1 [32][64], W2 [64][64], W3 [64][4]
// straight from global memory (debug views only).
__device__ __forceinline__ void mlp_f32_global(const float* __restrict__ blk, const float feat[kIn], float out[kOut]) {
  const float* W1 = blk;
  const float* W2 = blk + kIn * kWidth;
  const float* W3 = W2 + kWidth * kWidth;
  float h1[kWidth];
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
    for (int i = 0; i < kIn; ++i) acc = fmaf(feat[i], W1[i * kWidth + n], acc);
    h1[n] = fmaxf(acc, 0.0f);
  }
  for (int m = 0; m < kOut; ++m) out[m] = 0.0f;
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
    for (int i = 0; i < kWidth; ++i) acc = fmaf(h1[i], W2[i * kWidth + n], acc);
    const float h2 = fmaxf(acc, 0.0f);
    for (int m = 0; m < kOut; ++m) out[m] = fmaf(h2, W3[n * kOut + m], out[m]);
  }
}

}  // namespace nerfxl
