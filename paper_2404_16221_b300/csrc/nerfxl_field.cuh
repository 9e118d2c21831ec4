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

// Hash-grid encoding (F = 2): feat[2l + j] = sum_corners w * table[l][idx][j].
__device__ __forceinline__ void encode_f32(const LevelParams& lp, const float2* __restrict__ table, const float u[3],
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
    feat[2 * l] = s0;
    feat[2 * l + 1] = s1;
  }
}

// Gather of four consecutive levels l0..l0+3 (F = 2) of one sample: out[8]
// holds their features in level order; levels >= L give zeros.
template <typename TabT>
__device__ __forceinline__ void gather4(const LevelParams& lp, const TabT* __restrict__ table, const float u[3], int l0,
                                        float out[8]);

template <>
__device__ __forceinline__ void gather4<float2>(const LevelParams& lp, const float2* __restrict__ table,
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
      const float2* tl = table + lp.off[l];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
        const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
        const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
        const float4 qv = __ldg(reinterpret_cast<const float4*>(tl + (i0 & ~1u)));
        const bool odd = i0 & 1u;
        const float2 v0 = odd ? make_float2(qv.z, qv.w) : make_float2(qv.x, qv.y);
        float2 v1;
        if ((i0 ^ i1) == 1u) v1 = odd ? make_float2(qv.x, qv.y) : make_float2(qv.z, qv.w);
        else v1 = __ldg(tl + i1);
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

// Region-local volume rendering of one 32-sample chunk by one warp
// (Eq. 1-2 restricted to the chunk, transmittance restarting at 1). If `keep`
// is given, the lane also stores the quantities its adjoint reuses:
// keep[0] = Tn (transmittance after the sample), keep[stride] = w,
// keep[2 stride] = sum_j w_j |tr - tr_j| over the chunk.
__device__ __forceinline__ Partial render_chunk(float sigma, const float rgb[3], float tr, float dl, int lane,
                                                float* keep = nullptr, int stride = 0) {
  const float tau = sigma * dl;
  const float incl = warp_inclusive_scan(tau, lane);
  const float excl = warp_exclusive_from_inclusive(incl, lane);
  const float T = expf(-excl);
  const float alpha = -expm1f(-tau);
  const float w = T * alpha;
  const float wt = w * tr;
  const float Wx = warp_exclusive_from_inclusive(warp_inclusive_scan(w, lane), lane);
  const float WTx = warp_exclusive_from_inclusive(warp_inclusive_scan(wt, lane), lane);
  const float l = 2.0f * w * (tr * Wx - WTx) + w * w * dl * (1.0f / 3.0f);
  if (keep) {
    const float W_gt = warp_suffix_scan(w, lane) - w;
    const float WT_gt = warp_suffix_scan(wt, lane) - wt;
    keep[0] = expf(-incl);
    keep[stride] = w;
    keep[2 * stride] = (tr * Wx - WTx) + (WT_gt - tr * W_gt);
  }
  Partial p;
  p.tau = __shfl_sync(0xFFFFFFFFu, incl, 31);
  p.c0 = warp_sum(w * rgb[0]);
  p.c1 = warp_sum(w * rgb[1]);
  p.c2 = warp_sum(w * rgb[2]);
  p.A = warp_sum(w);
  p.D = warp_sum(wt);
  p.L = warp_sum(l);
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

// Adjoint of the chunk-local render for one warp (one chunk). Inputs per lane:
// sigma, rgb, t' (tbar - tn), delta; chunk adjoints gtc, gC, gA, gD, gL.
// Returns dL/d(sigma), dL/d(rgb).
__device__ __forceinline__ void render_chunk_adjoint(float sigma, const float rgb[3], float tr, float dl, int lane,
                                                     float gtc, const float gC[3], float gA, float gD, float gL,
                                                     float& g_sigma, float g_rgb[3]) {
  const float tau = sigma * dl;
  const float incl = warp_inclusive_scan(tau, lane);
  const float excl = warp_exclusive_from_inclusive(incl, lane);
  const float T = expf(-excl);
  const float Tn = expf(-incl);
  const float w = T * -expm1f(-tau);
  const float wt = w * tr;
  const float W_in = warp_inclusive_scan(w, lane);
  const float WT_in = warp_inclusive_scan(wt, lane);
  const float W_lt = warp_exclusive_from_inclusive(W_in, lane);
  const float WT_lt = warp_exclusive_from_inclusive(WT_in, lane);
  const float W_gt = warp_suffix_scan(w, lane) - w;
  const float WT_gt = warp_suffix_scan(wt, lane) - wt;
  // sum_j w_j |t_i - t_j| over the chunk
  const float pair = (tr * W_lt - WT_lt) + (WT_gt - tr * W_gt);
  const float gw = gC[0] * rgb[0] + gC[1] * rgb[1] + gC[2] * rgb[2] + gA + gD * tr +
                   gL * (2.0f * pair + (2.0f / 3.0f) * w * dl);
  const float gww = gw * w;
  const float later = warp_suffix_scan(gww, lane) - gww;  // sum_{j > i} g_w_j w_j
  const float g_tau = gtc + gw * Tn - later;
  g_sigma = g_tau * dl;
#pragma unroll
  for (int q = 0; q < 3; ++q) g_rgb[q] = w * gC[q];
}

// Adjoint of the chunk-local render from the forward's kept Tn, w and pair
// (see render_chunk): one suffix scan instead of the recomputed prefix sums.
__device__ __forceinline__ void render_chunk_adjoint_kept(float rgb_dot_gC, float tr, float dl, float Tn, float w,
                                                          float pair, int lane, float gtc, float gA, float gD, float gL,
                                                          float& g_tau) {
  const float gw = rgb_dot_gC + gA + gD * tr + gL * (2.0f * pair + (2.0f / 3.0f) * w * dl);
  const float gww = gw * w;
  const float later = warp_suffix_scan(gww, lane) - gww;  // sum_{j > i} g_w_j w_j
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
