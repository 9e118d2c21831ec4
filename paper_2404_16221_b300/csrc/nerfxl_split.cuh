// Split representation (App. A.1, after Instant-NGP): per region a hash
// encoding and a density MLP feat -> 64 -> 16 (g; density = exp(g0)); one
// colour MLP shared by all regions on [g, SH(d)] -> 64 -> 64 -> 3 (colour =
// sigmoid). FP32 building blocks used by the forward, backward and grid
// refresh kernels.
#pragma once

#include "nerfxl_field.cuh"

namespace nerfxl {

constexpr int kGeo = 16;                                  // density MLP outputs
constexpr int kSh = 16;                                   // SH coefficients, degrees 0..3
constexpr int kColorIn = kGeo + kSh;                      // 32
constexpr int kDensityParams = kIn * kWidth + kWidth * kGeo;  // Wd1 [32][64], Wd2 [64][16]
constexpr int kColorParams = kColorIn * kWidth + kWidth * kWidth + kWidth * kOut;  // Wc1, Wc2, Wc3 [64][4]
constexpr int kSplitSmemFloats = kDensityParams + kColorParams;

// Real spherical harmonics of degrees 0..3 of the unit vector d (Condon-Shortley
// phase, Y_l^m for m = -l..l): constant normalisations of the Cartesian forms.
__device__ __forceinline__ void sh4_f32(const float d[3], float y[kSh]) {
  const float x = d[0], yy = d[1], z = d[2];
  const float xx = x * x, y2 = yy * yy, zz = z * z;
  y[0] = 0.28209479177387814f;                 // 1 / (2 sqrt(pi))
  y[1] = -0.48860251190291992f * yy;           // sqrt(3 / (4 pi))
  y[2] = 0.48860251190291992f * z;
  y[3] = -0.48860251190291992f * x;
  y[4] = 1.0925484305920792f * x * yy;         // sqrt(15 / pi) / 2
  y[5] = -1.0925484305920792f * yy * z;
  y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);  // sqrt(5 / pi) / 4
  y[7] = -1.0925484305920792f * x * z;
  y[8] = 0.54627421529603959f * (xx - y2);     // sqrt(15 / pi) / 4
  y[9] = -0.59004358992664352f * yy * (3.0f * xx - y2);   // sqrt(35 / (2 pi)) / 4
  y[10] = 2.8906114426405538f * x * yy * z;               // sqrt(105 / pi) / 2
  y[11] = -0.45704579946446572f * yy * (5.0f * zz - 1.0f);  // sqrt(21 / (2 pi)) / 4
  y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);     // sqrt(7 / pi) / 4
  y[13] = -0.45704579946446572f * x * (5.0f * zz - 1.0f);
  y[14] = 1.4453057213202769f * z * (xx - y2);              // sqrt(105 / pi) / 4
  y[15] = -0.59004358992664352f * x * (xx - 3.0f * y2);
}

// Shared-memory layout of the split weights (FP32):
//   density: Wd1t [64][32] (row n = column n of Wd1), Wd2 [64][16] (as stored);
//   colour:  Wc1t [64][32], Wc2t [64][64], Wc3 [64][4].
__device__ __forceinline__ void load_density_f32(const float* __restrict__ blk, float* __restrict__ s_d) {
  for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;  // Wd1[row][col]
    s_d[col * kIn + row] = blk[i];
  }
  for (int i = threadIdx.x; i < kWidth * kGeo; i += blockDim.x) s_d[kIn * kWidth + i] = blk[kIn * kWidth + i];
}

__device__ __forceinline__ void load_color_f32(const float* __restrict__ blk, float* __restrict__ s_c) {
  for (int i = threadIdx.x; i < kColorIn * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;  // Wc1[row][col]
    s_c[col * kColorIn + row] = blk[i];
  }
  const float* W2 = blk + kColorIn * kWidth;
  float* s2 = s_c + kColorIn * kWidth;
  for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
    const int row = i / kWidth, col = i % kWidth;
    s2[col * kWidth + row] = W2[i];
  }
  const float* W3 = W2 + kWidth * kWidth;
  float* s3 = s2 + kWidth * kWidth;
  for (int i = threadIdx.x; i < kWidth * kOut; i += blockDim.x) s3[i] = W3[i];
}

// Density MLP: g = Wd2^T relu(Wd1^T feat).
__device__ __forceinline__ void density_f32_smem(const float* __restrict__ s_d, const float feat[kIn],
                                                 float g[kGeo]) {
  const float4* Wd1t = reinterpret_cast<const float4*>(s_d);
  const float4* Wd2 = reinterpret_cast<const float4*>(s_d + kIn * kWidth);
#pragma unroll
  for (int m = 0; m < kGeo; ++m) g[m] = 0.0f;
#pragma unroll 4
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
#pragma unroll
    for (int i4 = 0; i4 < kIn / 4; ++i4) {
      const float4 w = Wd1t[n * (kIn / 4) + i4];
      acc = fmaf(feat[4 * i4 + 0], w.x, acc);
      acc = fmaf(feat[4 * i4 + 1], w.y, acc);
      acc = fmaf(feat[4 * i4 + 2], w.z, acc);
      acc = fmaf(feat[4 * i4 + 3], w.w, acc);
    }
    const float h = fmaxf(acc, 0.0f);
#pragma unroll
    for (int m4 = 0; m4 < kGeo / 4; ++m4) {
      const float4 w = Wd2[n * (kGeo / 4) + m4];
      g[4 * m4 + 0] = fmaf(h, w.x, g[4 * m4 + 0]);
      g[4 * m4 + 1] = fmaf(h, w.y, g[4 * m4 + 1]);
      g[4 * m4 + 2] = fmaf(h, w.z, g[4 * m4 + 2]);
      g[4 * m4 + 3] = fmaf(h, w.w, g[4 * m4 + 3]);
    }
  }
}

// Colour MLP on xc = [g, SH(d)]: o = Wc3^T relu(Wc2^T relu(Wc1^T xc)) (o[0..2]).
__device__ __forceinline__ void color_f32_smem(const float* __restrict__ s_c, const float xc[kColorIn], float o[3]) {
  const float4* Wc1t = reinterpret_cast<const float4*>(s_c);
  const float4* Wc2t = reinterpret_cast<const float4*>(s_c + kColorIn * kWidth);
  const float4* Wc3 = reinterpret_cast<const float4*>(s_c + kColorIn * kWidth + kWidth * kWidth);
  float h1[kWidth];
#pragma unroll
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
#pragma unroll
    for (int i4 = 0; i4 < kColorIn / 4; ++i4) {
      const float4 w = Wc1t[n * (kColorIn / 4) + i4];
      acc = fmaf(xc[4 * i4 + 0], w.x, acc);
      acc = fmaf(xc[4 * i4 + 1], w.y, acc);
      acc = fmaf(xc[4 * i4 + 2], w.z, acc);
      acc = fmaf(xc[4 * i4 + 3], w.w, acc);
    }
    h1[n] = fmaxf(acc, 0.0f);
  }
  float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
#pragma unroll 2
  for (int n = 0; n < kWidth; ++n) {
    float acc = 0.0f;
#pragma unroll
    for (int i4 = 0; i4 < kWidth / 4; ++i4) {
      const float4 w = Wc2t[n * (kWidth / 4) + i4];
      acc = fmaf(h1[4 * i4 + 0], w.x, acc);
      acc = fmaf(h1[4 * i4 + 1], w.y, acc);
      acc = fmaf(h1[4 * i4 + 2], w.z, acc);
      acc = fmaf(h1[4 * i4 + 3], w.w, acc);
    }
    const float h2 = fmaxf(acc, 0.0f);
    const float4 w3 = Wc3[n];
    o0 = fmaf(h2, w3.x, o0);
    o1 = fmaf(h2, w3.y, o1);
    o2 = fmaf(h2, w3.z, o2);
  }
  o[0] = o0;
  o[1] = o1;
  o[2] = o2;
}

// Raw outputs of the split representation: out[0] = g0 (log density),
// out[1..3] = colour logits.
__device__ __forceinline__ void split_f32_smem(const float* __restrict__ s_d, const float* __restrict__ s_c,
                                               const float feat[kIn], const float sh[kSh], float out[kOut]) {
  float xc[kColorIn];
  density_f32_smem(s_d, feat, xc);
#pragma unroll
  for (int j = 0; j < kSh; ++j) xc[kGeo + j] = sh[j];
  float o[3];
  color_f32_smem(s_c, xc, o);
  out[0] = xc[0];
  out[1] = o[0];
  out[2] = o[1];
  out[3] = o[2];
}

}  // namespace nerfxl
