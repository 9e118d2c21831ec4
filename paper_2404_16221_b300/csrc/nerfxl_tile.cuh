// Register-tiled FP32 products over a tile of samples held unit-major in
// shared memory: A[unit][sample] with a row pitch of P floats (P = samples +
// 4, so unit rows sit 4 banks apart). A thread owns the 8 samples 4 sb ..
// 4 sb + 3 and H + 4 sb .. H + 4 sb + 3 (H = half the tile) and a block of
// units, so that each value read from shared memory feeds several
// multiply-adds, and both the sample-blocked and the unit-blocked reads are
// free of bank conflicts. Every output accumulates over its k in order with
// fused multiply-adds from zero, the order of a per-sample dot product.
#pragma once

namespace nerfxl {

// acc[i][j] = sum_k A[k][samples i] B[k][n0 + j]; B row-major [K][NB].
template <int P, int H, int K, int NJ, int NB>
__device__ __forceinline__ void tile_ab(const float* __restrict__ A, const float* __restrict__ B, int sb, int n0,
                                        float acc[8][NJ]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * P + 4 * sb);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * P + H + 4 * sb);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float b[NJ];
    if (NJ % 4 == 0) {
#pragma unroll
      for (int j4 = 0; j4 < NJ / 4; ++j4) {
        const float4 bv = *reinterpret_cast<const float4*>(B + k * NB + n0 + 4 * j4);
        b[4 * j4] = bv.x;
        b[4 * j4 + 1] = bv.y;
        b[4 * j4 + 2] = bv.z;
        b[4 * j4 + 3] = bv.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) b[j] = B[k * NB + n0 + j];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// acc[i][j] = sum_k A[k][samples i] W[j0 + j][k]; W row-major with rows of WS
// (the transposed weight of a dX product), NJ of its rows.
template <int P, int H, int K, int NJ, int WS>
__device__ __forceinline__ void tile_abt(const float* __restrict__ A, const float* __restrict__ W, int sb, int j0,
                                         float acc[8][NJ]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * P + 4 * sb);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * P + H + 4 * sb);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float b[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) b[j] = W[(j0 + j) * WS + k];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// Weight gradient: acc[a][c] = sum_s Pm[ib + 16 a][s] Q[nb + 16 c][s] over the
// tile's T samples (both unit-major).
template <int P, int T, int RA, int RC>
__device__ __forceinline__ void tile_dw(const float* __restrict__ Pm, const float* __restrict__ Q, int ib, int nb,
                                        float acc[RA][RC]) {
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[a][c] = 0.0f;
#pragma unroll 2
  for (int s = 0; s < T; s += 4) {
    float4 pv[RA], qv[RC];
#pragma unroll
    for (int a = 0; a < RA; ++a) pv[a] = *reinterpret_cast<const float4*>(Pm + (ib + 16 * a) * P + s);
#pragma unroll
    for (int c = 0; c < RC; ++c) qv[c] = *reinterpret_cast<const float4*>(Q + (nb + 16 * c) * P + s);
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        acc[a][c] = fmaf(pv[a].x, qv[c].x, acc[a][c]);
        acc[a][c] = fmaf(pv[a].y, qv[c].y, acc[a][c]);
        acc[a][c] = fmaf(pv[a].z, qv[c].z, acc[a][c]);
        acc[a][c] = fmaf(pv[a].w, qv[c].w, acc[a][c]);
      }
  }
}

// Stores a thread's 8 x NJ block (samples x units) unit-major.
template <int P, int H, int NJ>
__device__ __forceinline__ void tile_st(float* __restrict__ A, int sb, int n0, const float acc[8][NJ]) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    float* row = A + (n0 + j) * P;
    *reinterpret_cast<float4*>(row + 4 * sb) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    *reinterpret_cast<float4*>(row + H + 4 * sb) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
  }
}

template <int NI, int NJ>
__device__ __forceinline__ void tile_relu(float acc[NI][NJ]) {
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = fmaxf(acc[i][j], 0.0f);
}

}  // namespace nerfxl
