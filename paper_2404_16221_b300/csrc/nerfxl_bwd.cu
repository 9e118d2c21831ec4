// Backward (adjoint) pass of the one-GPU NeRF-XL hot path (arXiv 2404.16221).
//
// The forward keeps only per-ray headers, segments, the region buckets and
// the chunk partials; per-sample activations are recomputed here, never
// stored. Gradients of the loss reach a region's parameters only through
// that region's own samples (Sec. 4.2: each loss lives in a graph that only
// differentiates its local parameters), which on one GPU simply means the
// scatter targets the sample's own region block.
//
//   k_composite_bwd  per ray: reverse of Algorithm 1+2 over the chunk partials
//                    -> adjoints of every chunk partial (tau, C, A, D', L)
//   k_field_bwd_f32  persistent CTAs over the same tiles as the forward:
//                    recompute gather + MLP, chunk-local render adjoint (warp
//                    scans), MLP backward, weight gradients as CTA GEMMs over
//                    the tile's 256 samples (accumulated in shared memory per
//                    region), table gradients by vector atomics.

#include <cuda_runtime.h>

#include <string>

#include "nerfxl_split.cuh"
#include "nerfxl_host.h"

namespace nerfxl {

// ---------------------------------------------------------------------------
// k_composite_bwd. Forward step c (state before it: P_c, A_<c, D_<c):
//   L += P_c^2 L_c + 2 P_c (D_c A_<c - A_c D_<c);  C += P_c C_c;
//   A += P_c A_c;  D += P_c D_c;  P_{c+1} = P_c exp(-tau_c).
// Reverse, with adjoints gC, gA, gD, gL of the accumulators and gP of P_{c+1}:
//   g tau_c = -gP P_{c+1};  gP <- gP exp(-tau_c) + gC.C_c + gA A_c + gD D_c
//                                 + gL (2 P_c L_c + 2 S_c);
//   gC_c = P_c gC;  gA_c = P_c gA - 2 gL P_c D_<c;  gD_c = P_c gD + 2 gL P_c A_<c;
//   gL_c = P_c^2 gL;  then gA += 2 gL P_c D_c, gD -= 2 gL P_c A_c for earlier steps.
// depth = D' + A tn (D' relative to tn), so gA gets gdepth * tn.

__global__ void __launch_bounds__(256) k_composite_bwd(int64_t R, SampParams sp, const RayHdr* __restrict__ hdr,
                                                       const float4* __restrict__ partials,
                                                       const float* __restrict__ d_rgb,
                                                       const float* __restrict__ d_depth,
                                                       const float* __restrict__ d_opacity,
                                                       const float* __restrict__ d_dist, float4* __restrict__ dpart,
                                                       const int32_t* __restrict__ pos,
                                                       float4* __restrict__ dpart_tile) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const RayHdr h = hdr[r];
  const float4* src = partials + 2 * (size_t)r * sp.max_chunk;
  float4* dst = dpart + 2 * (size_t)r * sp.max_chunk;
  // forward sweep: remember P_c, A_<c, D_<c of every chunk (in the adjoint slots)
  float P = 1.0f, tau = 0.0f, comp = 0.0f, A = 0.0f, D = 0.0f;
  for (int c = 0; c < h.nchunk; ++c) {
    const float4 q0 = src[2 * c], q1 = src[2 * c + 1];
    dst[2 * c] = make_float4(P, A, D, 0.0f);
    A += P * q1.x;
    D += P * q1.y;
    const float y = q0.x - comp;
    const float s = tau + y;
    comp = (s - tau) - y;
    tau = s;
    P = expf(-tau);
  }
  float gC0 = d_rgb ? d_rgb[3 * r + 0] : 0.0f;
  float gC1 = d_rgb ? d_rgb[3 * r + 1] : 0.0f;
  float gC2 = d_rgb ? d_rgb[3 * r + 2] : 0.0f;
  const float gdep = d_depth ? d_depth[r] : 0.0f;
  float gA = (d_opacity ? d_opacity[r] : 0.0f) + gdep * h.tn;
  float gD = gdep;
  const float gL = d_dist ? d_dist[r] : 0.0f;
  float gP = 0.0f;        // adjoint of P_{c+1}
  float P_next = P;       // P_{c+1}
  for (int c = h.nchunk - 1; c >= 0; --c) {
    const float4 st = dst[2 * c];
    const float Pc = st.x, Ab = st.y, Db = st.z;
    const float4 q0 = src[2 * c], q1 = src[2 * c + 1];
    const float tc = q0.x, Ac = q1.x, Dc = q1.y, Lc = q1.z;
    const float g_tau = -gP * P_next;
    const float S = Dc * Ab - Ac * Db;
    const float gPc = gP * expf(-tc) + gC0 * q0.y + gC1 * q0.z + gC2 * q0.w + gA * Ac + gD * Dc +
                      gL * (2.0f * Pc * Lc + 2.0f * S);
    const float gAc = Pc * gA - 2.0f * gL * Pc * Db;
    const float gDc = Pc * gD + 2.0f * gL * Pc * Ab;
    const float4 a0 = make_float4(g_tau, Pc * gC0, Pc * gC1, Pc * gC2);
    const float4 a1 = make_float4(gAc, gDc, Pc * Pc * gL, 0.0f);
    dst[2 * c] = a0;
    dst[2 * c + 1] = a1;
    if (dpart_tile) {  // also in the tile order of the tensor-core backward's records
      const size_t at = 2 * (size_t)pos[(size_t)r * sp.max_chunk + c];
      dpart_tile[at] = a0;
      dpart_tile[at + 1] = a1;
    }
    gA += 2.0f * gL * Pc * Dc;
    gD -= 2.0f * gL * Pc * Ac;
    gP = gPc;
    P_next = Pc;
  }
}

// ---------------------------------------------------------------------------
// k_field_bwd_f32

constexpr int kBwdThreads = kChunksPerTile * kWarp;  // 256 samples per tile
constexpr int kActPitch = 68;

struct BwdParams {
  const float* rays_o;
  const float* rays_d;
  FieldPtrs fp;
  const void* tables;  // [K][E] of float2 or half2
  const void* mlp;     // [K][kMlpParams] of fp32, bf16 or fp16
  LevelParams lp;
  SampParams sp;
  int K;
  const RayHdr* hdr;
  const SegDesc* segs;
  const int32_t* base;
  const Slot* chunks;  // slots
  const int32_t* n_tiles;
  const float4* dpart;   // chunk partial adjoints
  const float* rec32;    // the forward's FP32 feature records [tiles][32][256], or NULL (encode again)
  float* grad_tables;    // [K][E][2] accumulated
  float* grad_mlp;       // [K][kMlpParams] accumulated
};


// Scatter dL/dfeat into the region table: entry += corner weight * gfeat.
__device__ __forceinline__ void scatter_table_grad(const LevelParams& lp, float2* __restrict__ gtab, const float u[3],
                                                   const float gfeat[kIn]) {
#pragma unroll
  for (int l = 0; l < kIn / 2; ++l) {
    if (l >= lp.L) break;
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
    float2* gl = gtab + lp.off[l];
    const float g0 = gfeat[2 * l], g1 = gfeat[2 * l + 1];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
      const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
      const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
      const float wyz = (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) * (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
      const float w0 = (1.0f - f[0]) * wyz, w1 = f[0] * wyz;
      if ((i0 ^ i1) == 1u) {
        // both corners in one aligned pair: one 16-byte atomic
        const bool odd = i0 & 1u;
        const float4 v = odd ? make_float4(w1 * g0, w1 * g1, w0 * g0, w0 * g1)
                             : make_float4(w0 * g0, w0 * g1, w1 * g0, w1 * g1);
        atomicAdd(reinterpret_cast<float4*>(gl + (i0 & ~1u)), v);
      } else {
        atomicAdd(gl + i0, make_float2(w0 * g0, w0 * g1));
        atomicAdd(gl + i1, make_float2(w1 * g0, w1 * g1));
      }
    }
  }
}

__device__ __forceinline__ void flush_mlp_grad(const float* __restrict__ s_acc, float* __restrict__ g) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    const float v = s_acc[i];
    if (v != 0.0f) atomicAdd(g + i, v);
  }
}

// The MLP part of the FP32 backward runs as register-tiled GEMMs over the
// 256-sample tile (each thread owns an 8 x 8, 8 x 4 or 4 x 4 block of
// outputs, so a weight or activation read from shared memory feeds 4-8
// multiply-adds). Activations are stored unit-major, A[unit][sample] with a
// pitch of kUPitch floats: a thread's samples are the two float4 groups
// 4 b .. 4 b + 3 and 128 + 4 b .. (b = thread % 32), and unit rows sit 4 banks
// apart, so that both the sample-blocked and the unit-blocked products read
// shared memory without bank conflicts.
constexpr int kUPitch = 260;
constexpr size_t kBwdSmemFloatsT = 2 * (size_t)kMlpParams + (size_t)kUPitch * (kIn + 2 * kWidth + kOut);

// acc[i][j] = sum_k A[k][samples i] B[k][n0 + j]; A unit-major, B row-major [K][64].
template <int K>
__device__ __forceinline__ void tile_gemm_ab(const float* __restrict__ A, const float* __restrict__ B, int sb, int n0,
                                             float acc[8][8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * kUPitch + 4 * sb);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * kUPitch + 128 + 4 * sb);
    const float4 b0 = *reinterpret_cast<const float4*>(B + k * kWidth + n0);
    const float4 b1 = *reinterpret_cast<const float4*>(B + k * kWidth + n0 + 4);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// acc[i][j] = sum_k A[k][samples i] W[j0 + j][k]; W row-major with rows of 64
// (the transposed weight of a dX product), NJ of its rows.
template <int K, int NJ>
__device__ __forceinline__ void tile_gemm_abt(const float* __restrict__ A, const float* __restrict__ W, int sb, int j0,
                                              float acc[8][NJ]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(A + k * kUPitch + 4 * sb);
    const float4 a1 = *reinterpret_cast<const float4*>(A + k * kUPitch + 128 + 4 * sb);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    float b[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) b[j] = W[(j0 + j) * kWidth + k];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// Weight gradient: acc[a][c] = sum_s P[ib + 16 a][s] Q[nb + 16 c][s] over the
// 256 samples (both unit-major).
template <int RA>
__device__ __forceinline__ void tile_gemm_dw(const float* __restrict__ P, const float* __restrict__ Q, int ib, int nb,
                                             float acc[RA][4]) {
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0f;
#pragma unroll 2
  for (int s = 0; s < kBwdThreads; s += 4) {
    float4 pv[RA], qv[4];
#pragma unroll
    for (int a = 0; a < RA; ++a) pv[a] = *reinterpret_cast<const float4*>(P + (ib + 16 * a) * kUPitch + s);
#pragma unroll
    for (int c = 0; c < 4; ++c) qv[c] = *reinterpret_cast<const float4*>(Q + (nb + 16 * c) * kUPitch + s);
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[a][c] = fmaf(pv[a].x, qv[c].x, acc[a][c]);
        acc[a][c] = fmaf(pv[a].y, qv[c].y, acc[a][c]);
        acc[a][c] = fmaf(pv[a].z, qv[c].z, acc[a][c]);
        acc[a][c] = fmaf(pv[a].w, qv[c].w, acc[a][c]);
      }
  }
}

// Stores a thread's 8 x NJ block (samples x units) unit-major, optionally
// through relu or a mask.
template <int NJ>
__device__ __forceinline__ void tile_store(float* __restrict__ A, int sb, int n0, const float acc[8][NJ]) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    float* row = A + (n0 + j) * kUPitch;
    *reinterpret_cast<float4*>(row + 4 * sb) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    *reinterpret_cast<float4*>(row + 128 + 4 * sb) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
  }
}

template <bool kF16Table, int kMlpType>
__global__ void __launch_bounds__(kBwdThreads, 1) k_field_bwd_f32(BwdParams p) {
  extern __shared__ __align__(16) float sm[];
  float* s_w = sm;                             // W1 [32][64], W2 [64][64], W3 [64][4], row-major
  float* s_acc = s_w + kMlpParams;             // gW1 [32][64], gW2 [64][64], gW3 [64][4]
  float* s_F = s_acc + kMlpParams;             // [32][pitch]: features, then dL/dfeatures
  float* s_H1 = s_F + kIn * kUPitch;           // [64][pitch]: h1, then dL/dz1
  float* s_H2 = s_H1 + kWidth * kUPitch;       // [64][pitch]: h2, then dL/dz2
  float* s_Go = s_H2 + kWidth * kUPitch;       // [4][pitch]: dL/d(raw outputs)
  int32_t* s_base = reinterpret_cast<int32_t*>(s_Go + kOut * kUPitch);
  for (int i = threadIdx.x; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  __syncthreads();
  const int n_tiles = *p.n_tiles;
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  const float* W1 = s_w;
  const float* W2 = s_w + kIn * kWidth;
  const float* W3 = W2 + kWidth * kWidth;
  float* gW1 = s_acc;
  float* gW2 = s_acc + kIn * kWidth;
  float* gW3 = gW2 + kWidth * kWidth;
  // this thread's blocks of the tiled products
  const int sb = tid & 31;        // samples 4 sb .. 4 sb + 3 and 128 + 4 sb ..
  const int ub = tid >> 5;        // units 8 ub .. 8 ub + 7 (or features 4 ub .. 4 ub + 3)
  const int ib = tid >> 4, nb = tid & 15;  // weight gradients: rows ib + 16 a, columns nb + 16 c
  int region = -1;
  const void* table = nullptr;
  float2* gtab = nullptr;
  using TabT = typename TableOf<kF16Table>::T;
  const size_t mlp_esize = kMlpType == 0 ? 4 : 2;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int k = region_of_chunk(s_base, p.K, t * kChunksPerTile);
    __syncthreads();  // previous tile's shared buffers fully consumed
    if (k != region) {
      if (region >= 0) flush_mlp_grad(s_acc, p.grad_mlp + (size_t)region * kMlpParams);
      __syncthreads();
      const char* blk = static_cast<const char*>(p.mlp) + (size_t)k * kMlpParams * mlp_esize;
      for (int i = tid; i < kMlpParams; i += blockDim.x) {
        s_w[i] = mlp_elem<kMlpType>(blk, i);
        s_acc[i] = 0.0f;
      }
      __syncthreads();
      region = k;
      table = static_cast<const char*>(p.tables) + (size_t)k * p.lp.E * sizeof(TabT);
      gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
    }
    // ---- per sample (thread = sample s = tid of slot `warp`): position, chunk adjoints, encoding
    const SlotLane sl = slot_lane(p.chunks[t * kChunksPerTile + warp], lane);
    const uint2 ref = sl.ref;
    const bool chunk_ok = sl.slot_ok;  // warp-uniform; lanes of an unused part of the slot are empty samples
    bool valid = false;
    float feat[kIn], u[3];
    float tr = 0.0f, dl = 0.0f;
    float gtc = 0.0f, gC[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f, gD = 0.0f, gL = 0.0f;
#pragma unroll
    for (int q = 0; q < kIn; ++q) feat[q] = 0.0f;
    if (sl.has) {
      const uint32_t ray = ref.x;
      const int seg = ref.y >> 16, c = ref.y & 0xFFFF;
      const RayHdr h = p.hdr[ray];
      const SegDesc sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
      const size_t slot = (size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c;
      const float4 g0 = p.dpart[2 * slot], g1 = p.dpart[2 * slot + 1];
      gtc = g0.x;
      gC[0] = g0.y;
      gC[1] = g0.z;
      gC[2] = g0.w;
      gA = g1.x;
      gD = g1.y;
      gL = g1.z;
      const SegSamples ss = seg_samples(p.sp, sd, ray, seg);
      const int i = c * kWarp + sl.sl;
      valid = i < ss.n;
      if (valid) {
        float o[3], d[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          o[ax] = p.rays_o[3 * (size_t)ray + ax];
          d[ax] = p.rays_d[3 * (size_t)ray + ax];
        }
        float a, b;
        segment_interval(sd, h.tn, h.delta, sample_interval(p.sp, ss, i), a, b);
        const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
        dl = __fsub_rn(b, a);
        tr = __fsub_rn(tbar, h.tn);
        float x[3];
        sample_point(o, d, tbar, x);
        region_coord(p.fp.boxes + 6 * k, x, u);
        if (p.rec32) {  // the forward's features, unit-major like s_F (coalesced)
          const float* rec = p.rec32 + (size_t)t * kIn * kBwdThreads + tid;
#pragma unroll
          for (int j = 0; j < kIn; ++j) feat[j] = __ldcs(rec + j * kBwdThreads);
        } else {
          TableOf<kF16Table>::encode(p.lp, table, u, feat);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kIn; ++j) s_F[j * kUPitch + tid] = feat[j];
    __syncthreads();
    float acc[8][8];
    // ---- forward recompute: H1 = relu(F W1), H2 = relu(H1 W2)
    tile_gemm_ab<kIn>(s_F, W1, sb, 8 * ub, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaxf(acc[i][j], 0.0f);
    tile_store<8>(s_H1, sb, 8 * ub, acc);
    __syncthreads();
    tile_gemm_ab<kWidth>(s_H1, W2, sb, 8 * ub, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaxf(acc[i][j], 0.0f);
    tile_store<8>(s_H2, sb, 8 * ub, acc);
    __syncthreads();
    // ---- per sample: raw outputs o = h2 W3, chunk-local render adjoint -> dL/d(raw outputs)
    float o4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
    for (int n = 0; n < kWidth; ++n) {
      const float h2 = s_H2[n * kUPitch + tid];
      const float4 w3 = *reinterpret_cast<const float4*>(W3 + 4 * n);
      o4[0] = fmaf(h2, w3.x, o4[0]);
      o4[1] = fmaf(h2, w3.y, o4[1]);
      o4[2] = fmaf(h2, w3.z, o4[2]);
      o4[3] = fmaf(h2, w3.w, o4[3]);
    }
    float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
      sigma = expf(o4[0]);
      rgb[0] = 1.0f / (1.0f + expf(-o4[1]));
      rgb[1] = 1.0f / (1.0f + expf(-o4[2]));
      rgb[2] = 1.0f / (1.0f + expf(-o4[3]));
    }
    float g_sigma = 0.0f, g_rgb[3] = {0.0f, 0.0f, 0.0f};
    if (chunk_ok) render_chunk_adjoint(sigma, rgb, tr, dl, sl.sl, gtc, gC, gA, gD, gL, g_sigma, g_rgb, sl.width);
    float go[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (valid) {
      go[0] = g_sigma * sigma;
#pragma unroll
      for (int q = 0; q < 3; ++q) go[1 + q] = g_rgb[q] * rgb[q] * (1.0f - rgb[q]);
    }
#pragma unroll
    for (int m = 0; m < kOut; ++m) s_Go[m * kUPitch + tid] = go[m];
    __syncthreads();
    // ---- gW3[n][m] += sum_s h2[s][n] go[s][m]   (one output per thread)
    {
      const int n = tid >> 2, m = tid & 3;
      float a = 0.0f;
#pragma unroll 4
      for (int s = 0; s < kBwdThreads; s += 4) {
        const float4 hv = *reinterpret_cast<const float4*>(s_H2 + n * kUPitch + s);
        const float4 gv = *reinterpret_cast<const float4*>(s_Go + m * kUPitch + s);
        a = fmaf(hv.x, gv.x, a);
        a = fmaf(hv.y, gv.y, a);
        a = fmaf(hv.z, gv.z, a);
        a = fmaf(hv.w, gv.w, a);
      }
      gW3[n * kOut + m] += a;
    }
    __syncthreads();
    // ---- dL/dz2 = (h2 > 0) (go W3^T), per sample, in place of h2
#pragma unroll 8
    for (int n = 0; n < kWidth; ++n) {
      const float4 w3 = *reinterpret_cast<const float4*>(W3 + 4 * n);
      float* at = s_H2 + n * kUPitch + tid;
      *at = *at > 0.0f ? w3.x * go[0] + w3.y * go[1] + w3.z * go[2] + w3.w * go[3] : 0.0f;
    }
    __syncthreads();
    // ---- gW2[i][n] += sum_s h1[s][i] dz2[s][n]
    {
      float dw[4][4];
      tile_gemm_dw<4>(s_H1, s_H2, ib, nb, dw);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) gW2[(ib + 16 * a) * kWidth + nb + 16 * c] += dw[a][c];
    }
    __syncthreads();
    // ---- dL/dz1 = (h1 > 0) (dz2 W2^T), in place of h1 (each thread reads the h1 it overwrites)
    tile_gemm_abt<kWidth, 8>(s_H2, W2, sb, 8 * ub, acc);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float* row = s_H1 + (8 * ub + j) * kUPitch;
      const float4 h0 = *reinterpret_cast<const float4*>(row + 4 * sb);
      const float4 h1 = *reinterpret_cast<const float4*>(row + 128 + 4 * sb);
      *reinterpret_cast<float4*>(row + 4 * sb) =
          make_float4(h0.x > 0.0f ? acc[0][j] : 0.0f, h0.y > 0.0f ? acc[1][j] : 0.0f, h0.z > 0.0f ? acc[2][j] : 0.0f,
                      h0.w > 0.0f ? acc[3][j] : 0.0f);
      *reinterpret_cast<float4*>(row + 128 + 4 * sb) =
          make_float4(h1.x > 0.0f ? acc[4][j] : 0.0f, h1.y > 0.0f ? acc[5][j] : 0.0f, h1.z > 0.0f ? acc[6][j] : 0.0f,
                      h1.w > 0.0f ? acc[7][j] : 0.0f);
    }
    __syncthreads();
    // ---- gW1[j][n] += sum_s feat[s][j] dz1[s][n]
    {
      float dw[2][4];
      tile_gemm_dw<2>(s_F, s_H1, ib, nb, dw);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) gW1[(ib + 16 * a) * kWidth + nb + 16 * c] += dw[a][c];
    }
    __syncthreads();
    // ---- dL/dfeatures = dz1 W1^T, in place of the features
    {
      float gx[8][4];
      tile_gemm_abt<kWidth, 4>(s_H1, W1, sb, 4 * ub, gx);
      tile_store<4>(s_F, sb, 4 * ub, gx);
    }
    __syncthreads();
    // ---- table gradients (thread = sample)
    if (valid) {
      float gfeat[kIn];
#pragma unroll
      for (int j = 0; j < kIn; ++j) gfeat[j] = s_F[j * kUPitch + tid];
      scatter_table_grad(p.lp, gtab, u, gfeat);
    }
  }
  __syncthreads();
  if (region >= 0) flush_mlp_grad(s_acc, p.grad_mlp + (size_t)region * kMlpParams);
}

// ---------------------------------------------------------------------------
// k_field_bwd_split_f32: the split representation's backward (FP32). Per
// 256-sample tile: recompute encoding, density MLP (g), colour MLP on
// [g, SH(d)]; chunk-local render adjoint; colour MLP backward (its weight
// gradients accumulate in registers over every tile the CTA takes, whatever
// the region, and reach the shared block once at the end); dL/dg0 from the
// density and from the colour MLP; density MLP backward (accumulated per
// region); table scatter. Activations of the tile live in three shared
// buffers that the phases reuse:
//   X [256][36]: xc = [g, SH] and dL/d(colour logits) -> dL/dg
//   B [256][68]: hc1 -> dL/dzc1 -> feat
//   C [256][68]: hc2 -> dL/dzc2 -> h1 -> dL/dz1
// Weight-gradient accumulators per thread (GEMM over the tile's samples):
//   Wc3 [n][m] n = t/4, m = t%4 | Wc2 [i][n0..+15] i = t/4, n0 = 16 (t%4) |
//   Wc1 [j][n0..+7] j = t/8, n0 = 8 (t%8) | Wd2 [n][m0..+3] n = t/4, m0 = 4 (t%4) |
//   Wd1 [j][n0..+7] j = t/8, n0 = 8 (t%8).

constexpr int kSplitXPitch = 36;
constexpr size_t kBwdSplitSmemFloats =
    (size_t)kSplitSmemFloats + (size_t)kBwdThreads * kSplitXPitch + 2 * (size_t)kBwdThreads * kActPitch;

__device__ __forceinline__ void flush_density_grad(float* __restrict__ g, const float aWd1[8], const float aWd2[4],
                                                   int tid) {
  const int j = tid >> 3, n0 = (tid & 7) * 8;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (aWd1[q] != 0.0f) atomicAdd(g + j * kWidth + n0 + q, aWd1[q]);
  const int n = tid >> 2, m0 = (tid & 3) * 4;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (aWd2[q] != 0.0f) atomicAdd(g + kIn * kWidth + n * kGeo + m0 + q, aWd2[q]);
}

// Stage the split weights from FP32, BF16 or FP16 blocks (FP32 in shared memory,
// the layouts of load_density_f32 / load_color_f32).
template <int kMlpType>
__device__ __forceinline__ void load_split_any(const void* dens, const void* color, float* __restrict__ s_d,
                                               float* __restrict__ s_c) {
  if (dens) {
    for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x)
      s_d[(i % kWidth) * kIn + i / kWidth] = mlp_elem<kMlpType>(dens, i);
    for (int i = threadIdx.x; i < kWidth * kGeo; i += blockDim.x)
      s_d[kIn * kWidth + i] = mlp_elem<kMlpType>(dens, kIn * kWidth + i);
  }
  if (color) {
    for (int i = threadIdx.x; i < kColorIn * kWidth; i += blockDim.x)
      s_c[(i % kWidth) * kColorIn + i / kWidth] = mlp_elem<kMlpType>(color, i);
    for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x)
      s_c[kColorIn * kWidth + (i % kWidth) * kWidth + i / kWidth] = mlp_elem<kMlpType>(color, kColorIn * kWidth + i);
    for (int i = threadIdx.x; i < kWidth * kOut; i += blockDim.x)
      s_c[kColorIn * kWidth + kWidth * kWidth + i] = mlp_elem<kMlpType>(color, kColorIn * kWidth + kWidth * kWidth + i);
  }
}

// kF16Table / kMlpType: the parameters the forward read (FP16 tables; the
// host launches the FP32 MLP form, 16-bit MLPs take the tensor-core backward);
// the recompute and every product run in FP32 and the gradients are FP32.
template <bool kF16Table, int kMlpType>
__global__ void __launch_bounds__(kBwdThreads, 1) k_field_bwd_split_f32(BwdParams p) {
  extern __shared__ __align__(16) float sm[];
  float* s_d = sm;                                  // Wd1t [64][32], Wd2 [64][16]
  float* s_c = s_d + kDensityParams;                // Wc1t [64][32], Wc2t [64][64], Wc3 [64][4]
  float* s_X = s_c + kColorParams;                  // [256][36]
  float* s_B = s_X + kBwdThreads * kSplitXPitch;    // [256][68]
  float* s_C = s_B + kBwdThreads * kActPitch;       // [256][68]
  int32_t* s_base = reinterpret_cast<int32_t*>(s_C + kBwdThreads * kActPitch);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  const char* mlp = static_cast<const char*>(p.mlp);
  constexpr size_t kEsize = kMlpType == 0 ? 4 : 2;
  using TabT = typename TableOf<kF16Table>::T;
  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  load_split_any<kMlpType>(nullptr, mlp + (size_t)p.K * kDensityParams * kEsize, s_d, s_c);
  __syncthreads();
  const int n_tiles = *p.n_tiles;
  const float4* Wd1t = reinterpret_cast<const float4*>(s_d);
  const float4* Wd2 = reinterpret_cast<const float4*>(s_d + kIn * kWidth);
  const float4* Wc1t = reinterpret_cast<const float4*>(s_c);
  const float4* Wc2t = reinterpret_cast<const float4*>(s_c + kColorIn * kWidth);
  const float* Wc3 = s_c + kColorIn * kWidth + kWidth * kWidth;
  float* my_X = s_X + tid * kSplitXPitch;
  float* my_B = s_B + tid * kActPitch;
  float* my_C = s_C + tid * kActPitch;
  float aWc3 = 0.0f, aWc2[16], aWc1[8], aWd2[4], aWd1[8];
#pragma unroll
  for (int q = 0; q < 16; ++q) aWc2[q] = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) aWc1[q] = aWd1[q] = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) aWd2[q] = 0.0f;
  int region = -1;
  const TabT* table = nullptr;
  float2* gtab = nullptr;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int k = region_of_chunk(s_base, p.K, t * kChunksPerTile);
    __syncthreads();  // previous tile's shared buffers fully consumed
    if (k != region) {
      if (region >= 0) flush_density_grad(p.grad_mlp + (size_t)region * kDensityParams, aWd1, aWd2, tid);
#pragma unroll
      for (int q = 0; q < 8; ++q) aWd1[q] = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) aWd2[q] = 0.0f;
      load_split_any<kMlpType>(mlp + (size_t)k * kDensityParams * kEsize, nullptr, s_d, s_c);
      __syncthreads();
      region = k;
      table = static_cast<const TabT*>(p.tables) + (size_t)k * p.lp.E;
      gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
    }
    const SlotLane sl = slot_lane(p.chunks[t * kChunksPerTile + warp], lane);
    const uint2 ref = sl.ref;
    const bool chunk_ok = sl.slot_ok;  // warp-uniform; lanes of an unused part of the slot are empty samples
    bool valid = false;
    float feat[kIn], u[3] = {0.0f, 0.0f, 0.0f}, dir[3] = {0.0f, 0.0f, 0.0f};
    float tr = 0.0f, dl = 0.0f;
    float gtc = 0.0f, gC[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f, gD = 0.0f, gL = 0.0f;
#pragma unroll
    for (int q = 0; q < kIn; ++q) feat[q] = 0.0f;
    if (sl.has) {
      const uint32_t ray = ref.x;
      const int seg = ref.y >> 16, c = ref.y & 0xFFFF;
      const RayHdr h = p.hdr[ray];
      const SegDesc sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
      const size_t slot = (size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c;
      const float4 g0 = p.dpart[2 * slot], g1 = p.dpart[2 * slot + 1];
      gtc = g0.x;
      gC[0] = g0.y;
      gC[1] = g0.z;
      gC[2] = g0.w;
      gA = g1.x;
      gD = g1.y;
      gL = g1.z;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) dir[ax] = p.rays_d[3 * (size_t)ray + ax];
      const SegSamples ss = seg_samples(p.sp, sd, ray, seg);
      const int i = c * kWarp + sl.sl;
      valid = i < ss.n;
      if (valid) {
        float o[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) o[ax] = p.rays_o[3 * (size_t)ray + ax];
        float a, b;
        segment_interval(sd, h.tn, h.delta, sample_interval(p.sp, ss, i), a, b);
        const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
        dl = __fsub_rn(b, a);
        tr = __fsub_rn(tbar, h.tn);
        float x[3];
        sample_point(o, dir, tbar, x);
        region_coord(p.fp.boxes + 6 * k, x, u);
        TableOf<kF16Table>::encode(p.lp, table, u, feat);
      }
    }
    // ---- forward recompute: g, xc -> X; hc1 -> B; hc2 -> C; colour logits
    float xc[kColorIn];
    density_f32_smem(s_d, feat, xc);
    sh4_f32(dir, xc + kGeo);
#pragma unroll
    for (int q = 0; q < kColorIn; q += 4)
      *reinterpret_cast<float4*>(my_X + q) = make_float4(xc[q], xc[q + 1], xc[q + 2], xc[q + 3]);
    {
      float hc1[kWidth];
#pragma unroll
      for (int n = 0; n < kWidth; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int i4 = 0; i4 < kColorIn / 4; ++i4) {
          const float4 w = Wc1t[n * (kColorIn / 4) + i4];
          acc = fmaf(xc[4 * i4], w.x, acc);
          acc = fmaf(xc[4 * i4 + 1], w.y, acc);
          acc = fmaf(xc[4 * i4 + 2], w.z, acc);
          acc = fmaf(xc[4 * i4 + 3], w.w, acc);
        }
        hc1[n] = fmaxf(acc, 0.0f);
      }
#pragma unroll
      for (int q = 0; q < kWidth; q += 4)
        *reinterpret_cast<float4*>(my_B + q) = make_float4(hc1[q], hc1[q + 1], hc1[q + 2], hc1[q + 3]);
    }
    float oc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 2
    for (int n = 0; n < kWidth; ++n) {
      float acc = 0.0f;
#pragma unroll
      for (int i4 = 0; i4 < kWidth / 4; ++i4) {
        const float4 w = Wc2t[n * (kWidth / 4) + i4];
        const float4 hv = *reinterpret_cast<const float4*>(my_B + 4 * i4);
        acc = fmaf(hv.x, w.x, acc);
        acc = fmaf(hv.y, w.y, acc);
        acc = fmaf(hv.z, w.z, acc);
        acc = fmaf(hv.w, w.w, acc);
      }
      const float h2 = fmaxf(acc, 0.0f);
      my_C[n] = h2;
#pragma unroll
      for (int m = 0; m < 3; ++m) oc[m] = fmaf(h2, Wc3[n * kOut + m], oc[m]);
    }
    // ---- chunk-local render adjoint -> dL/dg0 (density) and dL/d(colour logits)
    float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
      sigma = expf(xc[0]);
#pragma unroll
      for (int m = 0; m < 3; ++m) rgb[m] = 1.0f / (1.0f + expf(-oc[m]));
    }
    float g_sigma = 0.0f, g_rgb[3] = {0.0f, 0.0f, 0.0f};
    if (chunk_ok) render_chunk_adjoint(sigma, rgb, tr, dl, sl.sl, gtc, gC, gA, gD, gL, g_sigma, g_rgb, sl.width);
    const float go_d = valid ? g_sigma * sigma : 0.0f;
    float go[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
#pragma unroll
      for (int m = 0; m < 3; ++m) go[m] = g_rgb[m] * rgb[m] * (1.0f - rgb[m]);
    }
    *reinterpret_cast<float4*>(my_X + kColorIn) = make_float4(go[0], go[1], go[2], 0.0f);
    __syncthreads();
    // ---- Wc3[n][m] += sum_s hc2[s][n] go[s][m]
    {
      const int n = tid >> 2, m = tid & 3;
      float acc = 0.0f;
      for (int s = 0; s < kBwdThreads; ++s) acc = fmaf(s_C[s * kActPitch + n], s_X[s * kSplitXPitch + kColorIn + m], acc);
      aWc3 += acc;
    }
    // ---- dL/dzc2 = (hc2 > 0) Wc3 go, in place in the own C row once everyone has read C
    __syncthreads();
#pragma unroll 4
    for (int n = 0; n < kWidth; ++n) {
      const float h = my_C[n];
      my_C[n] = h > 0.0f ? Wc3[n * kOut] * go[0] + Wc3[n * kOut + 1] * go[1] + Wc3[n * kOut + 2] * go[2] : 0.0f;
    }
    __syncthreads();
    // ---- Wc2[i][n] += sum_s hc1[s][i] dzc2[s][n]
    {
      const int i = tid >> 2, n0 = (tid & 3) * 16;
      for (int s = 0; s < kBwdThreads; ++s) {
        const float hv = s_B[s * kActPitch + i];
        const float4* qr = reinterpret_cast<const float4*>(s_C + s * kActPitch + n0);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 v = qr[q4];
          aWc2[4 * q4] = fmaf(hv, v.x, aWc2[4 * q4]);
          aWc2[4 * q4 + 1] = fmaf(hv, v.y, aWc2[4 * q4 + 1]);
          aWc2[4 * q4 + 2] = fmaf(hv, v.z, aWc2[4 * q4 + 2]);
          aWc2[4 * q4 + 3] = fmaf(hv, v.w, aWc2[4 * q4 + 3]);
        }
      }
    }
    // ---- dL/dzc1 = (hc1 > 0) Wc2 dzc2   (Wc2[i][n] = Wc2t[n][i]; dzc2 read from the own C row)
    float gz1c[kWidth];
#pragma unroll
    for (int i = 0; i < kWidth; ++i) gz1c[i] = 0.0f;
#pragma unroll 1
    for (int n = 0; n < kWidth; ++n) {
      const float gzn = my_C[n];
#pragma unroll
      for (int i4 = 0; i4 < kWidth / 4; ++i4) {
        const float4 w = Wc2t[n * (kWidth / 4) + i4];
        gz1c[4 * i4] = fmaf(w.x, gzn, gz1c[4 * i4]);
        gz1c[4 * i4 + 1] = fmaf(w.y, gzn, gz1c[4 * i4 + 1]);
        gz1c[4 * i4 + 2] = fmaf(w.z, gzn, gz1c[4 * i4 + 2]);
        gz1c[4 * i4 + 3] = fmaf(w.w, gzn, gz1c[4 * i4 + 3]);
      }
    }
#pragma unroll
    for (int q = 0; q < kWidth; q += 4) {
      const float4 hv = *reinterpret_cast<const float4*>(my_B + q);
      gz1c[q] = hv.x > 0.0f ? gz1c[q] : 0.0f;
      gz1c[q + 1] = hv.y > 0.0f ? gz1c[q + 1] : 0.0f;
      gz1c[q + 2] = hv.z > 0.0f ? gz1c[q + 2] : 0.0f;
      gz1c[q + 3] = hv.w > 0.0f ? gz1c[q + 3] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kWidth; q += 4)
      *reinterpret_cast<float4*>(my_B + q) = make_float4(gz1c[q], gz1c[q + 1], gz1c[q + 2], gz1c[q + 3]);
    __syncthreads();
    // ---- Wc1[j][n] += sum_s xc[s][j] dzc1[s][n]
    {
      const int j = tid >> 3, n0 = (tid & 7) * 8;
      for (int s = 0; s < kBwdThreads; ++s) {
        const float xv = s_X[s * kSplitXPitch + j];
        const float4* qr = reinterpret_cast<const float4*>(s_B + s * kActPitch + n0);
#pragma unroll
        for (int q4 = 0; q4 < 2; ++q4) {
          const float4 v = qr[q4];
          aWc1[4 * q4] = fmaf(xv, v.x, aWc1[4 * q4]);
          aWc1[4 * q4 + 1] = fmaf(xv, v.y, aWc1[4 * q4 + 1]);
          aWc1[4 * q4 + 2] = fmaf(xv, v.z, aWc1[4 * q4 + 2]);
          aWc1[4 * q4 + 3] = fmaf(xv, v.w, aWc1[4 * q4 + 3]);
        }
      }
    }
    // ---- dL/dg = (Wc1 dzc1)[0..15] + dL/dg0 from the density (dzc1 read from the own B row)
    float gg[kGeo];
#pragma unroll
    for (int m = 0; m < kGeo; ++m) gg[m] = 0.0f;
#pragma unroll 1
    for (int n = 0; n < kWidth; ++n) {
      const float gzn = my_B[n];
#pragma unroll
      for (int m4 = 0; m4 < kGeo / 4; ++m4) {
        const float4 w = Wc1t[n * (kColorIn / 4) + m4];  // Wc1[4 m4 + j][n]
        gg[4 * m4] = fmaf(w.x, gzn, gg[4 * m4]);
        gg[4 * m4 + 1] = fmaf(w.y, gzn, gg[4 * m4 + 1]);
        gg[4 * m4 + 2] = fmaf(w.z, gzn, gg[4 * m4 + 2]);
        gg[4 * m4 + 3] = fmaf(w.w, gzn, gg[4 * m4 + 3]);
      }
    }
    gg[0] += go_d;
    // ---- recompute h1 of the density MLP into the own C row (after everyone read B and X)
    __syncthreads();
#pragma unroll 4
    for (int n = 0; n < kWidth; ++n) {
      float acc = 0.0f;
#pragma unroll
      for (int i4 = 0; i4 < kIn / 4; ++i4) {
        const float4 w = Wd1t[n * (kIn / 4) + i4];
        acc = fmaf(feat[4 * i4], w.x, acc);
        acc = fmaf(feat[4 * i4 + 1], w.y, acc);
        acc = fmaf(feat[4 * i4 + 2], w.z, acc);
        acc = fmaf(feat[4 * i4 + 3], w.w, acc);
      }
      my_C[n] = fmaxf(acc, 0.0f);
    }
#pragma unroll
    for (int q = 0; q < kGeo; q += 4)
      *reinterpret_cast<float4*>(my_X + q) = make_float4(gg[q], gg[q + 1], gg[q + 2], gg[q + 3]);
    __syncthreads();
    // ---- Wd2[n][m] += sum_s h1[s][n] dg[s][m]
    {
      const int n = tid >> 2, m0 = (tid & 3) * 4;
      for (int s = 0; s < kBwdThreads; ++s) {
        const float hv = s_C[s * kActPitch + n];
        const float4 v = *reinterpret_cast<const float4*>(s_X + s * kSplitXPitch + m0);
        aWd2[0] = fmaf(hv, v.x, aWd2[0]);
        aWd2[1] = fmaf(hv, v.y, aWd2[1]);
        aWd2[2] = fmaf(hv, v.z, aWd2[2]);
        aWd2[3] = fmaf(hv, v.w, aWd2[3]);
      }
    }
    // ---- dL/dz1 = (h1 > 0) Wd2 dg, in place in the own C row once everyone has read C; feat -> B
    __syncthreads();
#pragma unroll 4
    for (int n = 0; n < kWidth; ++n) {
      float acc = 0.0f;
#pragma unroll
      for (int m4 = 0; m4 < kGeo / 4; ++m4) {
        const float4 w = Wd2[n * (kGeo / 4) + m4];
        acc = fmaf(w.x, gg[4 * m4], acc);
        acc = fmaf(w.y, gg[4 * m4 + 1], acc);
        acc = fmaf(w.z, gg[4 * m4 + 2], acc);
        acc = fmaf(w.w, gg[4 * m4 + 3], acc);
      }
      my_C[n] = my_C[n] > 0.0f ? acc : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kIn; q += 4)
      *reinterpret_cast<float4*>(my_B + q) = make_float4(feat[q], feat[q + 1], feat[q + 2], feat[q + 3]);
    __syncthreads();
    // ---- Wd1[j][n] += sum_s feat[s][j] dz1[s][n]
    {
      const int j = tid >> 3, n0 = (tid & 7) * 8;
      for (int s = 0; s < kBwdThreads; ++s) {
        const float fv = s_B[s * kActPitch + j];
        const float4* qr = reinterpret_cast<const float4*>(s_C + s * kActPitch + n0);
#pragma unroll
        for (int q4 = 0; q4 < 2; ++q4) {
          const float4 v = qr[q4];
          aWd1[4 * q4] = fmaf(fv, v.x, aWd1[4 * q4]);
          aWd1[4 * q4 + 1] = fmaf(fv, v.y, aWd1[4 * q4 + 1]);
          aWd1[4 * q4 + 2] = fmaf(fv, v.z, aWd1[4 * q4 + 2]);
          aWd1[4 * q4 + 3] = fmaf(fv, v.w, aWd1[4 * q4 + 3]);
        }
      }
    }
    // ---- dL/dfeat = Wd1 dz1 (dz1 from the own C row), then the table scatter
    if (valid) {
      float gfeat[kIn];
#pragma unroll
      for (int j = 0; j < kIn; ++j) gfeat[j] = 0.0f;
#pragma unroll 1
      for (int n = 0; n < kWidth; ++n) {
        const float gzn = my_C[n];
#pragma unroll
        for (int i4 = 0; i4 < kIn / 4; ++i4) {
          const float4 w = Wd1t[n * (kIn / 4) + i4];
          gfeat[4 * i4] = fmaf(w.x, gzn, gfeat[4 * i4]);
          gfeat[4 * i4 + 1] = fmaf(w.y, gzn, gfeat[4 * i4 + 1]);
          gfeat[4 * i4 + 2] = fmaf(w.z, gzn, gfeat[4 * i4 + 2]);
          gfeat[4 * i4 + 3] = fmaf(w.w, gzn, gfeat[4 * i4 + 3]);
        }
      }
      scatter_table_grad(p.lp, gtab, u, gfeat);
    }
  }
  if (region >= 0) flush_density_grad(p.grad_mlp + (size_t)region * kDensityParams, aWd1, aWd2, tid);
  // the shared colour block: once per CTA
  float* gc = p.grad_mlp + (size_t)p.K * kDensityParams;
  {
    const int n = tid >> 2, m = tid & 3;
    if (aWc3 != 0.0f) atomicAdd(gc + kColorIn * kWidth + kWidth * kWidth + n * kOut + m, aWc3);
    const int i = tid >> 2, n0 = (tid & 3) * 16;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (aWc2[q] != 0.0f) atomicAdd(gc + kColorIn * kWidth + i * kWidth + n0 + q, aWc2[q]);
    const int j = tid >> 3, m0 = (tid & 7) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (aWc1[q] != 0.0f) atomicAdd(gc + j * kWidth + m0 + q, aWc1[q]);
  }
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_render_bwd(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                           const float* rays_o, const float* rays_d, const float* d_rgb,
                                           const float* d_depth, const float* d_opacity, const float* d_dist,
                                           float* grad_tables, float* grad_mlp, void* workspace, size_t ws_bytes,
                                           cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  if (s->flags & NERFXL_SAMPLE_COMPOSITE)
    return set_error(NERFXL_E_UNSUPPORTED, "sample-level composition is forward only");

  const bool f16tab = f->table_dtype == NERFXL_F16;
  if (!(f->table_dtype == NERFXL_F32 || f16tab) ||
      !(f->mlp_dtype == NERFXL_F32 || f->mlp_dtype == NERFXL_BF16 || f->mlp_dtype == NERFXL_F16))
    return set_error(NERFXL_E_UNSUPPORTED, "backward reads FP32/FP16 tables and an FP32/BF16/FP16 MLP");
  if (n_rays > 0 && (!rays_o || !rays_d || !grad_tables || !grad_mlp))
    return set_error(NERFXL_E_INVALID, "null ray or gradient pointer");
  const Layout L = layout(f, s, n_rays, 1);
  if (!workspace || ws_bytes < L.total)
    return set_error(NERFXL_E_WORKSPACE, "backward needs the forward's workspace sized with for_backward=1");
  if (n_rays == 0) return NERFXL_OK;
  char* ws = static_cast<char*>(workspace);
  const SampParams sp = samp_params(f, s, ws, L);
  float4* dpart = reinterpret_cast<float4*>(ws + L.dpartials);
  // the 16-bit forms of both representations run the tensor-core backward
  // from per-tile records; FP32 MLPs recompute on CUDA cores
  const bool tc = f->mlp_dtype == NERFXL_BF16 || f->mlp_dtype == NERFXL_F16;
  if (f->mlp_dtype == NERFXL_E4M3) return set_error(NERFXL_E_UNSUPPORTED, "the E4M3 MLP is forward-only");
  if (tc && !(s->flags & NERFXL_SAVE_FEATURES)) {
    // The forward did not keep the records: rebuild them (the forward's
    // partials are rewritten with identical values).
    st = launch_field_fwd_tc(f, sp, level_params(f), rays_o, rays_d, ws, L, record_out(ws, L), stream);
    if (st != NERFXL_OK) return st;
  }
  k_composite_bwd<<<(int)((n_rays + 255) / 256), 256, 0, stream>>>(
      n_rays, sp, reinterpret_cast<const RayHdr*>(ws + L.ray_hdr), reinterpret_cast<const float4*>(ws + L.partials),
      d_rgb, d_depth, d_opacity, d_dist, dpart, tc ? reinterpret_cast<const int32_t*>(ws + L.rec_pos) : nullptr,
      tc ? reinterpret_cast<float4*>(ws + L.rec_dpart) : nullptr);
  st = kernel_launched("k_composite_bwd");
  if (st != NERFXL_OK) return st;
  if (tc && f->arch == NERFXL_ARCH_SPLIT)
    return launch_field_bwd_split_tc(f, level_params(f), ws, L, grad_tables, grad_mlp, stream);
  if (tc) return launch_field_bwd_tc(f, level_params(f), ws, L, grad_tables, grad_mlp, stream);
  BwdParams p;
  p.rays_o = rays_o;
  p.rays_d = rays_d;
  p.fp.boxes = f->boxes;
  p.fp.tables = nullptr;
  p.fp.mlp = nullptr;
  p.tables = f->tables;
  p.mlp = f->mlp;
  p.lp = level_params(f);
  p.sp = sp;
  p.K = f->K;
  p.hdr = reinterpret_cast<const RayHdr*>(ws + L.ray_hdr);
  p.segs = reinterpret_cast<const SegDesc*>(ws + L.segs);
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.chunks = reinterpret_cast<const Slot*>(ws + L.chunks);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.dpart = dpart;
  p.rec32 = (s->flags & NERFXL_SAVE_FEATURES) && L.rec32 ? reinterpret_cast<const float*>(ws + L.rec32) : nullptr;
  p.grad_tables = grad_tables;
  p.grad_mlp = grad_mlp;
  if (f->arch == NERFXL_ARCH_SPLIT) {
    const size_t smem_s = sizeof(float) * kBwdSplitSmemFloats + sizeof(int32_t) * (f->K + 1);
    if (smem_s > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
    void (*ks)(BwdParams) = f16tab ? k_field_bwd_split_f32<true, 0> : k_field_bwd_split_f32<false, 0>;  // FP32 MLP
    if (cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448) != cudaSuccess)
      return launch_check("k_field_bwd_split_f32 smem attribute");
    const int grid = fwd_grid(L.chunk_cap / kChunksPerTile, 1);
    profile_mark(0, stream);
    ks<<<grid, kBwdThreads, smem_s, stream>>>(p);
    profile_mark(1, stream);
    return kernel_launched("k_field_bwd_split_f32");
  }
  const size_t smem = sizeof(float) * kBwdSmemFloatsT + sizeof(int32_t) * (f->K + 1);
  if (f16tab) return set_error(NERFXL_E_UNSUPPORTED, "FP16 tables go with a 16-bit MLP");
  if (smem > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
  void (*kern)(BwdParams) = k_field_bwd_f32<false, 0>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448) != cudaSuccess)
    return launch_check("k_field_bwd_f32 smem attribute");
  const int grid = fwd_grid(L.chunk_cap / kChunksPerTile, 1);
  profile_mark(0, stream);
  kern<<<grid, kBwdThreads, smem, stream>>>(p);
  profile_mark(1, stream);
  return kernel_launched("k_field_bwd_f32");
}
