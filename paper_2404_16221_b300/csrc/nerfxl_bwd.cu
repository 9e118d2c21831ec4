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
#include "nerfxl_scatter.cuh"
#include "nerfxl_tile.cuh"

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
  float* rec32;          // FP32 feature records [tiles][32][256], or NULL (encode again)
  int rec_in;            // rec32 holds the forward's records (else the split backward writes them)
  float* grad_tables;    // [K][E][2] accumulated
  float* grad_mlp;       // [K][kMlpParams] accumulated
};


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
// The scatter's inputs kept per tile row: region coordinates [3][256] and
// one valid-sample mask per chunk slot [8].
constexpr size_t kScatterSmemFloats = 3 * (size_t)kBwdThreads + kChunksPerTile;
constexpr size_t kBwdSmemFloatsT =
    2 * (size_t)kMlpParams + (size_t)kUPitch * (kIn + 2 * kWidth + kOut) + kScatterSmemFloats;

template <int K, int NJ = 8, int NB = kWidth>
__device__ __forceinline__ void tile_gemm_ab(const float* A, const float* B, int sb, int n0, float acc[8][NJ]) {
  tile_ab<kUPitch, kBwdThreads / 2, K, NJ, NB>(A, B, sb, n0, acc);
}
template <int K, int NJ, int WS = kWidth>
__device__ __forceinline__ void tile_gemm_abt(const float* A, const float* W, int sb, int j0, float acc[8][NJ]) {
  tile_abt<kUPitch, kBwdThreads / 2, K, NJ, WS>(A, W, sb, j0, acc);
}
template <int RA, int RC = 4>
__device__ __forceinline__ void tile_gemm_dw(const float* P, const float* Q, int ib, int nb, float acc[RA][RC]) {
  tile_dw<kUPitch, kBwdThreads, RA, RC>(P, Q, ib, nb, acc);
}
template <int NJ>
__device__ __forceinline__ void tile_store(float* A, int sb, int n0, const float acc[8][NJ]) {
  tile_st<kUPitch, kBwdThreads / 2, NJ>(A, sb, n0, acc);
}

// The scatter's per-row inputs: region coordinates (unit-major) and the
// slot's valid-sample mask (thread = row; called by every thread).
__device__ __forceinline__ void keep_scatter_inputs(float* __restrict__ s_U, uint32_t* __restrict__ s_V,
                                                    const float u[3], bool valid, int warp, int lane, int tid) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) s_U[ax * kBwdThreads + tid] = u[ax];
  const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
  if (lane == 0) s_V[warp] = vm;
}

// Table gradients of a tile from dL/dfeatures (unit-major, kUPitch): warp w
// takes windows w and w + 8 (rows 16 v .. 16 v + 15 of window v), one after
// the other; lane pair l (lanes 2l, 2l + 1) takes level l of the window, one
// lane per x-half of the cell corners, merging runs of samples in the same
// cell. All lanes of a warp read the same row of u (a broadcast).

__device__ __forceinline__ void scatter_tile(const LevelParams& lp, float2* __restrict__ gtab,
                                             const float* __restrict__ s_U, const uint32_t* __restrict__ s_V,
                                             const float* __restrict__ s_G, int tid) {
  const int warp = tid / kWarp, lane = tid % kWarp;
  const int l = lane >> 1, h = lane & 1;
  if (l >= lp.L) return;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int w = warp + 8 * j;
    const uint32_t vm = (s_V[w >> 1] >> (16 * (w & 1))) & 0xFFFFu;
    if (vm == 0u) continue;
    const int r0 = 16 * w;
    scatter_runs_half<16, false>(
        lp, gtab, l, h, vm,
        [&](int i, float* ui) {
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) ui[ax] = s_U[ax * kBwdThreads + r0 + i];
        },
        [&](int i) { return make_float2(s_G[2 * l * kUPitch + r0 + i], s_G[(2 * l + 1) * kUPitch + r0 + i]); });
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
  float* s_U = s_Go + kOut * kUPitch;                       // [3][256] region coordinates
  uint32_t* s_V = reinterpret_cast<uint32_t*>(s_U + 3 * kBwdThreads);  // [8] valid samples per slot
  int32_t* s_base = reinterpret_cast<int32_t*>(s_V + kChunksPerTile);
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
    keep_scatter_inputs(s_U, s_V, u, valid, warp, lane, tid);
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
    // ---- table gradients: thread (window, level) takes one level of 16 consecutive rows
    scatter_tile(p.lp, gtab, s_U, s_V, s_F, tid);
  }
  __syncthreads();
  if (region >= 0) flush_mlp_grad(s_acc, p.grad_mlp + (size_t)region * kMlpParams);
}

// ---------------------------------------------------------------------------
// k_field_bwd_split_f32: the split representation's backward (FP32), as
// register-tiled GEMMs over the 256-sample tile like k_field_bwd_f32. Per
// tile: the features (the forward's FP32 records; encoded and recorded here
// when the forward kept none), the density MLP (g), the colour MLP on
// [g, SH(d)], the chunk-local render adjoint, the colour MLP backward, dL/dg
// (through the colour MLP and, for g0, through the density), the density MLP
// backward with h1 recomputed from the features read back, and the table
// scatter. Four unit-major buffers of kUPitch-float rows serve the phases:
//   A [64]: h1 -> hc2 -> dL/dzc2 -> h1 -> dL/dz1
//   C [32]: xc = [g, SH(d)] -> dL/dg (rows 0..15)
//   D [64]: features -> hc1 -> dL/dzc1 -> features -> dL/dfeatures
//   O [4]:  dL/d(colour logits) (rows 0..2), dL/dg0 through the density (row 3)
// Weight gradients accumulate in registers (a thread owns rows ib + 16 a and
// columns nb + 16 c of each matrix): the shared colour MLP's over every tile
// the CTA takes, flushed once at the end; the density MLP's per region.

constexpr size_t kBwdSplitSmemFloats =
    (size_t)kSplitSmemFloats + (size_t)kUPitch * (2 * kWidth + kColorIn + kOut) + kScatterSmemFloats;

__device__ __forceinline__ void flush_density_grad(float* __restrict__ g, const float aWd1[2][4],
                                                   const float aWd2[4][1], int ib, int nb) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (aWd1[a][c] != 0.0f) atomicAdd(g + (ib + 16 * a) * kWidth + nb + 16 * c, aWd1[a][c]);
#pragma unroll
  for (int a = 0; a < 4; ++a)
    if (aWd2[a][0] != 0.0f) atomicAdd(g + kIn * kWidth + (ib + 16 * a) * kGeo + nb, aWd2[a][0]);
}

// Overwrites a thread's 8 x 8 block of A (samples 4 sb.., 128 + 4 sb..; units
// n0..n0 + 7) with acc where A is positive and 0 elsewhere: the gradient
// through a ReLU whose output A holds.
__device__ __forceinline__ void tile_store_masked(float* __restrict__ A, int sb, int n0, const float acc[8][8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float* row = A + (n0 + j) * kUPitch;
    const float4 h0 = *reinterpret_cast<const float4*>(row + 4 * sb);
    const float4 h1 = *reinterpret_cast<const float4*>(row + 128 + 4 * sb);
    *reinterpret_cast<float4*>(row + 4 * sb) =
        make_float4(h0.x > 0.0f ? acc[0][j] : 0.0f, h0.y > 0.0f ? acc[1][j] : 0.0f, h0.z > 0.0f ? acc[2][j] : 0.0f,
                    h0.w > 0.0f ? acc[3][j] : 0.0f);
    *reinterpret_cast<float4*>(row + 128 + 4 * sb) =
        make_float4(h1.x > 0.0f ? acc[4][j] : 0.0f, h1.y > 0.0f ? acc[5][j] : 0.0f, h1.z > 0.0f ? acc[6][j] : 0.0f,
                    h1.w > 0.0f ? acc[7][j] : 0.0f);
  }
}

template <int RA, int RC>
__device__ __forceinline__ void add_block(float acc[RA][RC], const float dw[RA][RC]) {
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[a][c] += dw[a][c];
}

// kF16Table / kMlpType: the parameters the forward read (the host launches
// the FP32 MLP form; 16-bit MLPs take the tensor-core backward); the
// recompute and every product run in FP32 and the gradients are FP32.
template <bool kF16Table, int kMlpType>
__global__ void __launch_bounds__(kBwdThreads, 1) k_field_bwd_split_f32(BwdParams p) {
  extern __shared__ __align__(16) float sm[];
  float* s_w = sm;  // Wd1 [32][64], Wd2 [64][16] | Wc1 [32][64], Wc2 [64][64], Wc3 [64][4], row-major
  float* s_A = s_w + kSplitSmemFloats;
  float* s_C = s_A + kWidth * kUPitch;
  float* s_D = s_C + kColorIn * kUPitch;
  float* s_O = s_D + kWidth * kUPitch;
  float* s_U = s_O + kOut * kUPitch;                        // [3][256] region coordinates
  uint32_t* s_V = reinterpret_cast<uint32_t*>(s_U + 3 * kBwdThreads);  // [8] valid samples per slot
  int32_t* s_base = reinterpret_cast<int32_t*>(s_V + kChunksPerTile);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  const char* mlp = static_cast<const char*>(p.mlp);
  constexpr size_t kEsize = kMlpType == 0 ? 4 : 2;
  using TabT = typename TableOf<kF16Table>::T;
  const float* Wd1 = s_w;
  const float* Wd2 = s_w + kIn * kWidth;
  const float* Wc1 = s_w + kDensityParams;
  const float* Wc2 = Wc1 + kColorIn * kWidth;
  const float* Wc3 = Wc2 + kWidth * kWidth;
  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  {
    const char* cblk = mlp + (size_t)p.K * kDensityParams * kEsize;
    for (int i = tid; i < kColorParams; i += blockDim.x) s_w[kDensityParams + i] = mlp_elem<kMlpType>(cblk, i);
  }
  __syncthreads();
  const int n_tiles = *p.n_tiles;
  const int sb = tid & 31, ub = tid >> 5;  // GEMM blocks: samples 4 sb.., 128 + 4 sb..; units of block ub
  const int ib = tid >> 4, nb = tid & 15;  // weight gradients: rows ib + 16 a, columns nb + 16 c
  float aWc3 = 0.0f, aWc2[4][4], aWc1[2][4], aWd2[4][1], aWd1[2][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    aWd2[a][0] = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) aWc2[a][c] = 0.0f;
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) aWc1[a][c] = aWd1[a][c] = 0.0f;
  int region = -1;
  const TabT* table = nullptr;
  float2* gtab = nullptr;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int k = region_of_chunk(s_base, p.K, t * kChunksPerTile);
    __syncthreads();  // previous tile's shared buffers fully consumed
    if (k != region) {
      if (region >= 0) flush_density_grad(p.grad_mlp + (size_t)region * kDensityParams, aWd1, aWd2, ib, nb);
#pragma unroll
      for (int a = 0; a < 4; ++a) aWd2[a][0] = 0.0f;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) aWd1[a][c] = 0.0f;
      const char* dblk = mlp + (size_t)k * kDensityParams * kEsize;
      for (int i = tid; i < kDensityParams; i += blockDim.x) s_w[i] = mlp_elem<kMlpType>(dblk, i);
      __syncthreads();
      region = k;
      table = static_cast<const TabT*>(p.tables) + (size_t)k * p.lp.E;
      gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
    }
    // ---- per sample (thread = sample tid of slot `warp`): chunk adjoints, geometry, features, SH(d)
    const SlotLane sl = slot_lane(p.chunks[t * kChunksPerTile + warp], lane);
    const uint2 ref = sl.ref;
    const bool chunk_ok = sl.slot_ok;  // warp-uniform; lanes of an unused part of the slot are empty samples
    bool valid = false;
    float u[3] = {0.0f, 0.0f, 0.0f}, dir[3] = {0.0f, 0.0f, 0.0f};
    float tr = 0.0f, dl = 0.0f;
    float gtc = 0.0f, gC[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f, gD = 0.0f, gL = 0.0f;
    float* rec = p.rec32 + (size_t)t * kIn * kBwdThreads + tid;  // feature j at rec[j * 256]
    {
      float feat[kIn];
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
          if (p.rec_in) {
#pragma unroll
            for (int j = 0; j < kIn; ++j) feat[j] = __ldcg(rec + j * kBwdThreads);
          } else {  // record them here: the density backward reads them again
            TableOf<kF16Table>::encode(p.lp, table, u, feat);
#pragma unroll
            for (int j = 0; j < kIn; ++j) __stcg(rec + j * kBwdThreads, feat[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kIn; ++j) s_D[j * kUPitch + tid] = feat[j];
      float sh[kSh];
      sh4_f32(dir, sh);
#pragma unroll
      for (int j = 0; j < kSh; ++j) s_C[(kGeo + j) * kUPitch + tid] = sh[j];
    }
    keep_scatter_inputs(s_U, s_V, u, valid, warp, lane, tid);
    __syncthreads();
    float acc[8][8];
    // ---- forward recompute: h1 = relu(F Wd1) -> A; g = h1 Wd2 -> C rows 0..15
    tile_gemm_ab<kIn>(s_D, Wd1, sb, 8 * ub, acc);
    tile_relu<8, 8>(acc);
    tile_store<8>(s_A, sb, 8 * ub, acc);
    __syncthreads();
    {
      float g2[8][2];
      tile_gemm_ab<kWidth, 2, kGeo>(s_A, Wd2, sb, 2 * ub, g2);
      tile_store<2>(s_C, sb, 2 * ub, g2);
    }
    __syncthreads();
    // ---- hc1 = relu(xc Wc1) -> D; hc2 = relu(hc1 Wc2) -> A
    tile_gemm_ab<kColorIn>(s_C, Wc1, sb, 8 * ub, acc);
    tile_relu<8, 8>(acc);
    tile_store<8>(s_D, sb, 8 * ub, acc);
    __syncthreads();
    tile_gemm_ab<kWidth>(s_D, Wc2, sb, 8 * ub, acc);
    tile_relu<8, 8>(acc);
    tile_store<8>(s_A, sb, 8 * ub, acc);
    __syncthreads();
    // ---- per sample: colour logits o = hc2 Wc3; chunk-local render adjoint
    float go[3] = {0.0f, 0.0f, 0.0f};
    {
      float oc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 8
      for (int n = 0; n < kWidth; ++n) {
        const float h2 = s_A[n * kUPitch + tid];
        const float4 w3 = *reinterpret_cast<const float4*>(Wc3 + 4 * n);
        oc[0] = fmaf(h2, w3.x, oc[0]);
        oc[1] = fmaf(h2, w3.y, oc[1]);
        oc[2] = fmaf(h2, w3.z, oc[2]);
      }
      float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
      if (valid) {
        sigma = expf(s_C[tid]);
#pragma unroll
        for (int m = 0; m < 3; ++m) rgb[m] = 1.0f / (1.0f + expf(-oc[m]));
      }
      float g_sigma = 0.0f, g_rgb[3] = {0.0f, 0.0f, 0.0f};
      if (chunk_ok) render_chunk_adjoint(sigma, rgb, tr, dl, sl.sl, gtc, gC, gA, gD, gL, g_sigma, g_rgb, sl.width);
      float go_d = 0.0f;
      if (valid) {
        go_d = g_sigma * sigma;
#pragma unroll
        for (int m = 0; m < 3; ++m) go[m] = g_rgb[m] * rgb[m] * (1.0f - rgb[m]);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) s_O[m * kUPitch + tid] = go[m];
      s_O[3 * kUPitch + tid] = go_d;
    }
    __syncthreads();
    // ---- Wc3[n][m] += sum_s hc2[s][n] go[s][m]   (one output per thread; column 3 unused)
    {
      const int n = tid >> 2, m = tid & 3;
      if (m < 3) {
        float a = 0.0f;
#pragma unroll 4
        for (int s = 0; s < kBwdThreads; s += 4) {
          const float4 hv = *reinterpret_cast<const float4*>(s_A + n * kUPitch + s);
          const float4 gv = *reinterpret_cast<const float4*>(s_O + m * kUPitch + s);
          a = fmaf(hv.x, gv.x, a);
          a = fmaf(hv.y, gv.y, a);
          a = fmaf(hv.z, gv.z, a);
          a = fmaf(hv.w, gv.w, a);
        }
        aWc3 += a;
      }
    }
    __syncthreads();
    // ---- dL/dzc2 = (hc2 > 0) (go Wc3^T), per sample, in place of hc2
#pragma unroll 8
    for (int n = 0; n < kWidth; ++n) {
      const float4 w3 = *reinterpret_cast<const float4*>(Wc3 + 4 * n);
      float* at = s_A + n * kUPitch + tid;
      *at = *at > 0.0f ? w3.x * go[0] + w3.y * go[1] + w3.z * go[2] : 0.0f;
    }
    __syncthreads();
    // ---- Wc2 += hc1^T dzc2
    {
      float dw[4][4];
      tile_gemm_dw<4>(s_D, s_A, ib, nb, dw);
      add_block<4, 4>(aWc2, dw);
    }
    __syncthreads();
    // ---- dL/dzc1 = (hc1 > 0) (dzc2 Wc2^T), in place of hc1
    tile_gemm_abt<kWidth, 8>(s_A, Wc2, sb, 8 * ub, acc);
    tile_store_masked(s_D, sb, 8 * ub, acc);
    __syncthreads();
    // ---- Wc1 += xc^T dzc1; dL/dg = (dzc1 Wc1^T)[0..15], plus dL/dg0 through the density
    {
      float dw[2][4];
      tile_gemm_dw<2>(s_C, s_D, ib, nb, dw);
      add_block<2, 4>(aWc1, dw);
    }
    {
      float dg[8][2];
      tile_gemm_abt<kWidth, 2>(s_D, Wc1, sb, 2 * ub, dg);
      if (ub == 0) {
        const float4 d0 = *reinterpret_cast<const float4*>(s_O + 3 * kUPitch + 4 * sb);
        const float4 d1 = *reinterpret_cast<const float4*>(s_O + 3 * kUPitch + 128 + 4 * sb);
        dg[0][0] += d0.x;
        dg[1][0] += d0.y;
        dg[2][0] += d0.z;
        dg[3][0] += d0.w;
        dg[4][0] += d1.x;
        dg[5][0] += d1.y;
        dg[6][0] += d1.z;
        dg[7][0] += d1.w;
      }
      __syncthreads();  // xc and dzc1 fully read
      tile_store<2>(s_C, sb, 2 * ub, dg);
    }
    // ---- the features again -> D rows 0..31
#pragma unroll
    for (int j = 0; j < kIn; ++j) s_D[j * kUPitch + tid] = valid ? __ldcs(rec + j * kBwdThreads) : 0.0f;
    __syncthreads();
    // ---- density MLP backward: h1 again -> A; Wd2 += h1^T dg; dz1 = (h1 > 0) (dg Wd2^T)
    tile_gemm_ab<kIn>(s_D, Wd1, sb, 8 * ub, acc);
    tile_relu<8, 8>(acc);
    tile_store<8>(s_A, sb, 8 * ub, acc);
    __syncthreads();
    {
      float dw[4][1];
      tile_gemm_dw<4, 1>(s_A, s_C, ib, nb, dw);
      add_block<4, 1>(aWd2, dw);
    }
    tile_gemm_abt<kGeo, 8, kGeo>(s_C, Wd2, sb, 8 * ub, acc);
    __syncthreads();  // h1 fully read
    tile_store_masked(s_A, sb, 8 * ub, acc);
    __syncthreads();
    // ---- Wd1 += F^T dz1; dL/dfeatures = dz1 Wd1^T -> D rows 0..31
    {
      float dw[2][4];
      tile_gemm_dw<2>(s_D, s_A, ib, nb, dw);
      add_block<2, 4>(aWd1, dw);
    }
    {
      float gx[8][4];
      tile_gemm_abt<kWidth, 4>(s_A, Wd1, sb, 4 * ub, gx);
      __syncthreads();  // features fully read
      tile_store<4>(s_D, sb, 4 * ub, gx);
    }
    __syncthreads();
    // ---- table gradients: thread (window, level) takes one level of 16 consecutive rows
    scatter_tile(p.lp, gtab, s_U, s_V, s_D, tid);
  }
  if (region >= 0) flush_density_grad(p.grad_mlp + (size_t)region * kDensityParams, aWd1, aWd2, ib, nb);
  // the shared colour block: once per CTA
  float* gc = p.grad_mlp + (size_t)p.K * kDensityParams;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (aWc1[a][c] != 0.0f) atomicAdd(gc + (ib + 16 * a) * kWidth + nb + 16 * c, aWc1[a][c]);
  float* gc2 = gc + kColorIn * kWidth;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (aWc2[a][c] != 0.0f) atomicAdd(gc2 + (ib + 16 * a) * kWidth + nb + 16 * c, aWc2[a][c]);
  if (aWc3 != 0.0f) atomicAdd(gc2 + kWidth * kWidth + tid, aWc3);  // [n][m] at n * 4 + m = tid
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
  if (f->mlp_dtype == NERFXL_F32 && f16tab)  // as the forward: the FP32 MLP reads FP32 tables
    return set_error(NERFXL_E_UNSUPPORTED, "FP16 tables go with a 16-bit MLP");
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
  p.rec_in = (s->flags & NERFXL_SAVE_FEATURES) != 0;
  // the fused kernel encodes again without the forward's records; the split
  // one records the features it encodes and reads them back
  p.rec32 = f->arch == NERFXL_ARCH_SPLIT || p.rec_in ? reinterpret_cast<float*>(ws + L.rec32) : nullptr;
  p.grad_tables = grad_tables;
  p.grad_mlp = grad_mlp;
  if (f->arch == NERFXL_ARCH_SPLIT) {
    const size_t smem_s = sizeof(float) * kBwdSplitSmemFloats + sizeof(int32_t) * (f->K + 1);
    if (smem_s > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
    void (*ks)(BwdParams) = k_field_bwd_split_f32<false, 0>;  // FP32 tables and MLP
    if (cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448) != cudaSuccess)
      return launch_check("k_field_bwd_split_f32 smem attribute");
    const int grid = fwd_grid(L.chunk_cap / kChunksPerTile, 1);
    profile_mark(0, stream);
    ks<<<grid, kBwdThreads, smem_s, stream>>>(p);
    profile_mark(1, stream);
    return kernel_launched("k_field_bwd_split_f32");
  }
  const size_t smem = sizeof(float) * kBwdSmemFloatsT + sizeof(int32_t) * (f->K + 1);
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
