// Backward (adjoint) of the field with the MLP on the tensor cores: the
// mixed-precision forms (BF16/FP16 MLP, FP32 or FP16 tables; FP32 gradients).
//
// One CTA = 16 warps on one 128-row tile (4 chunks of one region), the same
// row / lane-quarter / level-group mapping as the tensor-core forward. Per
// tile (all products K-major, 128-byte swizzled, FP32 accumulation in TMEM):
//   recompute  X (features) -> D1 = X W1 -> H1 = relu -> D2 = H1 W2 -> H2 = relu
//              -> D3 = H2 W3 -> sigma, rgb
//   adjoint    chunk-local render adjoint (warp scans) -> g_o [128 x 4]
//              G2 = (H2 > 0) * (g_o W3^T)                    (CUDA cores)
//              D4 = G2 W2^T, G1 = (H1 > 0) * D4             (tensor cores)
//              D5 = G1 W1^T = dL/dfeatures -> table scatter-add (vector atomics)
//              G2 and G1 enter these products as hi + lo pairs of 16-bit values
//              (two MMAs each), so the upstream gradient keeps ~16 mantissa
//              bits; the weights are exact in their 16-bit compute copy.
//   weights    DW += [G2^T ; G1^T] [H1 | X]  (M = 128, N = 96, K = 128 samples),
//              accumulated in TMEM over every tile of the region; its diagonal
//              blocks are dW2^T and dW1^T and are flushed once per region.
//              dW3 = H2^T g_o on CUDA cores (256 outputs).
// Bounded mbarrier waits flag kErrTimeout, free tensor memory and return.

#include <cuda_runtime.h>

#include "nerfxl_field.cuh"
#include "nerfxl_half.cuh"
#include "nerfxl_host.h"
#include "nerfxl_tc.cuh"

namespace nerfxl {
namespace {

constexpr int kRows = 128;
constexpr int kThreads = 512;
constexpr int kTileChunks = kRows / kWarp;
constexpr uint32_t kCols = 256;  // 0-63 D1/D3/D4, 64-127 D2/D5, 128-223 DW
constexpr uint32_t kDwCol = 128;
constexpr uint32_t kSpin = 1u << 24;

// Shared-memory plan (bytes from a 1024-aligned base).
constexpr uint32_t oX = 0;              // X  [128][64] (k < 32 used)
constexpr uint32_t oH1 = oX + 16384;    // H1 [128][64]
constexpr uint32_t oH2 = oH1 + 16384;   // H2 [128][64]
constexpr uint32_t oG2 = oH2 + 16384;   // G2 [128][64], 16-bit rounding (hi part)
constexpr uint32_t oG2l = oG2 + 16384;  // G2 - hi (lo part)
constexpr uint32_t oG1 = oG2l + 16384;  // G1 [128][64] hi
constexpr uint32_t oG1l = oG1 + 16384;  // G1 lo
constexpr uint32_t oAT = oG1l + 16384;  // [G2^T ; G1^T] (hi): 2 sub-tiles of [128 rows][64 samples]
constexpr uint32_t oBT = oAT + 32768;   // [H1^T ; X^T]: 2 sub-tiles of [96 rows][64 samples]
constexpr uint32_t kBTSub = 96 * 128;
constexpr uint32_t oB1 = oBT + 2 * kBTSub;  // W1^T [64][32]   (forward layer 1)
constexpr uint32_t oB2 = oB1 + 8192;        // W2^T [64][64]
constexpr uint32_t oB3 = oB2 + 8192;        // W3^T [16][64]
constexpr uint32_t oB4 = oB3 + 2048;        // W2 [64][64] (rows = h1 index)
constexpr uint32_t oB5 = oB4 + 8192;        // W1 [32][64] (rows = feature index)
constexpr uint32_t oW3f = oB5 + 4096;       // W3 fp32 [64][4]
constexpr uint32_t oGo = oW3f + 1024;       // g_o fp32 [128][4]
constexpr uint32_t oMisc = oGo + 2048;      // mbarrier, TMEM base
constexpr uint32_t oBase = oMisc + 64;      // int32 base[K+1]
constexpr size_t kSmemFixed = oBase + 1024;

struct BwdTcParams {
  const float* rays_o;
  const float* rays_d;
  const float* boxes;
  const void* tables;
  const void* mlp;  // 16-bit [K][kMlpParams]
  LevelParams lp;
  SampParams sp;
  int K;
  const RayHdr* hdr;
  const SegDesc* segs;
  const int32_t* base;
  const uint2* chunks;
  const int32_t* n_tiles;
  const float4* dpart;
  const uint4* feat_in;  // features saved by the forward, or NULL (gather again)
  float* grad_tables;  // FP32 [K][E][2]
  float* grad_mlp;     // FP32 [K][kMlpParams]
  int32_t* err;
};

template <bool BF16>
__device__ __forceinline__ void load_weights_bwd(const void* blk, char* sm) {
  uint16_t* b1 = reinterpret_cast<uint16_t*>(sm + oB1);
  uint16_t* b2 = reinterpret_cast<uint16_t*>(sm + oB2);
  uint16_t* b3 = reinterpret_cast<uint16_t*>(sm + oB3);
  uint16_t* b4 = reinterpret_cast<uint16_t*>(sm + oB4);
  uint16_t* b5 = reinterpret_cast<uint16_t*>(sm + oB5);
  float* w3f = reinterpret_cast<float*>(sm + oW3f);
  for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
    const int f = i / kWidth, n = i % kWidth;  // W1[f][n]
    const uint16_t v = Half2Of<BF16>::bits(blk, i);
    b1[tc::sw128_offset(n, f) >> 1] = v;  // forward: row n, k = f
    b5[tc::sw128_offset(f, n) >> 1] = v;  // backward: row f, k = n
  }
  for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
    const int a = i / kWidth, b = i % kWidth;  // W2[a][b]: h1 index a, z2 index b
    const uint16_t v = Half2Of<BF16>::bits(blk, kIn * kWidth + i);
    b2[tc::sw128_offset(b, a) >> 1] = v;  // forward: row b, k = a
    b4[tc::sw128_offset(a, b) >> 1] = v;  // backward: row a, k = b
  }
  for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
    const int n = i / 64, k = i % 64;
    b3[tc::sw128_offset(n, k) >> 1] =
        n < kOut ? Half2Of<BF16>::bits(blk, kIn * kWidth + kWidth * kWidth + k * kOut + n) : 0;
  }
  for (int i = threadIdx.x; i < kWidth * kOut; i += blockDim.x)
    w3f[i] = Half2Of<BF16>::load(blk, kIn * kWidth + kWidth * kWidth + i);
}

// Scatter dL/dfeat of levels l0..l0+3 (g8, level order) into the region's
// FP32 gradient table.
__device__ __forceinline__ void scatter4(const LevelParams& lp, float2* __restrict__ gtab, const float u[3], int l0,
                                         const float g8[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l = l0 + q;
    if (l >= lp.L) break;
    int c[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
    float2* gl = gtab + lp.off[l];
    const float g0 = g8[2 * q], g1 = g8[2 * q + 1];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const uint32_t y = c[1] + ((e >> 1) & 1), z = c[2] + ((e >> 2) & 1);
      const uint32_t i0 = vertex_index(lp, l, c[0], y, z);
      const uint32_t i1 = vertex_index(lp, l, c[0] + 1, y, z);
      const float wyz = (((e >> 1) & 1) ? f[1] : 1.0f - f[1]) * (((e >> 2) & 1) ? f[2] : 1.0f - f[2]);
      const float w0 = (1.0f - f[0]) * wyz, w1 = f[0] * wyz;
      if ((i0 ^ i1) == 1u) {
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

// Writes 16 values of row `row` as chunks 2g, 2g+1 of a normal tile and as
// column `row` of rows r0..r0+15 of a transposed (samples-contiguous) tile.
template <bool BF16>
__device__ __forceinline__ void store16(uint32_t tile, uint32_t row, int g, const float* v, uint32_t tt, uint32_t sub,
                                        uint32_t r0) {
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g), Half2Of<BF16>::pack(v[0], v[1]), Half2Of<BF16>::pack(v[2], v[3]),
                   Half2Of<BF16>::pack(v[4], v[5]), Half2Of<BF16>::pack(v[6], v[7]));
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g + 1), Half2Of<BF16>::pack(v[8], v[9]),
                   Half2Of<BF16>::pack(v[10], v[11]), Half2Of<BF16>::pack(v[12], v[13]),
                   Half2Of<BF16>::pack(v[14], v[15]));
  if (tt) {
    const uint32_t st = tt + (row >> 6) * sub;
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const uint32_t pk = Half2Of<BF16>::pack(v[i], v[i + 1]);
      tc::st_shared_u16(st + tc::sw128_offset(r0 + i, row & 63), (uint16_t)(pk & 0xFFFF));
      tc::st_shared_u16(st + tc::sw128_offset(r0 + i + 1, row & 63), (uint16_t)(pk >> 16));
    }
  }
}

// Writes 16 values of row `row` as a hi/lo pair of normal tiles (chunks 2g,
// 2g+1): hi = 16-bit rounding of v, lo = 16-bit rounding of v - hi.
template <bool BF16>
__device__ __forceinline__ void store16_lo(uint32_t tile_lo, uint32_t row, int g, const float* v) {
  float lo[16];
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    const float2 hv = Half2Of<BF16>::unpack(Half2Of<BF16>::pack(v[i], v[i + 1]));
    lo[i] = v[i] - hv.x;
    lo[i + 1] = v[i + 1] - hv.y;
  }
  tc::st_shared_v4(tile_lo + tc::sw128_chunk(row, 2 * g), Half2Of<BF16>::pack(lo[0], lo[1]),
                   Half2Of<BF16>::pack(lo[2], lo[3]), Half2Of<BF16>::pack(lo[4], lo[5]),
                   Half2Of<BF16>::pack(lo[6], lo[7]));
  tc::st_shared_v4(tile_lo + tc::sw128_chunk(row, 2 * g + 1), Half2Of<BF16>::pack(lo[8], lo[9]),
                   Half2Of<BF16>::pack(lo[10], lo[11]), Half2Of<BF16>::pack(lo[12], lo[13]),
                   Half2Of<BF16>::pack(lo[14], lo[15]));
}

// Bounded wait for the MMAs committed so far; false on timeout (all threads agree).
__device__ __forceinline__ bool mma_wait(uint64_t* mbar, uint32_t& phase) {
  const bool ok = tc::mbar_wait_bounded(mbar, phase, kSpin);
  phase ^= 1;
  return !__syncthreads_or(!ok);
}

template <bool kF16Table, bool BF16>
__global__ void __launch_bounds__(kThreads, 1) k_field_bwd_tc(BwdTcParams p) {
  extern __shared__ __align__(1024) char s_raw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = tc::smem_u32(sm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + oMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + oMisc + 8);
  int32_t* s_base = reinterpret_cast<int32_t*>(sm + oBase);
  const float* w3f = reinterpret_cast<const float*>(sm + oW3f);
  float* s_go = reinterpret_cast<float*>(sm + oGo);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  const int q = warp & 3, g = warp >> 2;
  const uint32_t row = (uint32_t)(q * kWarp + lane);

  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  if (warp == 0) tc::tmem_alloc(tmem_slot, kCols);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);

  constexpr uint32_t id64 = tc::idesc_f16(BF16, kRows, 64);
  constexpr uint32_t id32 = tc::idesc_f16(BF16, kRows, 32);
  constexpr uint32_t id16 = tc::idesc_f16(BF16, kRows, 16);
  constexpr uint32_t id96 = tc::idesc_f16(BF16, kRows, 96);
  using TabT = typename TableOf<kF16Table>::T;

  const int n_sub = *p.n_tiles * (kChunksPerTile / kTileChunks);
  int region = -1;
  const TabT* table = nullptr;
  float2* gtab = nullptr;
  uint32_t phase = 0;
  bool failed = false, dw_started = false;
  float acc3 = 0.0f;  // dW3 entry (tid < 256): row tid / 4, column tid % 4

  auto flush = [&]() {
    // dW accumulator -> global (diagonal blocks only); needs all MMAs complete.
    if (dw_started) {
      tc::fence_after_sync();
      float v[24];
      tc::tmem_ld16(tq + kDwCol + 24 * g, v);
      tc::tmem_ld8(tq + kDwCol + 24 * g + 16, v + 16);
      tc::tmem_ld_wait();
      float* gm = p.grad_mlp + (size_t)region * kMlpParams;
#pragma unroll
      for (int i = 0; i < 24; ++i) {
        const int c = 24 * g + i, r = (int)row;
        if (r < 64 && c < 64) {
          atomicAdd(gm + kIn * kWidth + c * kWidth + r, v[i]);  // dW2[h1 = c][z2 = r]
        } else if (r >= 64 && c >= 64 && c < 96) {
          atomicAdd(gm + (c - 64) * kWidth + (r - 64), v[i]);  // dW1[feat = c - 64][z1 = r - 64]
        }
      }
    }
    if (tid < kWidth * kOut && region >= 0 && acc3 != 0.0f)
      atomicAdd(p.grad_mlp + (size_t)region * kMlpParams + kIn * kWidth + kWidth * kWidth + tid, acc3);
    acc3 = 0.0f;
    dw_started = false;
  };

  for (int t = blockIdx.x; t < n_sub && !failed; t += gridDim.x) {
    const int k = region_of_chunk(s_base, p.K, t * kTileChunks);
    if (k != region) {
      tc::fence_before_sync();
      __syncthreads();
      if (region >= 0) flush();
      tc::fence_before_sync();
      __syncthreads();
      load_weights_bwd<BF16>(static_cast<const uint16_t*>(p.mlp) + (size_t)k * kMlpParams, sm);
      region = k;
      table = static_cast<const TabT*>(p.tables) + (size_t)k * p.lp.E;
      gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
    }
    // ---- gather (four threads per row, four levels each)
    const uint2 ref = p.chunks[t * kTileChunks + q];
    const bool chunk_ok = ref.x != kEmptyChunk;
    bool valid = false;
    float tr = 0.0f, dl = 0.0f, u[3] = {0.0f, 0.0f, 0.0f};
    float f8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) f8[i] = 0.0f;
    float gtc = 0.0f, gC[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f, gD = 0.0f, gL = 0.0f;
    if (chunk_ok) {
      const uint32_t ray = ref.x;
      const int seg = ref.y >> 16, c = ref.y & 0xFFFF;
      const RayHdr h = p.hdr[ray];
      const SegDesc sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
      const int i = c * kWarp + lane;
      valid = i < seg_n(sd);
      if (g == 0) {
        const size_t slot = (size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c;
        const float4 a0 = p.dpart[2 * slot], a1 = p.dpart[2 * slot + 1];
        gtc = a0.x;
        gC[0] = a0.y;
        gC[1] = a0.z;
        gC[2] = a0.w;
        gA = a1.x;
        gD = a1.y;
        gL = a1.z;
      }
      if (valid) {
        float o[3], d[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          o[ax] = p.rays_o[3 * (size_t)ray + ax];
          d[ax] = p.rays_d[3 * (size_t)ray + ax];
        }
        float a, b;
        segment_interval(sd, h.tn, h.delta, i, a, b);
        const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
        dl = __fsub_rn(b, a);
        tr = __fsub_rn(tbar, h.tn);
        float x[3];
        sample_point(o, d, tbar, x);
        region_coord(p.boxes + 6 * k, x, u);
        if (p.feat_in) {
          const uint4 pk = p.feat_in[((size_t)(t * kTileChunks + q) * 4 + g) * kWarp + lane];
          const uint32_t wv[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float2 fv = Half2Of<BF16>::unpack(wv[j]);
            f8[2 * j] = fv.x;
            f8[2 * j + 1] = fv.y;
          }
        } else {
          gather4<TabT>(p.lp, table, u, 4 * g, f8);
        }
      }
    }
    {
      // X (normal, chunk g) and X^T (rows 64 + 8g .. 64 + 8g + 7 of the B^T tile)
      tc::st_shared_v4(sb + oX + tc::sw128_chunk(row, g), Half2Of<BF16>::pack(f8[0], f8[1]),
                       Half2Of<BF16>::pack(f8[2], f8[3]), Half2Of<BF16>::pack(f8[4], f8[5]),
                       Half2Of<BF16>::pack(f8[6], f8[7]));
      const uint32_t st = sb + oBT + (row >> 6) * kBTSub;
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        const uint32_t pk = Half2Of<BF16>::pack(f8[i], f8[i + 1]);
        tc::st_shared_u16(st + tc::sw128_offset(64 + 8 * g + i, row & 63), (uint16_t)(pk & 0xFFFF));
        tc::st_shared_u16(st + tc::sw128_offset(64 + 8 * g + i + 1, row & 63), (uint16_t)(pk >> 16));
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- forward recompute: D1 = X W1
    if (tid == 0) {
      tc::fence_after_sync();
      for (int kk = 0; kk < 2; ++kk)
        tc::mma_f16(tmem, tc::desc_sw128(sb + oX + 32 * kk), tc::desc_sw128(sb + oB1 + 32 * kk), id64, kk);
      tc::mma_commit(mbar);
    }
    if (!mma_wait(mbar, phase)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    float v[16];
    tc::tmem_ld16(tq + 16 * g, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
    store16<BF16>(sb + oH1, row, g, v, sb + oBT, kBTSub, 16 * g);  // H1 and H1^T (B^T rows 0..63)
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // D2 = H1 W2
    if (tid == 0) {
      tc::fence_after_sync();
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem + 64, tc::desc_sw128(sb + oH1 + 32 * kk), tc::desc_sw128(sb + oB2 + 32 * kk), id64, kk);
      tc::mma_commit(mbar);
    }
    if (!mma_wait(mbar, phase)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    tc::tmem_ld16(tq + 64 + 16 * g, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
    store16<BF16>(sb + oH2, row, g, v, 0, 0, 0);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // D3 = H2 W3
    if (tid == 0) {
      tc::fence_after_sync();
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem, tc::desc_sw128(sb + oH2 + 32 * kk), tc::desc_sw128(sb + oB3 + 32 * kk), id16, kk);
      tc::mma_commit(mbar);
    }
    if (!mma_wait(mbar, phase)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // ---- chunk-local render adjoint -> g_o (warps of level group 0)
    if (g == 0) {
      tc::tmem_ld16(tq, v);
      tc::tmem_ld_wait();
      float go[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (chunk_ok) {
        float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
          sigma = expf(v[0]);
#pragma unroll
          for (int j = 0; j < 3; ++j) rgb[j] = 1.0f / (1.0f + expf(-v[1 + j]));
        }
        float g_sigma, g_rgb[3];
        render_chunk_adjoint(sigma, rgb, tr, dl, lane, gtc, gC, gA, gD, gL, g_sigma, g_rgb);
        if (valid) {
          go[0] = g_sigma * sigma;
#pragma unroll
          for (int j = 0; j < 3; ++j) go[1 + j] = g_rgb[j] * rgb[j] * (1.0f - rgb[j]);
        }
      }
      *reinterpret_cast<float4*>(s_go + 4 * row) = make_float4(go[0], go[1], go[2], go[3]);
    }
    tc::fence_before_sync();
    __syncthreads();
    // ---- G2 = (H2 > 0) * (g_o W3^T), columns 16g..16g+15 of this row; G2^T rows 0..63 of A^T
    {
      const float4 go = *reinterpret_cast<const float4*>(s_go + 4 * row);
      const uint4 h0 = tc::ld_shared_v4(sb + oH2 + tc::sw128_chunk(row, 2 * g));
      const uint4 h1 = tc::ld_shared_v4(sb + oH2 + tc::sw128_chunk(row, 2 * g + 1));
      const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 hv = Half2Of<BF16>::unpack(hw[i]);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int n = 16 * g + 2 * i + hh;
          const float4 w3 = *reinterpret_cast<const float4*>(w3f + 4 * n);
          const float s = w3.x * go.x + w3.y * go.y + w3.z * go.z + w3.w * go.w;
          v[2 * i + hh] = (hh ? hv.y : hv.x) > 0.0f ? s : 0.0f;
        }
      }
      store16<BF16>(sb + oG2, row, g, v, sb + oAT, 16384, 16 * g);
      store16_lo<BF16>(sb + oG2l, row, g, v);
    }
    // dW3[n][m] += sum_rows H2[row][n] g_o[row][m]
    if (tid < kWidth * kOut) {
      const int n = tid >> 2, m = tid & 3;
      float s = 0.0f;
      for (int r = 0; r < kRows; ++r)
        s = fmaf(Half2Of<BF16>::from_bits(tc::ld_shared_u16(sb + oH2 + tc::sw128_offset(r, n))), s_go[4 * r + m], s);
      acc3 += s;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- D4 = G2 W2^T (dL/dh1)
    if (tid == 0) {
      tc::fence_after_sync();
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem, tc::desc_sw128(sb + oG2 + 32 * kk), tc::desc_sw128(sb + oB4 + 32 * kk), id64, kk);
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem, tc::desc_sw128(sb + oG2l + 32 * kk), tc::desc_sw128(sb + oB4 + 32 * kk), id64, 1);
      tc::mma_commit(mbar);
    }
    if (!mma_wait(mbar, phase)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    tc::tmem_ld16(tq + 16 * g, v);
    tc::tmem_ld_wait();
    {
      // G1 = (H1 > 0) * D4; G1^T rows 64..127 of A^T
      const uint4 h0 = tc::ld_shared_v4(sb + oH1 + tc::sw128_chunk(row, 2 * g));
      const uint4 h1 = tc::ld_shared_v4(sb + oH1 + tc::sw128_chunk(row, 2 * g + 1));
      const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 hv = Half2Of<BF16>::unpack(hw[i]);
        if (!(hv.x > 0.0f)) v[2 * i] = 0.0f;
        if (!(hv.y > 0.0f)) v[2 * i + 1] = 0.0f;
      }
      store16<BF16>(sb + oG1, row, g, v, sb + oAT, 16384, 64 + 16 * g);
      store16_lo<BF16>(sb + oG1l, row, g, v);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- D5 = G1 W1^T (dL/dfeatures); DW += [G2^T; G1^T] [H1 | X]
    if (tid == 0) {
      tc::fence_after_sync();
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem + 64, tc::desc_sw128(sb + oG1 + 32 * kk), tc::desc_sw128(sb + oB5 + 32 * kk), id32, kk);
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_f16(tmem + 64, tc::desc_sw128(sb + oG1l + 32 * kk), tc::desc_sw128(sb + oB5 + 32 * kk), id32, 1);
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t off = (uint32_t)(kk & 3) * 32;  // 16 samples per K step, 4 steps per sub-tile
        tc::mma_f16(tmem + kDwCol, tc::desc_sw128(sb + oAT + (kk >> 2) * 16384 + off),
                    tc::desc_sw128(sb + oBT + (kk >> 2) * kBTSub + off), id96, (dw_started || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(mbar);
    }
    dw_started = true;
    if (!mma_wait(mbar, phase)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    float g8[8];
    tc::tmem_ld8(tq + 64 + 8 * g, g8);
    tc::tmem_ld_wait();
    if (valid) scatter4(p.lp, gtab, u, 4 * g, g8);
    tc::fence_before_sync();
    __syncthreads();  // tiles and TMEM free for the next tile
  }
  if (!failed && region >= 0) {
    tc::fence_before_sync();
    __syncthreads();
    flush();
  }
  if (failed && tid == 0) atomicOr(p.err, kErrTimeout);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace

nerfxl_status launch_field_bwd_tc(const nerfxl_field* f, const SampParams& sp, const LevelParams& lp,
                                  const float* rays_o, const float* rays_d, char* ws, const Layout& L,
                                  const float4* dpart, const uint4* feat_in, float* grad_tables, float* grad_mlp,
                                  cudaStream_t stream) {
  BwdTcParams p;
  p.feat_in = feat_in;
  p.rays_o = rays_o;
  p.rays_d = rays_d;
  p.boxes = f->boxes;
  p.tables = f->tables;
  p.mlp = f->mlp;
  p.lp = lp;
  p.sp = sp;
  p.K = f->K;
  p.hdr = reinterpret_cast<const RayHdr*>(ws + L.ray_hdr);
  p.segs = reinterpret_cast<const SegDesc*>(ws + L.segs);
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.chunks = reinterpret_cast<const uint2*>(ws + L.chunks);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.dpart = dpart;
  p.grad_tables = grad_tables;
  p.grad_mlp = grad_mlp;
  p.err = reinterpret_cast<int32_t*>(ws + L.hdr);
  const size_t smem = kSmemFixed + sizeof(int32_t) * (f->K + 1);
  if (smem > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
  const bool bf16 = f->mlp_dtype == NERFXL_BF16;
  const bool f16tab = f->table_dtype == NERFXL_F16;
  void (*kern)(BwdTcParams) = nullptr;
  if (f16tab) kern = bf16 ? k_field_bwd_tc<true, true> : k_field_bwd_tc<true, false>;
  else kern = bf16 ? k_field_bwd_tc<false, true> : k_field_bwd_tc<false, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return launch_check("k_field_bwd_tc smem attribute");
  const int grid = fwd_grid(L.chunk_cap / kTileChunks, 1);
  profile_mark(0, stream);
  kern<<<grid, kThreads, smem, stream>>>(p);
  profile_mark(1, stream);
  return launch_check("k_field_bwd_tc");
}

}  // namespace nerfxl
