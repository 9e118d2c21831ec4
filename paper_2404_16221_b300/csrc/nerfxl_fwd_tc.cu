// Field forward with the MLP on the tensor cores (tcgen05, accumulators in
// tensor memory): the mixed-precision forms (BF16 or FP16 MLP with FP32
// accumulation; FP32 or FP16 hash features).
//
// One CTA = 16 warps on one 128-row MMA tile (4 slots of 32 rows, each one
// chunk of up to 32 samples or two or four shorter ones, all of one region).
// Warp w serves rows 32 (w % 4) .. + 31 (its TMEM lane quarter)
// and level group / column block w / 4, so each sample's 16-level gather is
// spread over four threads that run concurrently. Per tile:
//   gather   thread (row, g) encodes levels 4g..4g+3 and writes their eight
//            features as one 16-byte chunk of row `row` of A0 (bf16/fp16)
//   layer 1  D1[128x64] = A0[128x32] W1            (2 MMAs, K = 16 each)
//   layer 2  h1 = relu(D1) -> A1; D2 = A1 W2        (4 MMAs)
//   layer 3  h2 = relu(D2) -> A0; D3[128x16] = A0 W3 (4 MMAs; columns 4..15 zero)
//   render   sigma = exp(D3[:,0]), rgb = sigmoid(D3[:,1..3]); chunk partial,
//            by the four warps of level group 0 while the other twelve
//            already gather the next tile (no barrier closes a tile)
// The split representation (kSplit) runs five layers on the same tile:
//   density  D1 = A0 Wd1 -> relu -> A1;  G[128x16] = A1 Wd2
//   colour   A0 = [G (16) | SH(d) (16)];  D1 = A0 Wc1 -> relu -> A1;
//            D2 = A1 Wc2 -> relu -> A0;  D3 = A0 Wc3;  sigma = exp(G[:,0])
// with the region's density weights reloaded per region and the shared
// colour weights staged once per CTA.
// One elected thread issues the MMAs and commits them to an mbarrier; each
// warp reads 16 accumulator columns of its lane quarter with tcgen05.ld.
// Waits on the mbarrier are bounded: on expiry the kernel flags
// kErrTimeout in the workspace, frees its tensor memory and returns.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "nerfxl_split.cuh"
#include "nerfxl_half.cuh"
#include "nerfxl_host.h"
#include "nerfxl_tc.cuh"

namespace nerfxl {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 512;  // 16 warps: 4 per TMEM lane quarter
constexpr int kTcChunks = kTcRows / kWarp;  // 4 chunks per MMA tile
constexpr uint32_t kTmemCols = 128;         // D1 at column 0, D2 at column 64, D3 reuses column 0
constexpr uint32_t kSpinLimit = 1u << 24;

// Shared-memory plan (offsets from a 1024-byte-aligned base).
constexpr uint32_t kOffA0 = 0;                    // 128 rows x 128 B
constexpr uint32_t kOffA1 = kOffA0 + 128 * 128;   // 128 rows x 128 B
constexpr uint32_t kOffB1 = kOffA1 + 128 * 128;   // 64 rows (n) x 128 B (k < 32 used)
constexpr uint32_t kOffB2 = kOffB1 + 64 * 128;    // 64 rows x 128 B
constexpr uint32_t kOffB3 = kOffB2 + 64 * 128;    // 16 rows x 128 B
constexpr uint32_t kOffC1 = kOffB3 + 16 * 128;    // split: Wc1, 64 rows x 128 B (k < 32 used)
constexpr uint32_t kOffC3 = kOffC1 + 64 * 128;    // split: Wc3, 16 rows x 128 B
constexpr uint32_t kOffMisc = kOffC3 + 16 * 128;  // mbarrier (8 B), tmem base (4 B)
constexpr uint32_t kOffBase = kOffMisc + 64;      // int32 base[K+1]
constexpr size_t kTcSmemFixed = kOffBase + 1024;  // + 1024 slack for the alignment of the base

// Operand kinds of the MLP MMAs: 0 = BF16, 1 = FP16 (kind::f16, 16 elements
// per 32-byte K step), 2 = E4M3 (kind::f8f6f4, 32 elements per K step, with a
// per-layer weight scale applied to the FP32 accumulator). In every kind a
// tile row is 128 bytes of the 128-byte swizzle and a K step is 32 bytes.
constexpr int kKindBF16 = 0, kKindF16 = 1, kKindE4M3 = 2;

template <int kKind>
struct MlpOp {
  static constexpr bool kBF16 = kKind == kKindBF16;
  static constexpr uint32_t idesc(int M, int N) { return tc::idesc_f16(kBF16, M, N); }
  static constexpr int steps(int K) { return K / 16; }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_f16(d, a, b, id, acc);
  }
  // eight features (levels 4g..4g+3) -> 16-byte chunk g of the row
  __device__ static void store8(uint32_t tile, uint32_t row, int g, const float* f) {
    tc::st_shared_v4(tile + tc::sw128_chunk(row, g), Half2Of<kBF16>::pack(f[0], f[1]), Half2Of<kBF16>::pack(f[2], f[3]),
                     Half2Of<kBF16>::pack(f[4], f[5]), Half2Of<kBF16>::pack(f[6], f[7]));
  }
  // sixteen activations (columns 16g..16g+15) -> chunks 2g, 2g+1 of the row
  __device__ static void store16(uint32_t tile, uint32_t row, int g, const float* v) {
    tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g), Half2Of<kBF16>::pack(v[0], v[1]),
                     Half2Of<kBF16>::pack(v[2], v[3]), Half2Of<kBF16>::pack(v[4], v[5]),
                     Half2Of<kBF16>::pack(v[6], v[7]));
    tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g + 1), Half2Of<kBF16>::pack(v[8], v[9]),
                     Half2Of<kBF16>::pack(v[10], v[11]), Half2Of<kBF16>::pack(v[12], v[13]),
                     Half2Of<kBF16>::pack(v[14], v[15]));
  }
  // B(row n, column k) = W[k][n] for the three layers (row-major 16-bit block)
  __device__ static void load_weights(const void* blk, char* sm) {
    uint16_t* b1 = reinterpret_cast<uint16_t*>(sm + kOffB1);
    uint16_t* b2 = reinterpret_cast<uint16_t*>(sm + kOffB2);
    uint16_t* b3 = reinterpret_cast<uint16_t*>(sm + kOffB3);
    for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
      const int k = i / kWidth, n = i % kWidth;
      b1[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, i);
    }
    for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
      const int k = i / kWidth, n = i % kWidth;
      b2[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, kIn * kWidth + i);
    }
    for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
      const int n = i / 64, k = i % 64;
      b3[tc::sw128_offset(n, k) >> 1] =
          n < kOut ? Half2Of<kBF16>::bits(blk, kIn * kWidth + kWidth * kWidth + k * kOut + n) : 0;
    }
  }
};

// Split representation, 16-bit kinds: B tiles of the region's density MLP
// (B1 <- Wd1 [32][64], B3 <- Wd2 [64][16]) and of the shared colour MLP
// (C1 <- Wc1 [32][64], B2 <- Wc2 [64][64], C3 <- Wc3 [64][4], rows >= 4 zero).
template <bool kBF16>
__device__ void load_density_tc(const void* blk, char* sm) {
  uint16_t* b1 = reinterpret_cast<uint16_t*>(sm + kOffB1);
  uint16_t* b3 = reinterpret_cast<uint16_t*>(sm + kOffB3);
  for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
    const int k = i / kWidth, n = i % kWidth;
    b1[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, i);
  }
  for (int i = threadIdx.x; i < 16 * kWidth; i += blockDim.x) {
    const int n = i / kWidth, k = i % kWidth;  // B3 row n = output n of Wd2
    b3[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, kIn * kWidth + k * kGeo + n);
  }
}

template <bool kBF16>
__device__ void load_color_tc(const void* blk, char* sm) {
  uint16_t* c1 = reinterpret_cast<uint16_t*>(sm + kOffC1);
  uint16_t* b2 = reinterpret_cast<uint16_t*>(sm + kOffB2);
  uint16_t* c3 = reinterpret_cast<uint16_t*>(sm + kOffC3);
  for (int i = threadIdx.x; i < kColorIn * kWidth; i += blockDim.x) {
    const int k = i / kWidth, n = i % kWidth;
    c1[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, i);
  }
  for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
    const int k = i / kWidth, n = i % kWidth;
    b2[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, kColorIn * kWidth + i);
  }
  for (int i = threadIdx.x; i < 16 * kWidth; i += blockDim.x) {
    const int n = i / kWidth, k = i % kWidth;
    c3[tc::sw128_offset(n, k) >> 1] =
        n < kOut ? Half2Of<kBF16>::bits(blk, kColorIn * kWidth + kWidth * kWidth + k * kOut + n) : 0;
  }
}

// E4M3: byte (row, k) of a swizzled tile sits at row*128 + ((k/16 ^ row%8) * 16) + k%16.
__device__ __forceinline__ uint32_t sw128_byte(uint32_t row, uint32_t k) {
  return row * 128u + ((((k >> 4) ^ (row & 7u)) & 7u) << 4) + (k & 15u);
}

__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

template <>
struct MlpOp<kKindE4M3> {
  static constexpr uint32_t idesc(int M, int N) { return tc::idesc_e4m3(M, N); }
  static constexpr int steps(int K) { return K / 32; }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_f8(d, a, b, id, acc);
  }
  __device__ static void store8(uint32_t tile, uint32_t row, int g, const float* f) {
    const uint32_t addr = tile + tc::sw128_chunk(row, g >> 1) + (uint32_t)(g & 1) * 8u;
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(e4m3x4(f[0], f[1], f[2], f[3])),
                 "r"(e4m3x4(f[4], f[5], f[6], f[7]))
                 : "memory");
  }
  __device__ static void store16(uint32_t tile, uint32_t row, int g, const float* v) {
    tc::st_shared_v4(tile + tc::sw128_chunk(row, g), e4m3x4(v[0], v[1], v[2], v[3]), e4m3x4(v[4], v[5], v[6], v[7]),
                     e4m3x4(v[8], v[9], v[10], v[11]), e4m3x4(v[12], v[13], v[14], v[15]));
  }
  __device__ static void load_weights(const void* blk, char* sm) {
    const uint8_t* w = static_cast<const uint8_t*>(blk);
    uint8_t* b1 = reinterpret_cast<uint8_t*>(sm + kOffB1);
    uint8_t* b2 = reinterpret_cast<uint8_t*>(sm + kOffB2);
    uint8_t* b3 = reinterpret_cast<uint8_t*>(sm + kOffB3);
    for (int i = threadIdx.x; i < kIn * kWidth; i += blockDim.x) {
      const int k = i / kWidth, n = i % kWidth;
      b1[sw128_byte(n, k)] = w[i];
    }
    for (int i = threadIdx.x; i < kWidth * kWidth; i += blockDim.x) {
      const int k = i / kWidth, n = i % kWidth;
      b2[sw128_byte(n, k)] = w[kIn * kWidth + i];
    }
    for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
      const int n = i / 64, k = i % 64;
      b3[sw128_byte(n, k)] = n < kOut ? w[kIn * kWidth + kWidth * kWidth + k * kOut + n] : 0;
    }
  }
};

// Reads 64 accumulator columns of this thread's row, applies relu.
__device__ __forceinline__ void tmem_row64_relu(uint32_t taddr, float* v) {
  tc::tmem_ld16(taddr + 0, v);
  tc::tmem_ld16(taddr + 16, v + 16);
  tc::tmem_ld16(taddr + 32, v + 32);
  tc::tmem_ld16(taddr + 48, v + 48);
  tc::tmem_ld_wait();
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = fmaxf(v[i], 0.0f);
}

struct FwdTcParams {
  const float* rays_o;
  const float* rays_d;
  const float* boxes;
  const void* tables;  // [K][E] of float2 or half2
  const void* mlp;     // [K][kMlpParams] 16-bit, or E4M3 bytes
  const float* mlp_scales;  // [K][3] per-layer weight scales (E4M3 only)
  LevelParams lp;
  SampParams sp;
  int K;
  const RayHdr* hdr;
  const SegDesc* segs;
  const int32_t* base;
  const Slot* chunks;  // slots
  const int32_t* n_tiles;  // tiles of kChunksPerTile chunks
  float4* partials;
  RecordOut rec;  // the backward's per-tile records, or all NULL
  int32_t* err;
  // Level-grouped gather (kFeatIn): level l of row r of tile t is the word
  // feat_in[(l * window + t - w0) * 128 + r]; the kernel covers tiles w0..w1-1.
  const uint32_t* feat_in;
  int64_t window;
  int64_t w0, w1;
};

template <bool kF16Table, int kKind, bool kRec, bool kSplit, bool kFeatIn = false>
__global__ void __launch_bounds__(kTcThreads, 2) k_field_fwd_tc(FwdTcParams p) {
  static_assert(!kSplit || kKind != kKindE4M3, "the split form is a 16-bit forward");
  using Op = MlpOp<kKind>;
  extern __shared__ __align__(1024) char s_raw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = tc::smem_u32(sm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
  int32_t* s_base = reinterpret_cast<int32_t*>(sm + kOffBase);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  // Warp w owns TMEM lane quarter q = w % 4 (rows 32q..32q+31, i.e. chunk q of
  // the tile) and level group / column block g = w / 4.
  const int q = warp & 3, g = warp >> 2;
  const uint32_t row = (uint32_t)(q * kWarp + lane);

  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_q = tmem + ((uint32_t)(q * 32) << 16);

  constexpr uint32_t idesc64 = Op::idesc(kTcRows, 64);
  constexpr uint32_t idesc16 = Op::idesc(kTcRows, 16);
  constexpr int kSteps32 = Op::steps(32), kSteps64 = Op::steps(64);
  constexpr size_t kElem = kKind == kKindE4M3 ? 1 : 2;
  float scale[3] = {1.0f, 1.0f, 1.0f};
  const uint32_t a0 = sbase + kOffA0, a1 = sbase + kOffA1;
  const uint32_t b1 = sbase + kOffB1, b2 = sbase + kOffB2, b3 = sbase + kOffB3;
  using TabT = typename TableOf<kF16Table>::T;

  const uint32_t c1 = sbase + kOffC1, c3 = sbase + kOffC3;
  if (kSplit) load_color_tc<kKind == kKindBF16>(static_cast<const char*>(p.mlp) + (size_t)p.K * kDensityParams * 2, sm);
  const int n_all = *p.n_tiles * (kChunksPerTile / kTcChunks);
  const int n_sub = (int)(p.w1 < (int64_t)n_all ? p.w1 : (int64_t)n_all);
  int region = -1;
  const TabT* table = nullptr;
  uint32_t phase = 0;
  bool failed = false;
  // kFeatIn: this thread's four levels (4g..4g+3) of the next tile's
  // features, loaded one tile ahead so that the HBM latency hides behind the
  // current tile
  uint32_t feat_next[4] = {0u, 0u, 0u, 0u};
  auto load_feat = [&](int64_t tl, uint32_t* w) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      w[j] = 4 * g + j < p.lp.L ? __ldcs(p.feat_in + ((size_t)(4 * g + j) * p.window + tl) * kTcRows + row) : 0u;
  };
  if (kFeatIn && (int)p.w0 + (int)blockIdx.x < n_sub) load_feat(blockIdx.x, feat_next);
  // The features record of tile t, exactly as the first MMA reads them: one
  // 16-byte chunk per thread (row tid / 4, chunk tid % 4) from the complete
  // layer-1 A tile, so that a warp writes eight whole 64-byte record rows.
  auto store_feat_record = [&](int t) {
    const uint32_t r = (uint32_t)tid >> 2, c = (uint32_t)tid & 3u;
    const uint4 w = tc::ld_shared_v4(a0 + tc::sw128_chunk(r, c));
    __stcs(p.rec.feat + (size_t)t * (kRecFeatBytes / 16) + r * 4 + (c ^ ((r >> 1) & 3u)), w);
  };
  static_assert(kTcThreads == 4 * kTcRows, "one feature chunk per thread");
  for (int t = (int)p.w0 + blockIdx.x; t < n_sub && !failed; t += gridDim.x) {
    const int k = region_of_chunk(s_base, p.K, t * kTcChunks);
    if (k != region) {
      __syncthreads();
      if (kSplit) load_density_tc<kKind == kKindBF16>(static_cast<const char*>(p.mlp) + (size_t)k * kDensityParams * 2, sm);
      else Op::load_weights(static_cast<const char*>(p.mlp) + (size_t)k * kMlpParams * kElem, sm);
      if (kKind == kKindE4M3) {
#pragma unroll
        for (int l = 0; l < 3; ++l) scale[l] = p.mlp_scales[3 * k + l];
      }
      region = k;
      table = static_cast<const TabT*>(p.tables) + (size_t)k * p.lp.E;
    }
    // ---- gather: the four threads of a row each gather four levels
    const SlotLane sl = slot_lane(p.chunks[t * kTcChunks + q], lane);
    const uint2 ref = sl.ref;
    const bool chunk_ok = sl.slot_ok;  // warp-uniform; lanes of an unused part of the slot are empty samples
    bool valid = false;
    float tr = 0.0f, dl = 0.0f, u[3] = {0.0f, 0.0f, 0.0f};
    float f8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) f8[i] = 0.0f;
    SegDesc sd = {0.0f, 0.0f, 0, 0};
    int c = 0, seg_count = 0;
    uint32_t ray = 0;
    float dir[3] = {0.0f, 0.0f, 0.0f};  // the ray's direction (the split form's colour input)
    if (sl.has) {
      ray = ref.x;
      const int seg = ref.y >> 16;
      c = ref.y & 0xFFFF;
      const RayHdr h = p.hdr[ray];
      sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
      const SegSamples ss = seg_samples(p.sp, sd, ray, seg);
      seg_count = ss.n;
      const int i = c * kWarp + sl.sl;
      valid = i < ss.n;
      if (valid) {
        float o[3], d[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          o[ax] = p.rays_o[3 * (size_t)ray + ax];
          d[ax] = p.rays_d[3 * (size_t)ray + ax];
          dir[ax] = d[ax];
        }
        float a, b;
        segment_interval(sd, h.tn, h.delta, sample_interval(p.sp, ss, i), a, b);
        const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
        dl = __fsub_rn(b, a);
        tr = __fsub_rn(tbar, h.tn);
        float x[3];
        sample_point(o, d, tbar, x);
        region_coord(p.boxes + 6 * k, x, u);
        if (!kFeatIn) gather4<TabT>(p.lp, table, u, 4 * g, f8);
      }
    }
    uint4 fw = make_uint4(0u, 0u, 0u, 0u);  // kFeatIn: this thread's packed features
    if (kFeatIn) {  // the level-grouped gather's words of row `row`, levels 4g..4g+3
      fw = make_uint4(feat_next[0], feat_next[1], feat_next[2], feat_next[3]);
      if (t + (int)gridDim.x < n_sub) load_feat(t + gridDim.x - p.w0, feat_next);
      tc::st_shared_v4(a0 + tc::sw128_chunk(row, g), fw.x, fw.y, fw.z, fw.w);
    } else {
      Op::store8(a0, row, g, f8);
    }
    if (kRec) {
      // Records for the backward: the sample's region coordinates / position /
      // length (thread g stores one of u0, u1, u2, tr; g == 0 also dl), the
      // slot's sample counts, and each chunk's tile-order position for the
      // composite adjoint (the features are copied from the layer-1 A tile
      // while its MMA runs; Tn, w, pair, sigma and rgb follow from the chunk
      // render below). Streaming stores: the records are read once, by the
      // backward, and should not push the region's tables out of L2 meanwhile.
      float* geo = p.rec.geom + (size_t)t * kGeomFloats;
      __stcs(geo + g * kTcRows + row, g == 0 ? u[0] : (g == 1 ? u[1] : (g == 2 ? u[2] : tr)));
      if (kSplit && g == 1) {  // the split form's colour input: the ray direction, rows 5..7
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) __stcs(geo + (5 + ax) * kTcRows + row, dir[ax]);
      }
      if (g == 0) {
        __stcs(geo + 4 * kTcRows + row, dl);
        // the slot's sample counts, one per part (see slot_count)
        const int n_mine = sl.has ? min(kWarp, seg_count - c * kWarp) : 0;
        int n4[4];
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) n4[pp] = __shfl_sync(0xFFFFFFFFu, n_mine, (pp * sl.width) & (kWarp - 1));
        if (sl.width == kWarp) n4[1] = n4[2] = n4[3] = 0;
        else if (sl.width == 16) n4[2] = n4[3] = 0;
        if (lane == 0)
          reinterpret_cast<int32_t*>(geo)[kGeomRowFields * kTcRows + q] = chunk_ok ? slot_count_word(sl.width, n4) : 0;
        if (sl.has && sl.sl == 0)  // tile-order position of the chunk's adjoints: 4 per slot
          p.rec.pos[(size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c] = 4 * (t * kTcChunks + q) + sl.part;
      }
    }
    if constexpr (kSplit) {
      // one layer: issue its MMAs (one thread), wait (bounded), make TMEM visible
      auto layer = [&](uint32_t d_tm, uint32_t a_sm, uint32_t b_sm, uint32_t id, int steps) -> bool {
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after_sync();
          for (int kk = 0; kk < steps; ++kk)
            Op::mma(d_tm, tc::desc_sw128(a_sm + 32 * kk), tc::desc_sw128(b_sm + 32 * kk), id, kk);
          tc::mma_commit(mbar);
        }
        const bool done = tc::mbar_wait_bounded(mbar, phase, kSpinLimit);
        phase ^= 1;
        if (__syncthreads_or(!done)) return false;
        tc::fence_after_sync();
        return true;
      };
      float v[16];
      // density: D1 = X Wd1 -> relu -> A1; G = A1 Wd2 (columns 64..79)
      if (!layer(tmem, a0, b1, idesc64, kSteps32)) { failed = true; break; }
      if (kRec) store_feat_record(t);  // A0 holds X until the colour input overwrites it
      tc::tmem_ld16(tmem_q + 16 * g, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
      Op::store16(a1, row, g, v);
      if (!layer(tmem + 64, a1, b3, idesc16, kSteps64)) { failed = true; break; }
      // colour input [G | SH(d)] -> A0 columns 0..31
      float g0 = 0.0f;
      if (g == 0) {
        tc::tmem_ld16(tmem_q + 64, v);
        tc::tmem_ld_wait();
        g0 = v[0];
        Op::store16(a0, row, 0, v);
      } else if (g == 1) {
        float sh[kSh];
        sh4_f32(dir, sh);
        Op::store16(a0, row, 1, sh);
      }
      if (!layer(tmem, a0, c1, idesc64, kSteps32)) { failed = true; break; }
      tc::tmem_ld16(tmem_q + 16 * g, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
      Op::store16(a1, row, g, v);
      if (!layer(tmem + 64, a1, b2, idesc64, kSteps64)) { failed = true; break; }
      tc::tmem_ld16(tmem_q + 64 + 16 * g, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
      Op::store16(a0, row, g, v);
      if (!layer(tmem, a0, c3, idesc16, kSteps64)) { failed = true; break; }
      if (g == 0) {
        tc::tmem_ld16(tmem_q, v);
        tc::tmem_ld_wait();
        if (chunk_ok) {
          float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
          if (valid) {
            sigma = expf(g0);
#pragma unroll
            for (int j = 0; j < 3; ++j) rgb[j] = 1.0f / (1.0f + expf(-v[j]));
          }
          const Partial pt = render_chunk(sigma, rgb, tr, dl, sl.sl, nullptr, kTcRows, sl.width);
          if (sl.has && sl.sl == 0) {
            float4* dst = p.partials + 2 * ((size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c);
            dst[0] = make_float4(pt.tau, pt.c0, pt.c1, pt.c2);
            dst[1] = make_float4(pt.A, pt.D, pt.L, 0.0f);
          }
        }
      }
      tc::fence_before_sync();  // no barrier: as at the end of the fused form's tile below
      continue;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- layer 1
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kSteps32; ++kk)
        Op::mma(tmem, tc::desc_sw128(a0 + 32 * kk), tc::desc_sw128(b1 + 32 * kk), idesc64, kk);
      tc::mma_commit(mbar);
    }
    if (kRec) store_feat_record(t);  // while the layer-1 MMA runs (it only reads A0)
    bool ok = tc::mbar_wait_bounded(mbar, phase, kSpinLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    float v[16];
    tc::tmem_ld16(tmem_q + 16 * g, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] * scale[0], 0.0f);
    Op::store16(a1, row, g, v);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- layer 2
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kSteps64; ++kk)
        Op::mma(tmem + 64, tc::desc_sw128(a1 + 32 * kk), tc::desc_sw128(b2 + 32 * kk), idesc64, kk);
      tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait_bounded(mbar, phase, kSpinLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    tc::tmem_ld16(tmem_q + 64 + 16 * g, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] * scale[1], 0.0f);
    Op::store16(a0, row, g, v);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // ---- layer 3
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kSteps64; ++kk)
        Op::mma(tmem, tc::desc_sw128(a0 + 32 * kk), tc::desc_sw128(b3 + 32 * kk), idesc16, kk);
      tc::mma_commit(mbar);
    }
    ok = tc::mbar_wait_bounded(mbar, phase, kSpinLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // ---- chunk render by the warps of level group 0 (one slot per warp, scans segmented per chunk)
    if (g == 0) {
      tc::tmem_ld16(tmem_q, v);
      tc::tmem_ld_wait();
      if (chunk_ok) {
        float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
          sigma = expf(v[0] * scale[2]);
#pragma unroll
          for (int j = 0; j < 3; ++j) rgb[j] = 1.0f / (1.0f + expf(-v[1 + j] * scale[2]));
        }
        const Partial pt = render_chunk(sigma, rgb, tr, dl, sl.sl,
                                        kRec ? p.rec.geom + (size_t)t * kGeomFloats + 5 * kTcRows + row : nullptr,
                                        kTcRows, sl.width);
        if (kRec) {
          float* geo = p.rec.geom + (size_t)t * kGeomFloats;
          __stcs(geo + 8 * kTcRows + row, sigma);
#pragma unroll
          for (int j = 0; j < 3; ++j) __stcs(geo + (9 + j) * kTcRows + row, rgb[j]);
        }
        if (sl.has && sl.sl == 0) {
          float4* dst = p.partials + 2 * ((size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c);
          dst[0] = make_float4(pt.tau, pt.c0, pt.c1, pt.c2);
          dst[1] = make_float4(pt.A, pt.D, pt.L, 0.0f);
        }
      }
    }
    // No barrier here: the warps of level groups 1-3 start the next tile's
    // gather while those of group 0 render this one. The A tiles are free
    // (every MMA of this tile has completed), and the next layer-1 MMA, which
    // overwrites the TMEM columns the render reads, is issued only after the
    // barrier that ends the next gather, which the render warps reach after
    // their TMEM reads (fenced before it).
    tc::fence_before_sync();
  }
  if (failed && tid == 0) atomicOr(p.err, kErrTimeout);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Host dispatch (called from nerfxl_render_fwd).
nerfxl_status launch_field_fwd_tc(const nerfxl_field* f, const SampParams& sp, const LevelParams& lp,
                                  const float* rays_o, const float* rays_d, char* ws, const Layout& L,
                                  const RecordOut& rec, cudaStream_t stream) {
  FwdTcParams p;
  p.rec = rec;
  p.rays_o = rays_o;
  p.rays_d = rays_d;
  p.boxes = f->boxes;
  p.tables = f->tables;
  p.mlp = f->mlp;
  p.mlp_scales = f->mlp_scales;
  p.lp = lp;
  p.sp = sp;
  p.K = f->K;
  p.hdr = reinterpret_cast<const RayHdr*>(ws + L.ray_hdr);
  p.segs = reinterpret_cast<const SegDesc*>(ws + L.segs);
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.chunks = reinterpret_cast<const Slot*>(ws + L.chunks);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.partials = reinterpret_cast<float4*>(ws + L.partials);
  p.err = reinterpret_cast<int32_t*>(ws + L.hdr);
  p.feat_in = nullptr;
  p.window = 0;
  p.w0 = 0;
  p.w1 = INT64_MAX;
  const size_t smem = kTcSmemFixed + sizeof(int32_t) * (f->K + 1);
  const int kind = f->mlp_dtype == NERFXL_BF16 ? kKindBF16 : (f->mlp_dtype == NERFXL_F16 ? kKindF16 : kKindE4M3);
  if (kind == kKindE4M3 && !f->mlp_scales) return set_error(NERFXL_E_INVALID, "E4M3 MLP needs mlp_scales");
  const bool f16tab = f->table_dtype == NERFXL_F16;
  const bool recs = rec.feat != nullptr;
  if (recs && kind == kKindE4M3) return set_error(NERFXL_E_UNSUPPORTED, "E4M3 is forward-only");
  const bool split = f->arch == NERFXL_ARCH_SPLIT;
  if (split && kind == kKindE4M3)
    return set_error(NERFXL_E_UNSUPPORTED, "the split representation's tensor-core form is a BF16/FP16 forward");
  const bool bf = kind == kKindBF16;
  const int64_t max_tiles = L.chunk_cap / kTcChunks;
  if (L.gfeat_tiles > 0) {
    // Level-grouped gather into the layout's window of level-major feature
    // words (the backward layout's when the forward writes records), then the
    // MLP and render from those words, window by window.
    uint32_t* feat = recs ? rec.gfeat : reinterpret_cast<uint32_t*>(ws + L.gfeat);
    const int64_t window = recs ? rec.gfeat_tiles : L.gfeat_tiles;
    if (!feat || window < 1) return set_error(NERFXL_E_WORKSPACE, "workspace has no feature tiles for the grouped gather");
    void (*kern)(FwdTcParams) = nullptr;
    if (split)
      kern = recs ? (bf ? k_field_fwd_tc<true, kKindBF16, true, true, true> : k_field_fwd_tc<true, kKindF16, true, true, true>)
                  : (bf ? k_field_fwd_tc<true, kKindBF16, false, true, true> : k_field_fwd_tc<true, kKindF16, false, true, true>);
    else
      kern = recs ? (bf ? k_field_fwd_tc<true, kKindBF16, true, false, true> : k_field_fwd_tc<true, kKindF16, true, false, true>)
                  : (bf ? k_field_fwd_tc<true, kKindBF16, false, false, true> : k_field_fwd_tc<true, kKindF16, false, false, true>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return launch_check("k_field_fwd_tc smem attribute");
    profile_mark(0, stream);
    for (int64_t w0 = 0; w0 < max_tiles; w0 += window) {
      const int64_t w1 = std::min(max_tiles, w0 + window);
      nerfxl_status st = launch_gather_groups(f, sp, lp, rays_o, rays_d, ws, L, feat, window, w0, w1, stream);
      if (st != NERFXL_OK) return st;
      p.feat_in = feat;
      p.window = window;
      p.w0 = w0;
      p.w1 = w1;
      kern<<<fwd_grid(w1 - w0, 2), kTcThreads, smem, stream>>>(p);
      st = kernel_launched("k_field_fwd_tc");
      if (st != NERFXL_OK) return st;
    }
    profile_mark(1, stream);
    return NERFXL_OK;
  }
  void (*kern)(FwdTcParams) = nullptr;
  if (split) {
    if (f16tab)
      kern = recs ? (bf ? k_field_fwd_tc<true, kKindBF16, true, true> : k_field_fwd_tc<true, kKindF16, true, true>)
                  : (bf ? k_field_fwd_tc<true, kKindBF16, false, true> : k_field_fwd_tc<true, kKindF16, false, true>);
    else
      kern = recs ? (bf ? k_field_fwd_tc<false, kKindBF16, true, true> : k_field_fwd_tc<false, kKindF16, true, true>)
                  : (bf ? k_field_fwd_tc<false, kKindBF16, false, true> : k_field_fwd_tc<false, kKindF16, false, true>);
  } else if (f16tab) {
    if (recs) kern = kind == kKindBF16 ? k_field_fwd_tc<true, kKindBF16, true, false> : k_field_fwd_tc<true, kKindF16, true, false>;
    else
      kern = kind == kKindBF16 ? k_field_fwd_tc<true, kKindBF16, false, false>
                               : (kind == kKindF16 ? k_field_fwd_tc<true, kKindF16, false, false>
                                                   : k_field_fwd_tc<true, kKindE4M3, false, false>);
  } else {
    if (recs) kern = kind == kKindBF16 ? k_field_fwd_tc<false, kKindBF16, true, false> : k_field_fwd_tc<false, kKindF16, true, false>;
    else
      kern = kind == kKindBF16 ? k_field_fwd_tc<false, kKindBF16, false, false>
                               : (kind == kKindF16 ? k_field_fwd_tc<false, kKindF16, false, false>
                                                   : k_field_fwd_tc<false, kKindE4M3, false, false>);
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return launch_check("k_field_fwd_tc smem attribute");
  const int grid = fwd_grid(max_tiles, 2);
  profile_mark(0, stream);
  kern<<<grid, kTcThreads, smem, stream>>>(p);
  profile_mark(1, stream);
  return kernel_launched("k_field_fwd_tc");
}

}  // namespace nerfxl
