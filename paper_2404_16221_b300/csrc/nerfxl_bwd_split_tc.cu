// Backward of the split representation on the tensor cores (16-bit MLPs,
// FP32 accumulation in tensor memory). One CTA of 12 warps per SM takes
// 128-row tiles (4 chunk slots of one region), in two roles:
//   compute warps 0-7   the MMA chain of one tile at a time; warp w serves
//                       rows 32 (w % 4) + lane (its TMEM lane quarter) and
//                       columns 32 (w / 4) .. + 31 of the 64-wide products
//   scatter warps 8-11  scatter the previous tile's dL/dX into the region's
//                       table gradient: warp 8 + w moves lane quarter w's 32
//                       columns of one of two dL/dX buffers in TMEM into a
//                       shared staging, then each thread takes two levels of 8
//                       consecutive rows and sends one set of reductions per
//                       run of samples in the same cell, while the compute
//                       warps run the next tile; hand-off through full / empty
//                       mbarriers. Four scatter warps contend less with the
//                       chain than eight (16.3 against 19.9 ms per grid8 step)
// The table scatter is bound by the SM's rate for scattered vector atomics,
// so it runs beside the chain instead of on its critical path. Per tile:
//   records   written by the forward for this tile: X exactly as its first
//             MMA read it; per row the region coordinates, interval and ray
//             direction; per chunk the sample count and, from the composite
//             adjoint, the chunk's partial adjoints in tile order. One thread
//             bulk-copies the next tile's records into the other of two
//             shared-memory stages while this tile runs.
//   density   D = X Wd1 -> H1 = relu; G = H1 Wd2 (N = 16)
//   colour    Xc = [G | SH(d)]; D = Xc Wc1 -> Hc1; D = Hc1 Wc2 -> Hc2; o = Hc2 Wc3
//   adjoint   sigma = exp(G0), rgb = sigmoid(o); chunk-local render adjoint
//             (one warp per slot, scans segmented per chunk) -> dL/d(colour
//             logits) goC, dL/dG0
//   colour    Gz2 = (Hc2 > 0) (goC Wc3^T); Gz1 = (Hc1 > 0) (Gz2 Wc2^T);
//             dG = (Gz1 Wc1^T)[0..15] + dL/dG0 e0
//   density   Gz0 = (H1 > 0) (dG Wd2^T); dX = Gz0 Wd1^T into TMEM buffer
//             (tile & 1) -> table scatter-add by the scatter warps
//   weights   DW3 += [Hc2 | Hc1]^T goC, DWc += [Gz2 | Gz1]^T [Hc1 | Xc],
//             DWd += [Gz0 | dG]^T [X | H1], MN-major reads of the row-major
//             activation tiles (the samples are the contraction); DW3 and
//             DWc run behind the next chain step, DWd under the tile's last
//             commit; accumulated in TMEM over a region's tiles and flushed
//             at region changes (density block of the region, shared colour
//             block) by atomics.
// The transposed weights of the dX products are MN-major reads of the
// forward's weight tiles (K = the layer's output index), except the two with
// 32 outputs (Wc1^T and Wd1^T), staged K-major. Gradients enter the products
// as single 16-bit values.
// Every wait is bounded: on expiry the kernel flags kErrTimeout, frees its
// tensor memory and returns. One compute-warp barrier per MMA step: it
// publishes the step's shared-memory operands and carries any timed-out wait
// of the step before; each compute thread waits on the commit itself.

#include <cuda_runtime.h>

#include "nerfxl_half.cuh"
#include "nerfxl_host.h"
#include "nerfxl_scatter.cuh"
#include "nerfxl_split.cuh"
#include "nerfxl_tc.cuh"

namespace nerfxl {
namespace {

constexpr int kRowsS = 128;
constexpr int kThreadsS = 384;
constexpr int kGroupS = 256;  // compute threads
constexpr int kScatS = 128;   // scatter threads
constexpr int kBarComputeS = 1, kBarScatterS = 2;
constexpr int kChunksS = kRowsS / kWarp;
// TMEM columns: 0 D_A, 64 D_B, 128 D_S (N <= 32), 192 DWc, 288 DWd, 384 DW3, 416 and 448 dX (two buffers)
constexpr uint32_t kColsS = 512;
constexpr uint32_t kDA = 0, kDB = 64, kDS = 128, kDWc = 192, kDWd = 288, kDW3 = 384, kDX = 416;
constexpr uint32_t kSpinS = 1u << 24;
constexpr uint32_t kTile = 128 * 128;  // one 128-row, 128-byte-swizzled tile

// Shared-memory plan (offsets from a 1024-byte-aligned base).
constexpr uint32_t oX = 0;                 // SW64 [128][32]: features, record stage 0
constexpr uint32_t oXc = oX + 8192;        // SW64 [128][32]: [G | SH]
constexpr uint32_t oH1 = oXc + 8192;       // SW128 [128][64]
constexpr uint32_t oHc2 = oH1 + kTile;     // SW128, then Hc1 right after (DW3's A = [Hc2 | Hc1])
constexpr uint32_t oHc1 = oHc2 + kTile;
constexpr uint32_t oGoC = oHc1 + kTile;    // SW128, 16 columns used
constexpr uint32_t oGz2 = oGoC + kTile;    // [Gz2 | Gz1]: DWc's A
constexpr uint32_t oGz1 = oGz2 + kTile;
constexpr uint32_t oGz0 = oGz1 + kTile;    // [Gz0 | dG]: DWd's A
constexpr uint32_t oGG = oGz0 + kTile;     // 16 columns used
constexpr uint32_t oWd1 = oGG + kTile;     // B: 64 rows (out) x 32 (in), SW128
constexpr uint32_t oWd2 = oWd1 + 64 * 128;  // B: 16 rows x 64
constexpr uint32_t oWc1 = oWd2 + 16 * 128;  // B: 64 rows x 32
constexpr uint32_t oWc2 = oWc1 + 64 * 128;  // B: 64 rows x 64
constexpr uint32_t oWc3 = oWc2 + 64 * 128;  // B: 16 rows x 64 (rows >= 4 zero)
constexpr uint32_t oWd1t = oWc3 + 16 * 128;  // B of dX: 32 rows (in) x 64 (out), K-major
constexpr uint32_t oWc1t = oWd1t + 32 * 128;  // B of dXc: 32 rows (in) x 64 (out)
constexpr uint32_t oX1 = oWc1t + 32 * 128;    // SW64 [128][32]: features, record stage 1
// Geometry + chunk adjoints of record stages 0, 1 (the bulk copies' images).
constexpr uint32_t kGeoBytesS = 4 * kGeomFloats;
constexpr uint32_t kGeoStageS = kGeoBytesS + 2 * 16 * 16;  // + 16 chunk positions (4 per slot) x 2 float4
constexpr uint32_t oGeoS = oX1 + 8192;
constexpr uint32_t kStageTxS = 8192 + kGeoStageS;  // bytes per stage fill
// Hand-off slots 0, 1 from the compute to the scatter warps (dL/dX itself
// stays in TMEM): the rows' region coordinates u as float [3][128], the 4
// chunk slots' count words, the region.
constexpr uint32_t oHandS = oGeoS + 2 * kGeoStageS;
constexpr uint32_t kHdUS = 0, kHdNvS = 3 * 4 * kRowsS, kHdRegionS = kHdNvS + 16;
constexpr uint32_t kHandS = kHdRegionS + 16;
// The scatter warps' staging of one tile's dL/dX out of tensor memory: float4
// [8 = level pairs][128 rows], row r at position srow(r) (and u likewise in the
// hand-off slot), so that the row-wise writes and the run threads' reads (rows
// 8 apart) both spread over the banks.
constexpr uint32_t oDxS = oHandS + 2 * kHandS;
constexpr uint32_t kDxBytesS = 16 * 8 * kRowsS;
constexpr uint32_t oMiscS = (oDxS + kDxBytesS + 63) / 64 * 64;  // 8 mbarriers, TMEM base, abort flag
constexpr uint32_t oBaseS = oMiscS + 128;
constexpr size_t kSmemS = oBaseS + 1024;
static_assert(kRowsS == kRecRows, "one backward tile is one record tile");
static_assert(oX1 % 1024 == 0, "X stages keep the swizzle phase");
static_assert(kGeoBytesS % 16 == 0 && kGeoStageS % 16 == 0 && oGeoS % 16 == 0, "bulk copies need 16 B");
static_assert(oHandS % 16 == 0 && kHandS % 16 == 0 && oDxS % 16 == 0, "hand-off slot alignment");
static_assert(kDX + 64 <= kColsS, "tensor memory columns");
static_assert(kSmemS + 1024 + 4 * 1024 <= 232448, "shared memory");

struct BwdSplitTcParams {
  const void* mlp;  // 16-bit: K density blocks, then the colour block
  LevelParams lp;
  int K;
  const int32_t* base;
  const int32_t* n_tiles;
  const uint4* rec_feat;    // per tile: the 128 x 32 feature tile, 64-byte swizzled
  const float* rec_geom;    // per tile: rows u0 u1 u2 tr dl d0 d1 d2 (of kGeomRowFields), chunk counts
  const float4* rec_dpart;  // per tile: 16 chunk positions (4 per slot) x 2 partial adjoints
  float* grad_tables;
  float* grad_mlp;
  int32_t* err;
};

// Position of row r in the scatter's row-major staging (an XOR swizzle of the
// row's low three bits with its group of eight).
__device__ __forceinline__ uint32_t srow(uint32_t r) { return r ^ ((r >> 3) & 7u); }

// 16-byte chunk c of row r of a 64-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw64_chunk(uint32_t row, uint32_t c) {
  return row * 64u + ((c ^ ((row >> 1) & 3u)) << 4);
}

template <bool kBF16>
__device__ __forceinline__ void st_chunk8(uint32_t addr, const float* f) {
  tc::st_shared_v4(addr, Half2Of<kBF16>::pack(f[0], f[1]), Half2Of<kBF16>::pack(f[2], f[3]),
                   Half2Of<kBF16>::pack(f[4], f[5]), Half2Of<kBF16>::pack(f[6], f[7]));
}

// Sixteen values -> columns 16 c .. 16 c + 15 of a 128-byte-swizzled row.
template <bool kBF16>
__device__ __forceinline__ void st_row16(uint32_t tile, uint32_t row, int c, const float* v) {
  st_chunk8<kBF16>(tile + tc::sw128_chunk(row, 2 * c), v);
  st_chunk8<kBF16>(tile + tc::sw128_chunk(row, 2 * c + 1), v + 8);
}

// B tiles of the forward products (row = output n, column = input k) and the
// K-major transposed tiles of the two dX products with 32 outputs.
template <bool kBF16>
__device__ void load_density_bwd(const void* blk, char* sm, int tid, int nthreads) {
  uint16_t* wd1 = reinterpret_cast<uint16_t*>(sm + oWd1);
  uint16_t* wd2 = reinterpret_cast<uint16_t*>(sm + oWd2);
  uint16_t* wd1t = reinterpret_cast<uint16_t*>(sm + oWd1t);
  for (int i = tid; i < kIn * kWidth; i += nthreads) {
    const int k = i / kWidth, n = i % kWidth;  // Wd1[k][n]
    const uint16_t b = Half2Of<kBF16>::bits(blk, i);
    wd1[tc::sw128_offset(n, k) >> 1] = b;
    wd1t[tc::sw128_offset(k, n) >> 1] = b;
  }
  for (int i = tid; i < kGeo * kWidth; i += nthreads) {
    const int n = i / kWidth, k = i % kWidth;  // B row n = output n of Wd2 [64][16]
    wd2[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, kIn * kWidth + k * kGeo + n);
  }
}

template <bool kBF16>
__device__ void load_color_bwd(const void* blk, char* sm, int tid, int nthreads) {
  uint16_t* wc1 = reinterpret_cast<uint16_t*>(sm + oWc1);
  uint16_t* wc2 = reinterpret_cast<uint16_t*>(sm + oWc2);
  uint16_t* wc3 = reinterpret_cast<uint16_t*>(sm + oWc3);
  uint16_t* wc1t = reinterpret_cast<uint16_t*>(sm + oWc1t);
  for (int i = tid; i < kColorIn * kWidth; i += nthreads) {
    const int k = i / kWidth, n = i % kWidth;  // Wc1[k][n]
    const uint16_t b = Half2Of<kBF16>::bits(blk, i);
    wc1[tc::sw128_offset(n, k) >> 1] = b;
    wc1t[tc::sw128_offset(k, n) >> 1] = b;
  }
  for (int i = tid; i < kWidth * kWidth; i += nthreads) {
    const int k = i / kWidth, n = i % kWidth;
    wc2[tc::sw128_offset(n, k) >> 1] = Half2Of<kBF16>::bits(blk, kColorIn * kWidth + i);
  }
  for (int i = tid; i < 16 * kWidth; i += nthreads) {
    const int n = i / kWidth, k = i % kWidth;
    wc3[tc::sw128_offset(n, k) >> 1] =
        n < 3 ? Half2Of<kBF16>::bits(blk, kColorIn * kWidth + kWidth * kWidth + k * kOut + n) : 0;
  }
}

template <bool kBF16>
__global__ void __launch_bounds__(kThreadsS, 1) k_field_bwd_split_tc(BwdSplitTcParams p) {
  extern __shared__ __align__(1024) char s_raw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = tc::smem_u32(sm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + oMiscS);  // MMA completion
  uint64_t* full = mbar + 1;                                   // record stages 0, 1 filled
  uint64_t* hfull = mbar + 3;                                  // hand-off slots 0, 1 written
  uint64_t* hempty = mbar + 5;                                 // hand-off slots 0, 1 read
  uint64_t* drain = mbar + 7;                                  // error path: all MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + oMiscS + 64);
  volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(sm + oMiscS + 68);
  int32_t* s_base = reinterpret_cast<int32_t*>(sm + oBaseS);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;

  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  // zero the activation and gradient tiles once (unused columns of the
  // 16-column tiles feed rows of the weight gradients that are never read)
  for (uint32_t i = tid; i < oWd1 / 16; i += blockDim.x) tc::st_shared_v4(sb + 16 * i, 0u, 0u, 0u, 0u);
  load_color_bwd<kBF16>(static_cast<const char*>(p.mlp) + (size_t)p.K * kDensityParams * 2, sm, tid, blockDim.x);
  if (warp == 0) tc::tmem_alloc(tmem_slot, kColsS);
  if (tid == 0) {
    for (int i = 0; i < 8; ++i) tc::mbar_init(mbar + i, 1);
    *s_abort = 0;
  }
  tc::fence_proxy_async();  // the zeroed stage-0 tile before the first record copy overwrites it
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int n_sub = *p.n_tiles * (kChunksPerTile / kChunksS);
  const int G = (int)gridDim.x;

  if (warp >= kGroupS / kWarp) {
    // ===================== scatter warps =====================
    // Warp w = warp - 8 first moves its TMEM lane quarter's dL/dX (rows 32 w .. 32 w + 31,
    // all 16 levels) into the shared staging. Then warp w takes levels 4 w .. 4 w + 3,
    // one after the other: lane pair (lanes 2v, 2v + 1) takes 8 consecutive rows of a chunk slot
    // (window v: slot qq = v / 4, rows 8 (v % 4) ..), one lane per x-half of the cell
    // corners, and sends one set of reductions per run of samples in the same cell,
    // the two halves of an x-pair in the same instructions (nearly rolled loops,
    // see k_field_bwd_tc).
    const int sw = warp - kGroupS / kWarp, q = sw;
    const uint32_t row = (uint32_t)(q * kWarp + lane);
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    const int hx = lane & 1, qq = lane >> 3, wd = (lane >> 1) & 3;
    float4* sdx = reinterpret_cast<float4*>(sm + oDxS);
    int it = 0;
    for (int t = blockIdx.x; t < n_sub; t += G, ++it) {
      const int b = it & 1;
      const bool ok = tc::mbar_wait_bounded(hfull + b, (uint32_t)(it >> 1) & 1u, kSpinS);
      if (tc::bar_or(kBarScatterS, kScatS, !ok || *s_abort != 0)) {
        if (!ok && tid == kGroupS) atomicOr(p.err, kErrTimeout);
        break;
      }
      tc::fence_after_sync();
      for (int h = 0; h < 2; ++h) {
        float gx[16];
        tc::tmem_ld16(tq + kDX + 32 * (uint32_t)b + 16 * (uint32_t)h, gx);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 4; ++j)
          sdx[(4 * h + j) * kRowsS + srow(row)] = make_float4(gx[4 * j], gx[4 * j + 1], gx[4 * j + 2], gx[4 * j + 3]);
      }
      const char* hd = sm + oHandS + (uint32_t)b * kHandS;
      const float* hu = reinterpret_cast<const float*>(hd + kHdUS);
      const int32_t nw = reinterpret_cast<const int32_t*>(hd + kHdNvS)[qq];
      const int k = *reinterpret_cast<const int32_t*>(hd + kHdRegionS);
      tc::fence_before_sync();
      tc::bar_sync(kBarScatterS, kScatS);  // the staging holds the tile's dL/dX
      uint32_t vmask = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const SlotCount sc = slot_count(nw, 8 * wd + i);
        vmask |= (sc.sl < sc.n ? 1u : 0u) << i;
      }
      const uint32_t r0 = (uint32_t)(qq * kWarp + 8 * wd);
      float2* gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
      const float2* sdx2 = reinterpret_cast<const float2*>(sdx);
#pragma unroll 1
      for (int e = 0; e < 4 && vmask != 0u; ++e) {
        const int l = 4 * sw + e;
        if (l >= p.lp.L) break;
        const float2* dl = sdx2 + 2 * (size_t)(l >> 1) * kRowsS + (l & 1);  // row r: dl[2 srow(r)]
        scatter_runs_half<8, true>(
            p.lp, gtab, l, hx, vmask,
            [&](int i, float* ui) {
              const uint32_t r = srow(r0 + (uint32_t)i);
#pragma unroll
              for (int ax = 0; ax < 3; ++ax) ui[ax] = hu[ax * kRowsS + r];
            },
            [&](int i) { return dl[2 * srow(r0 + (uint32_t)i)]; });
      }
      tc::fence_before_sync();
      tc::bar_sync(kBarScatterS, kScatS);  // slot and TMEM buffer read by every scatter thread
      if (tid == kGroupS) tc::mbar_arrive(hempty + b);
    }
  } else {
    // ===================== compute warps =====================
    // warp (q, g): rows 32 q .. 32 q + 31, columns 32 g .. 32 g + 31 of the 64-wide products
    const int q = warp & 3, g = warp >> 2;
    const uint32_t row = (uint32_t)(q * kWarp + lane);
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    constexpr uint32_t id64 = tc::idesc_f16(kBF16, kRowsS, 64);
    constexpr uint32_t id32 = tc::idesc_f16(kBF16, kRowsS, 32);
    constexpr uint32_t id16 = tc::idesc_f16(kBF16, kRowsS, 16);
    constexpr uint32_t id64_bt = id64 | tc::kMnMajorB;
    constexpr uint32_t id64_abt = id64 | tc::kMnMajorA | tc::kMnMajorB;
    constexpr uint32_t id32_abt = id32 | tc::kMnMajorA | tc::kMnMajorB;
    constexpr uint32_t id16_abt = id16 | tc::kMnMajorA | tc::kMnMajorB;

    int region = -1;
    uint32_t phase = 0;
    bool failed = false, dw_started = false;

    // One compute barrier per step: it publishes the step's shared-memory
    // operands and agrees on any earlier timed-out wait; every compute thread
    // then waits on the step's commit itself.
    bool timed_out = false;
    auto step = [&](auto&& issue) -> bool {
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (tc::bar_or(kBarComputeS, kGroupS, timed_out)) return false;
      if (tid == 0) {
        tc::fence_after_sync();
        issue();
      }
      timed_out = !tc::mbar_wait_bounded(mbar, phase, kSpinS);
      phase ^= 1;
      tc::fence_after_sync();
      return true;
    };
    // relu of this thread's 32 columns of accumulator `col` -> 16-bit tile;
    // returns the mask of positive values
    auto relu_store = [&](uint32_t col, uint32_t tile) -> uint32_t {
      float v[32];
      tc::tmem_ld16(tq + col + 32 * g, v);
      tc::tmem_ld16(tq + col + 32 * g + 16, v + 16);
      tc::tmem_ld_wait();
      uint32_t m = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (v[i] > 0.0f) m |= 1u << i;
        else v[i] = 0.0f;
      }
      st_row16<kBF16>(tile, row, 2 * g, v);
      st_row16<kBF16>(tile, row, 2 * g + 1, v + 16);
      return m;
    };
    // this thread's 32 columns of accumulator `col`, zero where `mask` is clear -> 16-bit tile
    auto mask_store = [&](uint32_t col, uint32_t tile, uint32_t mask) {
      float v[32];
      tc::tmem_ld16(tq + col + 32 * g, v);
      tc::tmem_ld16(tq + col + 32 * g + 16, v + 16);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (!((mask >> i) & 1u)) v[i] = 0.0f;
      st_row16<kBF16>(tile, row, 2 * g, v);
      st_row16<kBF16>(tile, row, 2 * g + 1, v + 16);
    };

    // weight-gradient accumulators -> global (all MMAs complete)
    auto flush = [&]() {
      if (!dw_started) return;
      tc::fence_after_sync();
      float* gd = p.grad_mlp + (size_t)region * kDensityParams;
      float* gc = p.grad_mlp + (size_t)p.K * kDensityParams;
      const int r = (int)row;
      float v[16];
      for (int hh = g; hh < 6; hh += 2) {  // DWc: 96 columns
        tc::tmem_ld16(tq + kDWc + 16 * hh, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = 16 * hh + i;
          if (r < 64 && c < 64) atomicAdd(gc + kColorIn * kWidth + c * kWidth + r, v[i]);          // dWc2[c][r]
          else if (r >= 64 && c >= 64) atomicAdd(gc + (c - 64) * kWidth + (r - 64), v[i]);        // dWc1[c-64][r-64]
        }
      }
      for (int hh = g; hh < 6; hh += 2) {  // DWd: 96 columns
        tc::tmem_ld16(tq + kDWd + 16 * hh, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = 16 * hh + i;
          if (r < 64 && c < 32) atomicAdd(gd + c * kWidth + r, v[i]);                                // dWd1[c][r]
          else if (r >= 64 && r < 64 + kGeo && c >= 32) atomicAdd(gd + kIn * kWidth + (c - 32) * kGeo + (r - 64), v[i]);
        }
      }
      if (g == 0) {  // DW3: rows 0..63 = Hc2 index, columns 0..2
        tc::tmem_ld8(tq + kDW3, v);
        tc::tmem_ld_wait();
        if (r < 64)
#pragma unroll
          for (int m = 0; m < 3; ++m) atomicAdd(gc + kColorIn * kWidth + kWidth * kWidth + r * kOut + m, v[m]);
      }
      dw_started = false;
    };

    // Thread kCopier issues the record copies (thread 0 issues the MMAs);
    // pend0 / pend1 = iteration whose records are in flight into stage 0 / 1 (-1: none).
    constexpr int kCopier = kWarp;
    int pend0 = -1, pend1 = -1;
    auto issue = [&](int it, int t) {
      const int s = it & 1;
      tc::fence_proxy_async();  // order earlier generic accesses of the stage before the overwrite
      tc::mbar_expect_tx(full + s, kStageTxS);
      const uint32_t geo = sb + oGeoS + (uint32_t)s * kGeoStageS;
      const uint64_t pol = tc::policy_evict_first();  // read once: keep the gradient lines in L2
      tc::bulk_g2s_hint(sb + (s ? oX1 : oX), p.rec_feat + (size_t)t * (kRecFeatBytes / 16), 8192, full + s, pol);
      tc::bulk_g2s_hint(geo, p.rec_geom + (size_t)t * kGeomFloats, kGeoBytesS, full + s, pol);
      tc::bulk_g2s_hint(geo + kGeoBytesS, p.rec_dpart + (size_t)t * 32, 512, full + s, pol);
      (s ? pend1 : pend0) = it;
    };
    if (tid == kCopier && (int)blockIdx.x < n_sub) issue(0, blockIdx.x);

    int it = 0;
    for (int t = blockIdx.x; t < n_sub; t += G, ++it) {
      const int k = region_of_chunk(s_base, p.K, t * kChunksS);
      const int s = it & 1;
      if (k != region) {
        flush();
        tc::fence_before_sync();
        tc::bar_sync(kBarComputeS, kGroupS);
        load_density_bwd<kBF16>(static_cast<const char*>(p.mlp) + (size_t)k * kDensityParams * 2, sm, tid, kGroupS);
        region = k;
      }
      // ---- the next tile's records into the other stage (free: its last readers,
      //      the previous tile's first and last MMAs, have completed)
      if (tid == kCopier && t + G < n_sub) issue(it + 1, t + G);
      // ---- this tile's records: X (the record is the tile's shared-memory image,
      //      read in place by the MMAs), the row's region coordinates (for the
      //      hand-off), interval (render adjoint, g == 0) and direction (SH,
      //      g == 1), the chunk's adjoints
      if (!tc::mbar_wait_bounded(full + s, (uint32_t)(it >> 1) & 1u, kSpinS)) timed_out = true;
      else if (tid == kCopier) (s ? pend1 : pend0) = -1;
      const uint32_t xs = sb + (s ? oX1 : oX);
      const float* geo = reinterpret_cast<const float*>(sm + oGeoS + (uint32_t)s * kGeoStageS);
      const float4* dps = reinterpret_cast<const float4*>(sm + oGeoS + (uint32_t)s * kGeoStageS + kGeoBytesS);
      const int32_t nword = reinterpret_cast<const int32_t*>(geo + kGeomRowFields * kRecRows)[q];
      const SlotCount sc = slot_count(nword, lane);
      const bool chunk_ok = nword != 0, valid = sc.sl < sc.n;  // chunk_ok: warp-uniform
      float tr = 0.0f, dl = 0.0f, dir[3] = {0.0f, 0.0f, 0.0f};
      float gtc = 0.0f, gC[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f, gD = 0.0f, gL = 0.0f;
      if (g == 0) {
        tr = geo[3 * kRecRows + row];
        dl = geo[4 * kRecRows + row];
        if (chunk_ok && sc.n > 0) {  // (an unused part of the slot keeps zero adjoints)
          const float4 a0 = dps[2 * (4 * q + sc.part)], a1 = dps[2 * (4 * q + sc.part) + 1];
          gtc = a0.x;
          gC[0] = a0.y;
          gC[1] = a0.z;
          gC[2] = a0.w;
          gA = a1.x;
          gD = a1.y;
          gL = a1.z;
        }
      } else {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) dir[ax] = geo[(5 + ax) * kRecRows + row];
      }
      float v[16];
      // ---- density: D_A = X Wd1 -> H1
      if (!step([&] {
            for (int kk = 0; kk < 2; ++kk)
              tc::mma_f16(tmem + kDA, tc::desc_sw64(xs + 32 * kk, 16), tc::desc_sw128(sb + oWd1 + 32 * kk), id64,
                          kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      const uint32_t mH1 = relu_store(kDA, sb + oH1);
      // ---- G = H1 Wd2 (16 outputs) -> Xc = [G | SH(d)]
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDS, tc::desc_sw128(sb + oH1 + 32 * kk), tc::desc_sw128(sb + oWd2 + 32 * kk), id16,
                          kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      float g0 = 0.0f;
      if (g == 0) {
        tc::tmem_ld16(tq + kDS, v);
        tc::tmem_ld_wait();
        g0 = v[0];
        st_chunk8<kBF16>(sb + oXc + sw64_chunk(row, 0), v);
        st_chunk8<kBF16>(sb + oXc + sw64_chunk(row, 1), v + 8);
      } else {
        float sh[kSh];
        sh4_f32(dir, sh);
        st_chunk8<kBF16>(sb + oXc + sw64_chunk(row, 2), sh);
        st_chunk8<kBF16>(sb + oXc + sw64_chunk(row, 3), sh + 8);
      }
      // ---- colour: D_A = Xc Wc1 -> Hc1
      if (!step([&] {
            for (int kk = 0; kk < 2; ++kk)
              tc::mma_f16(tmem + kDA, tc::desc_sw64(sb + oXc + 32 * kk, 16), tc::desc_sw128(sb + oWc1 + 32 * kk),
                          id64, kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      const uint32_t mHc1 = relu_store(kDA, sb + oHc1);
      // ---- D_B = Hc1 Wc2 -> Hc2
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDB, tc::desc_sw128(sb + oHc1 + 32 * kk), tc::desc_sw128(sb + oWc2 + 32 * kk), id64,
                          kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      const uint32_t mHc2 = relu_store(kDB, sb + oHc2);
      // ---- o = Hc2 Wc3 (3 of 16 outputs)
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDS, tc::desc_sw128(sb + oHc2 + 32 * kk), tc::desc_sw128(sb + oWc3 + 32 * kk), id16,
                          kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      // ---- chunk-local render adjoint (warp g == 0 of each lane quarter = one slot)
      float go_d = 0.0f;
      if (g == 0) {
        tc::tmem_ld16(tq + kDS, v);
        tc::tmem_ld_wait();
        float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
          sigma = expf(g0);
#pragma unroll
          for (int m = 0; m < 3; ++m) rgb[m] = 1.0f / (1.0f + expf(-v[m]));
        }
        float g_sigma = 0.0f, g_rgb[3] = {0.0f, 0.0f, 0.0f};
        if (chunk_ok) render_chunk_adjoint(sigma, rgb, tr, dl, sc.sl, gtc, gC, gA, gD, gL, g_sigma, g_rgb, sc.width);
        float go[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) go[m] = 0.0f;
        if (valid) {
          go_d = g_sigma * sigma;
#pragma unroll
          for (int m = 0; m < 3; ++m) go[m] = g_rgb[m] * rgb[m] * (1.0f - rgb[m]);
        }
        st_row16<kBF16>(sb + oGoC, row, 0, go);
      }
      const bool acc = dw_started;
      // ---- Gz2 = (Hc2 > 0) goC Wc3^T (Wc3 tile read MN-major, K = 16); DW3 += [Hc2 | Hc1]^T goC behind it
      if (!step([&] {
            tc::mma_f16(tmem + kDA, tc::desc_sw128(sb + oGoC), tc::desc_sw128_mn(sb + oWc3, 1024), id64_bt, 0);
            tc::mma_commit(mbar);
            for (int kk = 0; kk < 8; ++kk)
              tc::mma_f16(tmem + kDW3, tc::desc_sw128_mn(sb + oHc2 + 2048 * kk, kTile),
                          tc::desc_sw128_mn(sb + oGoC + 2048 * kk, 1024), id16_abt, (acc || kk > 0) ? 1u : 0u);
          })) {
        failed = true;
        break;
      }
      mask_store(kDA, sb + oGz2, mHc2);
      // ---- Gz1 = (Hc1 > 0) Gz2 Wc2^T (Wc2 tile read MN-major, K = 64)
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDB, tc::desc_sw128(sb + oGz2 + 32 * kk),
                          tc::desc_sw128_mn(sb + oWc2 + 2048 * kk, 1024), id64_bt, kk);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      mask_store(kDB, sb + oGz1, mHc1);
      // ---- dXc = Gz1 Wc1^T (32 outputs; G's are the first 16); DWc += [Gz2 | Gz1]^T [Hc1 | Xc] behind it
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDS, tc::desc_sw128(sb + oGz1 + 32 * kk), tc::desc_sw128(sb + oWc1t + 32 * kk), id32,
                          kk);
            tc::mma_commit(mbar);
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t a = tc::desc_sw128_mn(sb + oGz2 + 2048 * kk, kTile);
              const uint32_t on = (acc || kk > 0) ? 1u : 0u;
              tc::mma_f16(tmem + kDWc, a, tc::desc_sw128_mn(sb + oHc1 + 2048 * kk, 1024), id64_abt, on);
              tc::mma_f16(tmem + kDWc + 64, a, tc::desc_sw64(sb + oXc + 1024 * kk, 512), id32_abt, on);
            }
          })) {
        failed = true;
        break;
      }
      if (g == 0) {
        tc::tmem_ld16(tq + kDS, v);
        tc::tmem_ld_wait();
        v[0] += go_d;  // G0 is also the log density
        st_row16<kBF16>(sb + oGG, row, 0, v);
      }
      // ---- Gz0 = (H1 > 0) dG Wd2^T (Wd2 tile read MN-major, K = 16)
      if (!step([&] {
            tc::mma_f16(tmem + kDA, tc::desc_sw128(sb + oGG), tc::desc_sw128_mn(sb + oWd2, 1024), id64_bt, 0);
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      mask_store(kDA, sb + oGz0, mH1);
      // ---- hand-off slot b: free once the scatter warps have read it (and TMEM buffer b) two tiles ago
      const int b = it & 1;
      if (it >= 2 && !tc::mbar_wait_bounded(hempty + b, (uint32_t)((it >> 1) + 1) & 1u, kSpinS)) timed_out = true;
      if (g == 0) {
        char* hd = sm + oHandS + (uint32_t)b * kHandS;
        float* hu = reinterpret_cast<float*>(hd + kHdUS);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) hu[ax * kRowsS + srow(row)] = geo[ax * kRecRows + row];
        if (lane == 0) reinterpret_cast<int32_t*>(hd + kHdNvS)[q] = nword;
        if (tid == 0) *reinterpret_cast<int32_t*>(hd + kHdRegionS) = k;
      }
      // ---- dX = Gz0 Wd1^T (32 outputs) into TMEM buffer b for the scatter warps, and
      //      DWd += [Gz0 | dG]^T [X | H1], under one commit: the next tile after next
      //      overwrites this stage's X at its start
      if (!step([&] {
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + kDX + 32 * (uint32_t)b, tc::desc_sw128(sb + oGz0 + 32 * kk),
                          tc::desc_sw128(sb + oWd1t + 32 * kk), id32, kk);
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t a = tc::desc_sw128_mn(sb + oGz0 + 2048 * kk, kTile);
              const uint32_t on = (acc || kk > 0) ? 1u : 0u;
              tc::mma_f16(tmem + kDWd, a, tc::desc_sw64(xs + 1024 * kk, 512), id32_abt, on);
              tc::mma_f16(tmem + kDWd + 32, a, tc::desc_sw128_mn(sb + oH1 + 2048 * kk, 1024), id64_abt, on);
            }
            tc::mma_commit(mbar);
          })) {
        failed = true;
        break;
      }
      dw_started = true;
      tc::fence_before_sync();
      if (tc::bar_or(kBarComputeS, kGroupS, timed_out)) {  // slot written, dX landed; tiles free for the next tile
        failed = true;
        break;
      }
      if (tid == 0) tc::mbar_arrive(hfull + b);
    }
    if (!failed) flush();  // every tile ends with all of its MMAs complete
    if (failed && tid == 0) {
      atomicOr(p.err, kErrTimeout);
      *s_abort = 1;  // wake the scatter warps; they see the flag and stop
      tc::mbar_arrive(hfull);
      tc::mbar_arrive(hfull + 1);
      // let MMAs still in flight land before the tensor memory is freed
      tc::mma_commit(drain);
      tc::mbar_wait_bounded(drain, 0u, kSpinS);
    }
    if (failed && tid == kCopier) {  // and the record copies still in flight
      if (pend0 >= 0) tc::mbar_wait_bounded(full, (uint32_t)(pend0 >> 1) & 1u, kSpinS);
      if (pend1 >= 0) tc::mbar_wait_bounded(full + 1, (uint32_t)(pend1 >> 1) & 1u, kSpinS);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kColsS);
}

}  // namespace

// Host dispatch (called from nerfxl_render_bwd for the split representation's
// 16-bit forms, after the composite adjoint wrote the tile-order chunk adjoints).
nerfxl_status launch_field_bwd_split_tc(const nerfxl_field* f, const LevelParams& lp, char* ws, const Layout& L,
                                        float* grad_tables, float* grad_mlp, cudaStream_t stream) {
  if (L.rec_tiles == 0) return set_error(NERFXL_E_WORKSPACE, "workspace has no tensor-core backward records");
  BwdSplitTcParams p;
  p.mlp = f->mlp;
  p.lp = lp;
  p.K = f->K;
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.rec_feat = reinterpret_cast<const uint4*>(ws + L.rec_feat);
  p.rec_geom = reinterpret_cast<const float*>(ws + L.rec_geom);
  p.rec_dpart = reinterpret_cast<const float4*>(ws + L.rec_dpart);
  p.grad_tables = grad_tables;
  p.grad_mlp = grad_mlp;
  p.err = reinterpret_cast<int32_t*>(ws + L.hdr);
  const size_t smem = kSmemS + sizeof(int32_t) * (f->K + 1);
  if (smem > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
  void (*kern)(BwdSplitTcParams) =
      f->mlp_dtype == NERFXL_BF16 ? k_field_bwd_split_tc<true> : k_field_bwd_split_tc<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return launch_check("k_field_bwd_split_tc smem attribute");
  const int grid = fwd_grid(L.chunk_cap / kChunksS, 1);
  profile_mark(0, stream);
  kern<<<grid, kThreadsS, smem, stream>>>(p);
  profile_mark(1, stream);
  return kernel_launched("k_field_bwd_split_tc");
}

}  // namespace nerfxl
