// Backward (adjoint) of the field with the MLP on the tensor cores: the
// mixed-precision forms (BF16/FP16 MLP, FP32 or FP16 tables; FP32 gradients).
//
// The kernel works from per-tile records in tile order, written by the
// tensor-core forward: every row's 16-bit features exactly as the forward's
// first MMA read them (already laid out as that MMA's 64-byte-swizzled A
// tile), its region coordinates u, position tr and length dl, the chunk-local
// Tn, w, distortion pair sum, sigma and rgb of the forward's render, each chunk's sample
// count, and (written by the composite backward) each chunk's partial
// adjoints. One thread copies the next tile's records into a second
// shared-memory stage with bulk asynchronous copies while the CTA works on the
// current tile, so no ray, segment or hash-table read sits between tiles.
//
// One CTA per SM, 16 warps in two roles. The table-gradient scatter is bound
// by the SM's throughput for scattered vector atomics (about one address per
// clock), so it runs concurrently with the MMA pipeline instead of after it:
//   compute warps 0-7   one 128-row tile (4 chunk slots of one region) at a time;
//                       warp w serves TMEM lane quarter q = w % 4 (rows
//                       32q..32q+31) and column half / level half g = w / 4
//   scatter warps 8-15  scatter the previous tile's dL/dfeatures, handed over
//                       through a double-buffered shared-memory slot guarded
//                       by full / empty mbarriers; a thread takes one level of
//                       8 consecutive rows and sends one set of reductions per
//                       run of samples in the same cell
// Per tile, on the compute warps (FP32 accumulation in TMEM, four MMA round
// trips):
//   1  D1 = X W1 (X straight from the record stage); meanwhile the chunk-local
//      render adjoint from the kept Tn, w, pair, sigma, rgb (one warp suffix
//      scan) -> g_o [128 x 4], stored as a 16-bit tile row [g_o hi | g_o lo | 0]
//   2  H1 = relu(D1); [g_o hi | g_o lo] [W3 | W3]^T (one K = 16 MMA, the G2 of
//      the next step before its mask); D2 = H1 W2
//   3  H2 = relu(D2), G2 = (H2 > 0) * that product; D4 = G2 W2^T, G1 = (H1 > 0) * D4
//   4  D5 = G1 W1^T = dL/dfeatures -> hand-off slot -> table scatter-add by the
//      scatter warps (vector atomics)
//   G2 and G1 enter the products as hi + lo pairs of 16-bit values (two MMAs
//   each), keeping ~16 mantissa bits of the upstream gradient; the weights are
//   exact in their 16-bit copy.
//   weights    DW  += [G2 | G1]^T [H1 | X]        (M = 128, N = 64 + 32, K = 128 samples)
//              DW3 += [H2 | H1]^T [g_o hi | g_o lo]  (M = 128, N = 16;
//                                                     dW3 = columns 0-3 + 4-7)
//              Both read the row-major activation tiles as MN-major operands
//              (the samples are the contraction), run behind the next step
//              (no wait: a later commit covers them before their operands are
//              overwritten), accumulate in TMEM over all of a region's tiles
//              and are flushed once per region: DW's diagonal blocks are dW2
//              and dW1, DW3's first 64 rows are dW3.
// Bounded waits flag kErrTimeout, wait (bounded) for copies still in flight,
// free tensor memory and return.

#include <cuda_runtime.h>

#include "nerfxl_field.cuh"
#include "nerfxl_half.cuh"
#include "nerfxl_host.h"
#include "nerfxl_scatter.cuh"
#include "nerfxl_tc.cuh"

namespace nerfxl {
namespace {

constexpr int kRows = kRecRows;
constexpr int kThreads = 512;
constexpr int kGroup = 256;  // threads per role
constexpr int kBarCompute = 1, kBarScatter = 2;
constexpr int kTileChunks = kRows / kWarp;
constexpr uint32_t kCols = 512;  // 0-63 D1/D5, 64-127 D2/D4, 128-223 DW, 224-239 DW3, 256-319 G2 before the mask
constexpr uint32_t kDwCol = 128, kDw3Col = 224, kG2Col = 256;
constexpr uint32_t kSpin = 1u << 24;

// Shared-memory plan (bytes from a 1024-aligned base). Activation tiles are
// 128 rows x 128 B (128-byte swizzle); pairs read as one MN-major operand of
// M = 128 sit one tile apart: (H2, H1) and (G2, G1).
constexpr uint32_t kTileBytes = 16384;
constexpr uint32_t oH2 = 0;
constexpr uint32_t oH1 = oH2 + kTileBytes;
constexpr uint32_t oG2 = oH1 + kTileBytes;    // G2, 16-bit rounding (hi part)
constexpr uint32_t oG1 = oG2 + kTileBytes;    // G1 hi
constexpr uint32_t oG2l = oG1 + kTileBytes;   // G2 - hi (lo part)
constexpr uint32_t oG1l = oG2l + kTileBytes;  // G1 lo
constexpr uint32_t oB1 = oG1l + kTileBytes;   // W1^T [64 rows z1][k = feature < 32]  (layer 1)
constexpr uint32_t oB2 = oB1 + 8192;          // W2^T [64 rows z2][k = h1] (layer 2; MN-major W2 for D4)
constexpr uint32_t oB5 = oB2 + 8192;          // W1 [32 rows feature][k = z1]
constexpr uint32_t oB6 = oB5 + 4096;          // [W3 | W3] [64 rows n][k: 0-3, 4-7 = W3[n][0..3], 8-15 zero]
constexpr uint32_t oGO = oB6 + 8192;          // g_o tile [128 rows][k: 0-3 hi, 4-7 lo, 8-15 zero]
// Record stages 0, 1: the feature tile X (64-byte swizzle, the A operand of
// layer 1 and the MN-major B operand of dW1), then geometry + chunk adjoints.
constexpr uint32_t oXs = oGO + kTileBytes;
constexpr uint32_t kXBytes = (uint32_t)kRecFeatBytes;
constexpr uint32_t oGeo = oXs + 2 * kXBytes;
constexpr uint32_t kGeoBytes = 4 * kGeomFloats;
constexpr uint32_t kGeoStage = kGeoBytes + 2 * 16 * 16;  // + 16 chunk positions (4 per slot) x 2 float4
constexpr uint32_t kStageTx = kXBytes + kGeoStage;      // bytes per stage fill
// Hand-off slot of one tile: dL/dfeatures as float4 [8 = g*4 + j][kPRows], u
// as float [3][kPRows], then the 4 slots' count words (int32) and the region.
// Row r sits at padded position r + r / 8, so that the compute warps' row-wise
// writes and the scatter threads' reads (rows 8 apart) both spread over the banks.
constexpr uint32_t kPRows = kRows + kRows / 8;
__device__ __forceinline__ uint32_t prow(uint32_t r) { return r + (r >> 3); }
constexpr uint32_t oHand = oGeo + 2 * kGeoStage;
constexpr uint32_t kHdDf = 0, kHdU = 16 * 8 * kPRows, kHdNv = kHdU + 3 * 4 * kPRows, kHdRegion = kHdNv + 16;
constexpr uint32_t kHandBytes = kHdRegion + 16;
constexpr uint32_t oMisc = oHand + 2 * kHandBytes;  // 8 mbarriers, TMEM base, abort flag
constexpr uint32_t oBase = oMisc + 128;             // int32 base[K+1]
constexpr size_t kSmemFixed = oBase + 1024;
static_assert(oXs % 1024 == 0 && kXBytes % 1024 == 0, "X tiles must keep the swizzle phase");
static_assert(kGeoBytes % 16 == 0 && kGeoStage % 16 == 0 && oGeo % 16 == 0, "bulk copies need 16 B");
static_assert(oHand % 16 == 0 && kHandBytes % 16 == 0 && oMisc % 8 == 0, "alignment");

struct BwdTcParams {
  const void* mlp;  // 16-bit [K][kMlpParams]
  LevelParams lp;
  int K;
  const int32_t* base;
  const int32_t* n_tiles;
  const char* rec_feat;   // kRecFeatBytes per tile
  const char* rec_geom;   // kGeomFloats floats per tile
  const char* rec_dpart;  // 16 chunk positions x 2 float4 per tile
  float* grad_tables;     // FP32 [K][E][2]
  float* grad_mlp;        // FP32 [K][kMlpParams]
  int32_t* err;
};

template <bool BF16>
__device__ __forceinline__ void load_weights_bwd(const void* blk, char* sm, int tid, int nthreads) {
  uint16_t* b1 = reinterpret_cast<uint16_t*>(sm + oB1);
  uint16_t* b2 = reinterpret_cast<uint16_t*>(sm + oB2);
  uint16_t* b5 = reinterpret_cast<uint16_t*>(sm + oB5);
  uint16_t* b6 = reinterpret_cast<uint16_t*>(sm + oB6);
  for (int i = tid; i < kIn * kWidth; i += nthreads) {
    const int f = i / kWidth, n = i % kWidth;  // W1[f][n]
    const uint16_t v = Half2Of<BF16>::bits(blk, i);
    b1[tc::sw128_offset(n, f) >> 1] = v;  // forward: row n, k = f
    b5[tc::sw128_offset(f, n) >> 1] = v;  // backward: row f, k = n
  }
  for (int i = tid; i < kWidth * kWidth; i += nthreads) {
    const int a = i / kWidth, b = i % kWidth;  // W2[a][b]: h1 index a, z2 index b
    b2[tc::sw128_offset(b, a) >> 1] = Half2Of<BF16>::bits(blk, kIn * kWidth + i);
  }
  for (int i = tid; i < kWidth * 16; i += nthreads) {
    const int n = i / 16, k = i % 16;  // W3[n][k % 4] for k < 8
    b6[tc::sw128_offset(n, k) >> 1] = k < 8 ? Half2Of<BF16>::bits(blk, kIn * kWidth + kWidth * kWidth + n * kOut + (k & 3)) : 0;
  }
}

// 16-bit value > 0 (sign clear, not zero).
__device__ __forceinline__ uint32_t positive16(uint32_t bits16) { return (uint32_t)((bits16 - 1u) & 0xFFFFu) < 0x7FFFu; }

// relu of 16 accumulator values -> chunks 2g, 2g+1 of row `row` of a tile;
// returns the mask of stored values that are > 0.
template <bool BF16>
__device__ __forceinline__ uint32_t store16_relu(uint32_t tile, uint32_t row, int g, const float* v) {
  uint32_t w[8], mask = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    w[i] = Half2Of<BF16>::pack(fmaxf(v[2 * i], 0.0f), fmaxf(v[2 * i + 1], 0.0f));
    mask |= positive16(w[i] & 0xFFFFu) << (2 * i);
    mask |= positive16(w[i] >> 16) << (2 * i + 1);
  }
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g), w[0], w[1], w[2], w[3]);
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g + 1), w[4], w[5], w[6], w[7]);
  return mask;
}

// 16 values -> chunks 2g, 2g+1 of row `row` as a hi/lo pair of tiles:
// hi = 16-bit rounding of v, lo = 16-bit rounding of v - hi.
template <bool BF16>
__device__ __forceinline__ void store16_hilo(uint32_t tile, uint32_t tile_lo, uint32_t row, int g, const float* v) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hi[i] = Half2Of<BF16>::pack(v[2 * i], v[2 * i + 1]);
    const float2 h = Half2Of<BF16>::unpack(hi[i]);
    lo[i] = Half2Of<BF16>::pack(v[2 * i] - h.x, v[2 * i + 1] - h.y);
  }
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g), hi[0], hi[1], hi[2], hi[3]);
  tc::st_shared_v4(tile + tc::sw128_chunk(row, 2 * g + 1), hi[4], hi[5], hi[6], hi[7]);
  tc::st_shared_v4(tile_lo + tc::sw128_chunk(row, 2 * g), lo[0], lo[1], lo[2], lo[3]);
  tc::st_shared_v4(tile_lo + tc::sw128_chunk(row, 2 * g + 1), lo[4], lo[5], lo[6], lo[7]);
}

// Bounded wait of the compute warps for the MMAs committed so far; false on
// timeout (all compute threads agree).
__device__ __forceinline__ bool mma_wait(uint64_t* mbar, uint32_t& phase, bool ok_before = true) {
  const bool ok = tc::mbar_wait_bounded(mbar, phase, kSpin);
  phase ^= 1;
  return !tc::bar_or(kBarCompute, kGroup, !ok || !ok_before);
}
__device__ __forceinline__ void compute_sync() { tc::bar_sync(kBarCompute, kGroup); }

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) k_field_bwd_tc(BwdTcParams p) {
  extern __shared__ __align__(1024) char s_raw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = tc::smem_u32(sm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + oMisc);  // MMA completion
  uint64_t* full = mbar + 1;                                  // record stages 0, 1
  uint64_t* hfull = mbar + 3;                                 // hand-off slots 0, 1 written
  uint64_t* hempty = mbar + 5;                                // hand-off slots 0, 1 read
  uint64_t* drain = mbar + 7;                                 // error path: all MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + oMisc + 64);
  volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(sm + oMisc + 68);
  int32_t* s_base = reinterpret_cast<int32_t*>(sm + oBase);
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;

  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  for (int i = tid; i < (int)(kTileBytes / 16); i += blockDim.x) tc::st_shared_v4(sb + oGO + 16 * i, 0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(tmem_slot, kCols);
  if (tid == 0) {
    for (int i = 0; i < 8; ++i) tc::mbar_init(mbar + i, 1);
    *s_abort = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int n_sub = *p.n_tiles * (kChunksPerTile / kTileChunks);
  const int G = (int)gridDim.x;

  if (warp >= kGroup / kWarp) {
    // ===================== scatter warps =====================
    // Warp sw takes levels 2 sw and 2 sw + 1 of the tile, one after the
    // other; lane pair w (lanes 2w, 2w + 1) takes 8 consecutive rows of a
    // slot (window w: slot qq = w / 4, rows 8 (w % 4) ..), one lane per
    // x-half h of the cell corners. Consecutive samples along a ray often
    // fall in the same cell (most at the coarse levels), so a lane sums their
    // contributions in registers and sends one set of reductions per run of
    // equal cells, its partner's reductions of the same x-pairs in the same
    // instructions. The loops stay (nearly) rolled and read the rows from the
    // hand-off slot: the compute warps' code runs beside this on the same SM,
    // and a fully unrolled scatter's size showed as instruction-fetch stalls.
    const int sw = warp - kGroup / kWarp;
    const int h = lane & 1, qq = lane >> 3, wd = (lane >> 1) & 3;
    int it = 0;
    for (int t = blockIdx.x; t < n_sub; t += G, ++it) {
      const int b = it & 1;
      const bool ok = tc::mbar_wait_bounded(hfull + b, (uint32_t)(it >> 1) & 1u, kSpin);
      if (tc::bar_or(kBarScatter, kGroup, !ok || *s_abort != 0)) {
        if (!ok && tid == kGroup) atomicOr(p.err, kErrTimeout);
        break;
      }
      const char* hd = sm + oHand + (uint32_t)b * kHandBytes;
      const int32_t nw = reinterpret_cast<const int32_t*>(hd + kHdNv)[qq];
      const int k = *reinterpret_cast<const int32_t*>(hd + kHdRegion);
      const float* hu = reinterpret_cast<const float*>(hd + kHdU);
      const float2* df = reinterpret_cast<const float2*>(hd + kHdDf);
      uint32_t vmask = 0;  // rows of the window that hold a sample
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const SlotCount sc = slot_count(nw, 8 * wd + i);
        vmask |= (sc.sl < sc.n ? 1u : 0u) << i;
      }
      const uint32_t r0 = (uint32_t)(qq * kWarp + 8 * wd);  // prow(r0 + i) = prow(r0) + i for i < 8
      float2* gtab = reinterpret_cast<float2*>(p.grad_tables) + (size_t)k * p.lp.E;
#pragma unroll 1
      for (int j = 0; j < 2 && vmask != 0u; ++j) {
        const int l = 2 * sw + j;
        if (l >= p.lp.L) break;
        const float2* dl = df + 2 * (size_t)sw * kPRows + j;  // features 2l, 2l + 1 of row r: dl[2 prow(r)]
        scatter_runs_half<8, true>(
            p.lp, gtab, l, h, vmask,
            [&](int i, float* ui) {
              const uint32_t r = prow(r0) + (uint32_t)i;
#pragma unroll
              for (int ax = 0; ax < 3; ++ax) ui[ax] = hu[ax * kPRows + r];
            },
            [&](int i) { return dl[2 * (prow(r0) + (uint32_t)i)]; });
      }
      tc::bar_sync(kBarScatter, kGroup);  // slot read by every scatter thread
      if (tid == kGroup) tc::mbar_arrive(hempty + b);
    }
  } else {
    // ===================== compute warps =====================
    const int q = warp & 3, g = warp >> 2;
    const uint32_t row = (uint32_t)(q * kWarp + lane);
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    constexpr uint32_t id32 = tc::idesc_f16(BF16, kRows, 32);
    constexpr uint32_t id64 = tc::idesc_f16(BF16, kRows, 64);
    constexpr uint32_t id64_bt = tc::idesc_f16(BF16, kRows, 64) | tc::kMnMajorB;
    constexpr uint32_t id16_abt = tc::idesc_f16(BF16, kRows, 16) | tc::kMnMajorA | tc::kMnMajorB;
    constexpr uint32_t id64_abt = tc::idesc_f16(BF16, kRows, 64) | tc::kMnMajorA | tc::kMnMajorB;
    constexpr uint32_t id32_abt = tc::idesc_f16(BF16, kRows, 32) | tc::kMnMajorA | tc::kMnMajorB;

    // Thread kCopier issues the record copies (thread 0 issues the MMAs);
    // pend[s] = iteration whose records are in flight into stage s (-1: none).
    constexpr int kCopier = kWarp;
    int pend[2] = {-1, -1};
    auto issue = [&](int it, int t) {
      const int s = it & 1;
      tc::fence_proxy_async();  // order earlier generic reads of the stage before the overwrite
      tc::mbar_expect_tx(full + s, kStageTx);
      const uint32_t geo = sb + oGeo + (uint32_t)s * kGeoStage;
      // records are read once: evict-first, so they do not push the region's
      // gradient lines (the scatter's atomics) out of L2
      const uint64_t pol = tc::policy_evict_first();
      tc::bulk_g2s_hint(sb + oXs + (uint32_t)s * kXBytes, p.rec_feat + (size_t)t * kXBytes, kXBytes, full + s, pol);
      tc::bulk_g2s_hint(geo, p.rec_geom + (size_t)t * kGeoBytes, kGeoBytes, full + s, pol);
      tc::bulk_g2s_hint(geo + kGeoBytes, p.rec_dpart + (size_t)t * 512, 512, full + s, pol);
      pend[s] = it;
    };
    if (tid == kCopier && (int)blockIdx.x < n_sub) issue(0, blockIdx.x);

    int region = -1;
    uint32_t phase = 0;
    bool failed = false, dw_started = false;

    auto flush = [&]() {
      // DW / DW3 accumulators -> global (needs all MMAs complete).
      if (!dw_started) return;
      tc::fence_after_sync();
      float* gm = p.grad_mlp + (size_t)region * kMlpParams;
      float v[16];
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        tc::tmem_ld16(tq + kDwCol + 48 * g + 16 * h, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = 48 * g + 16 * h + i, r = (int)row;
          if (r < 64 && c < 64) {
            atomicAdd(gm + kIn * kWidth + c * kWidth + r, v[i]);  // dW2[h1 = c][z2 = r]
          } else if (r >= 64 && c >= 64 && c < 96) {
            atomicAdd(gm + (c - 64) * kWidth + (r - 64), v[i]);  // dW1[feat = c - 64][z1 = r - 64]
          }
        }
      }
      if (g == 0 && q < 2) {  // rows 0..63: dW3[h2 = row][m] = hi column m + lo column 4 + m
        tc::tmem_ld8(tq + kDw3Col, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int m = 0; m < kOut; ++m)
          atomicAdd(gm + kIn * kWidth + kWidth * kWidth + row * kOut + m, v[m] + v[kOut + m]);
      }
      dw_started = false;
    };

    int it = 0;
    for (int t = blockIdx.x; t < n_sub; t += G, ++it) {
      const int s = it & 1;
      const int k = region_of_chunk(s_base, p.K, t * kTileChunks);
      if (k != region) {
        if (dw_started) {  // the last tile's weight-gradient MMAs are not waited on per tile
          if (tid == 0) tc::mma_commit(mbar);
          if (!mma_wait(mbar, phase)) {
            failed = true;
            break;
          }
          flush();
        }
        tc::fence_before_sync();
        compute_sync();
        load_weights_bwd<BF16>(static_cast<const uint16_t*>(p.mlp) + (size_t)k * kMlpParams, sm, tid, kGroup);
        // the weight tiles are complete and visible to the tensor core before
        // this tile's first MMA
        tc::fence_proxy_async();
        tc::fence_before_sync();
        compute_sync();
        region = k;
      }
      const bool staged = tc::mbar_wait_bounded(full + s, (uint32_t)(it >> 1) & 1u, kSpin);
      // ---- this tile's records
      const uint32_t xs = sb + oXs + (uint32_t)s * kXBytes;
      const char* gst = sm + oGeo + (uint32_t)s * kGeoStage;
      const float* geo = reinterpret_cast<const float*>(gst);
      const int32_t nword = reinterpret_cast<const int32_t*>(geo)[kGeomRowFields * kRows + q];
      const SlotCount sc = slot_count(nword, lane);
      const bool valid = sc.sl < sc.n;
      // ---- forward recompute: D1 = X W1
      if (tid == 0 && staged) {
        tc::fence_after_sync();
        for (int kk = 0; kk < 2; ++kk)
          tc::mma_f16(tmem, tc::desc_sw64(xs + 32 * kk, 16), tc::desc_sw128(sb + oB1 + 32 * kk), id64, kk);
        tc::mma_commit(mbar);  // also tracks the previous tile's weight-gradient MMAs
      }
      // ---- meanwhile: chunk-local render adjoint from the records -> g_o tile
      //      row (warps of level half 0); every row is rewritten, zeros for
      //      samples outside the chunks
      if (g == 0 && staged) {
        float go[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (nword != 0) {  // (warp-uniform; an unused part of the slot has n = 0 and zero adjoints)
          const char* ap = gst + kGeoBytes + 32 * (4 * q + sc.part);
          const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          const float4 a0 = sc.n ? *reinterpret_cast<const float4*>(ap) : z;
          const float4 a1 = sc.n ? *reinterpret_cast<const float4*>(ap + 16) : z;
          const float tr = geo[3 * kRows + row], dl = geo[4 * kRows + row];
          const float Tn = geo[5 * kRows + row], w = geo[6 * kRows + row], pair = geo[7 * kRows + row];
          const float sigma = geo[8 * kRows + row];
          const float rgb[3] = {geo[9 * kRows + row], geo[10 * kRows + row], geo[11 * kRows + row]};
          float g_tau;
          render_chunk_adjoint_kept(a0.y * rgb[0] + a0.z * rgb[1] + a0.w * rgb[2], tr, dl, Tn, w, pair, sc.sl, a0.x,
                                    a1.x, a1.y, a1.z, g_tau, sc.width);
          if (valid) {
            const float gC[3] = {a0.y, a0.z, a0.w};
            go[0] = g_tau * dl * sigma;
#pragma unroll
            for (int j = 0; j < 3; ++j) go[1 + j] = w * gC[j] * rgb[j] * (1.0f - rgb[j]);
          }
        }
        const uint32_t h01 = Half2Of<BF16>::pack(go[0], go[1]), h23 = Half2Of<BF16>::pack(go[2], go[3]);
        const float2 f01 = Half2Of<BF16>::unpack(h01), f23 = Half2Of<BF16>::unpack(h23);
        tc::st_shared_v4(sb + oGO + tc::sw128_chunk(row, 0), h01, h23,
                         Half2Of<BF16>::pack(go[0] - f01.x, go[1] - f01.y),
                         Half2Of<BF16>::pack(go[2] - f23.x, go[3] - f23.y));
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (!mma_wait(mbar, phase, staged)) {
        failed = true;
        break;
      }
      if (tid == kCopier) {
        pend[s] = -1;
        // stage s ^ 1 held the previous tile, whose MMAs have all completed
        if (t + G < n_sub) issue(it + 1, t + G);
      }
      // G2 before the mask: [g_o hi | g_o lo] [W3 | W3]^T (one K = 16 MMA),
      // completed by the next commit
      if (tid == 0) {
        tc::fence_after_sync();
        tc::mma_f16(tmem + kG2Col, tc::desc_sw128(sb + oGO), tc::desc_sw128(sb + oB6), id64, 0u);
      }
      tc::fence_after_sync();
      float v[16];
      uint32_t mask1 = 0, mask2 = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tc::tmem_ld16(tq + 32 * g + 16 * h, v);
        tc::tmem_ld_wait();
        mask1 |= store16_relu<BF16>(sb + oH1, row, 2 * g + h, v) << (16 * h);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      compute_sync();
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
      // ---- H2 = relu(D2) and G2 = (H2 > 0) * (G2 before the mask), columns 32g..32g+31
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tc::tmem_ld16(tq + 64 + 32 * g + 16 * h, v);
        tc::tmem_ld_wait();
        const uint32_t m2 = store16_relu<BF16>(sb + oH2, row, 2 * g + h, v);
        mask2 |= m2 << (16 * h);
        tc::tmem_ld16(tq + kG2Col + 32 * g + 16 * h, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (!((m2 >> i) & 1u)) v[i] = 0.0f;
        store16_hilo<BF16>(sb + oG2, sb + oG2l, row, 2 * g + h, v);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      compute_sync();
      const bool acc_on = dw_started;
      // ---- D4 = G2 W2^T (dL/dh1; W2 read MN-major from the layer-2 tile)
      if (tid == 0) {
        tc::fence_after_sync();
        for (int kk = 0; kk < 4; ++kk)
          tc::mma_f16(tmem + 64, tc::desc_sw128(sb + oG2 + 32 * kk), tc::desc_sw128_mn(sb + oB2 + 2048 * kk, 1024),
                      id64_bt, kk);
        for (int kk = 0; kk < 4; ++kk)
          tc::mma_f16(tmem + 64, tc::desc_sw128(sb + oG2l + 32 * kk), tc::desc_sw128_mn(sb + oB2 + 2048 * kk, 1024),
                      id64_bt, 1);
        tc::mma_commit(mbar);
        // DW3 += [H2 | H1]^T [g_o hi | g_o lo] (16 samples per K step = two
        // 8-row groups of both MN-major operands); only read at the region
        // flush, so not waited on here: H2 and the g_o tile are next written
        // after the following commit has completed
        for (int kk = 0; kk < 8; ++kk)
          tc::mma_f16(tmem + kDw3Col, tc::desc_sw128_mn(sb + oH2 + 2048 * kk, kTileBytes),
                      tc::desc_sw128_mn(sb + oGO + 2048 * kk, 1024), id16_abt, (acc_on || kk > 0) ? 1u : 0u);
      }
      if (!mma_wait(mbar, phase)) {
        failed = true;
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tc::tmem_ld16(tq + 64 + 32 * g + 16 * h, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (!((mask1 >> (16 * h + i)) & 1u)) v[i] = 0.0f;  // G1 = (H1 > 0) * D4
        store16_hilo<BF16>(sb + oG1, sb + oG1l, row, 2 * g + h, v);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      compute_sync();
      // ---- D5 = G1 W1^T (dL/dfeatures); DW += [G2 | G1]^T [H1 | X]
      if (tid == 0) {
        tc::fence_after_sync();
        for (int kk = 0; kk < 4; ++kk)
          tc::mma_f16(tmem, tc::desc_sw128(sb + oG1 + 32 * kk), tc::desc_sw128(sb + oB5 + 32 * kk), id32, kk);
        for (int kk = 0; kk < 4; ++kk)
          tc::mma_f16(tmem, tc::desc_sw128(sb + oG1l + 32 * kk), tc::desc_sw128(sb + oB5 + 32 * kk), id32, 1);
        tc::mma_commit(mbar);
        // DW likewise runs behind the next tile: its operands (G2, G1, H1 and
        // this stage's X) are next overwritten only after the next tile's
        // first commit, which tracks these MMAs, has completed.
        for (int kk = 0; kk < 8; ++kk) {
          const uint64_t a = tc::desc_sw128_mn(sb + oG2 + 2048 * kk, kTileBytes);
          const uint32_t acc = (acc_on || kk > 0) ? 1u : 0u;
          tc::mma_f16(tmem + kDwCol, a, tc::desc_sw128_mn(sb + oH1 + 2048 * kk, 1024), id64_abt, acc);
          tc::mma_f16(tmem + kDwCol + 64, a, tc::desc_sw64(xs + 1024 * kk, 512), id32_abt, acc);
        }
      }
      dw_started = true;
      if (!mma_wait(mbar, phase)) {
        failed = true;
        break;
      }
      tc::fence_after_sync();
      tc::tmem_ld16(tq + 16 * g, v);  // dL/dfeatures of levels 8g..8g+7
      tc::tmem_ld_wait();
      // ---- hand the tile's dL/dfeatures to the scatter warps
      const int b = it & 1;
      if (it >= 2) {
        const bool ok = tc::mbar_wait_bounded(hempty + b, (uint32_t)((it >> 1) + 1) & 1u, kSpin);
        if (tc::bar_or(kBarCompute, kGroup, !ok)) {
          failed = true;
          break;
        }
      }
      char* hd = sm + oHand + (uint32_t)b * kHandBytes;
      float4* df = reinterpret_cast<float4*>(hd + kHdDf);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        df[(g * 4 + j) * kPRows + prow(row)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      if (g == 0) {
        float* hu = reinterpret_cast<float*>(hd + kHdU);
#pragma unroll
        for (int a = 0; a < 3; ++a) hu[a * kPRows + prow(row)] = geo[a * kRows + row];
        if (lane == 0) reinterpret_cast<int32_t*>(hd + kHdNv)[q] = nword;
        if (tid == 0) *reinterpret_cast<int32_t*>(hd + kHdRegion) = k;
      }
      tc::fence_before_sync();
      compute_sync();  // slot written; tiles, stage and TMEM free for the next tile
      if (tid == 0) tc::mbar_arrive(hfull + b);
    }
    if (!failed && dw_started) {
      if (tid == 0) tc::mma_commit(mbar);  // drain the last weight-gradient MMAs
      if (mma_wait(mbar, phase)) flush();
      else failed = true;
    }
    if (failed && tid == 0) {
      atomicOr(p.err, kErrTimeout);
      *s_abort = 1;  // wake the scatter warps; they see the flag and stop
      tc::mbar_arrive(hfull);
      tc::mbar_arrive(hfull + 1);
      // let MMAs still in flight land before the CTA exits
      tc::mma_commit(drain);
      tc::mbar_wait_bounded(drain, 0u, kSpin);
    }
    if (failed && tid == kCopier) {  // and the record copies
      for (int s = 0; s < 2; ++s)
        if (pend[s] >= 0) tc::mbar_wait_bounded(full + s, (uint32_t)(pend[s] >> 1) & 1u, kSpin);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace

nerfxl_status launch_field_bwd_tc(const nerfxl_field* f, const LevelParams& lp, char* ws, const Layout& L,
                                  float* grad_tables, float* grad_mlp, cudaStream_t stream) {
  if (L.rec_tiles == 0) return set_error(NERFXL_E_WORKSPACE, "workspace has no tensor-core backward records");
  BwdTcParams p;
  p.mlp = f->mlp;
  p.lp = lp;
  p.K = f->K;
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.rec_feat = ws + L.rec_feat;
  p.rec_geom = ws + L.rec_geom;
  p.rec_dpart = ws + L.rec_dpart;
  p.grad_tables = grad_tables;
  p.grad_mlp = grad_mlp;
  p.err = reinterpret_cast<int32_t*>(ws + L.hdr);
  const size_t smem = kSmemFixed + sizeof(int32_t) * (f->K + 1);
  if (smem > 232448) return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the backward's shared memory");
  void (*kern)(BwdTcParams) = f->mlp_dtype == NERFXL_BF16 ? k_field_bwd_tc<true> : k_field_bwd_tc<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return launch_check("k_field_bwd_tc smem attribute");
  const int grid = fwd_grid(L.chunk_cap / kTileChunks, 1);
  profile_mark(0, stream);
  kern<<<grid, kThreads, smem, stream>>>(p);
  profile_mark(1, stream);
  return kernel_launched("k_field_bwd_tc");
}

}  // namespace nerfxl
