// Occupancy-grid refresh: the spatial-skipping structure of the paper's
// experimental system (Sec. 5.1; the grid of the cited Instant-NGP paper),
// one G^3 grid per region over the region box. Each refresh draws one point
// per cell, evaluates the region's density there and keeps a decaying maximum;
// a cell is occupied while that estimate exceeds the threshold. Rendering
// skips samples in cells whose bit is clear (k_skip_empty).
//
// Kernel: a CTA takes 2048 consecutive cells of one region, stages the
// region's FP32 MLP in shared memory, and evaluates one cell per thread (the
// same encode_f32 / mlp_f32_smem path as the FP32 field kernel); each warp's
// 32 consecutive cells form one word of the bitfield, written from a ballot.

#include <cuda_runtime.h>

#include "nerfxl_split.cuh"
#include "nerfxl_host.h"

namespace nerfxl {
namespace {

constexpr int kOccThreads = 256;
constexpr int kOccCellsPerBlock = 2048;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): each round multiplies words 0 and 2 by the round
// multipliers, XORs the high halves into words 1 and 3 with the key, and the
// key advances by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += kW0;
      k.y += kW1;
    }
    const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
    const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// xi = (w >> 8) * 2^-24 in [0, 1): a 24-bit integer scaled by a power of two, exact in FP32.
__device__ __forceinline__ float unit_float(uint32_t w) { return __uint2float_rn(w >> 8) * (1.0f / 16777216.0f); }

// kSplit: the split representation, whose density needs only the region's
// density MLP.
template <bool kSplit>
__global__ void __launch_bounds__(kOccThreads) k_occupancy_update(FieldPtrs fp, LevelParams lp, int G, int64_t cells,
                                                                  int blocks_per_region, uint32_t step_lo,
                                                                  uint32_t step_hi, uint2 key, float decay,
                                                                  float threshold, float* __restrict__ density,
                                                                  uint32_t* __restrict__ bits) {
  extern __shared__ __align__(16) float s_w[];  // the region's (density) MLP block
  const int k = blockIdx.x / blocks_per_region;
  const int64_t first = (int64_t)(blockIdx.x % blocks_per_region) * kOccCellsPerBlock;
  if (kSplit) load_density_f32(fp.mlp + (size_t)k * kDensityParams, s_w);
  else load_mlp_f32(fp.mlp + (size_t)k * kMlpParams, s_w);
  __syncthreads();
  const float2* table = reinterpret_cast<const float2*>(fp.tables) + (size_t)k * lp.E;
  const int64_t words = (cells + 31) / 32;
  const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
  const int64_t end = min(first + (int64_t)kOccCellsPerBlock, cells);
  for (int64_t c0 = first; c0 < end; c0 += kOccThreads) {  // uniform over the CTA
    const int64_t cell = c0 + threadIdx.x;
    bool on = false;
    if (cell < cells) {
      const int64_t GG = (int64_t)G * G;
      const int c3[3] = {(int)(cell % G), (int)((cell / G) % G), (int)(cell / GG)};
      const uint4 r = philox4x32_10(make_uint4((uint32_t)cell, (uint32_t)k, step_lo, step_hi), key);
      const float xi[3] = {unit_float(r.x), unit_float(r.y), unit_float(r.z)};
      float u[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) u[ax] = __fdiv_rn(__fadd_rn((float)c3[ax], xi[ax]), (float)G);
      float feat[kIn];
      encode_f32(lp, table, u, feat);
      float raw0;
      if (kSplit) {
        float g[kGeo];
        density_f32_smem(s_w, feat, g);
        raw0 = g[0];
      } else {
        float raw[kOut];
        mlp_f32_smem(s_w, feat, raw);
        raw0 = raw[0];
      }
      const float sigma = expf(raw0);
      const size_t at = (size_t)k * cells + cell;
      const float dn = fmaxf(__fmul_rn(decay, density[at]), sigma);
      density[at] = dn;
      on = dn > threshold;
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, on);
    const int64_t w0 = c0 + warp * kWarp;  // first cell of this warp's word (a multiple of 32)
    if (lane == 0 && w0 < cells) bits[(size_t)k * words + w0 / 32] = m;
  }
}

}  // namespace
}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_occupancy_update(const nerfxl_field* f, int32_t G, int64_t step, uint64_t seed,
                                                 float decay, float threshold, float* density, uint32_t* bits,
                                                 cudaStream_t stream) {
  nerfxl_sampling s = {1, 1, 0.0f, 0};
  nerfxl_field plain = f ? *f : nerfxl_field{};
  plain.occupancy = nullptr;  // the refresh does not read the grid it rebuilds
  nerfxl_status st = validate(f ? &plain : nullptr, &s, 0);
  if (st != NERFXL_OK) return st;
  if (f->table_dtype != NERFXL_F32 || f->mlp_dtype != NERFXL_F32)
    return set_error(NERFXL_E_UNSUPPORTED, "the occupancy refresh evaluates FP32 tables and an FP32 MLP");
  if (G < 1 || G > 1024) return set_error(NERFXL_E_INVALID, "G must be in [1, 1024]");
  const int64_t cells = (int64_t)G * G * G;
  if ((int64_t)f->K * cells >= ((int64_t)1 << 31)) return set_error(NERFXL_E_INVALID, "K * G^3 must be below 2^31");
  if (!(decay >= 0.0f && decay <= 1.0f)) return set_error(NERFXL_E_INVALID, "decay must be in [0, 1]");
  if (!density || !bits) return set_error(NERFXL_E_INVALID, "null density or bits");
  const int64_t bpr = (cells + kOccCellsPerBlock - 1) / kOccCellsPerBlock;
  FieldPtrs fp;
  fp.boxes = f->boxes;
  fp.tables = static_cast<const float*>(f->tables);
  fp.mlp = static_cast<const float*>(f->mlp);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const bool split = f->arch == NERFXL_ARCH_SPLIT;
  (split ? k_occupancy_update<true> : k_occupancy_update<false>)<<<(unsigned)(bpr * f->K), kOccThreads,
                                                                    sizeof(float) * kMlpParams, stream>>>(
      fp, level_params(f), G, cells, (int)bpr, (uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), key, decay,
      threshold, density, bits);
  return kernel_launched("k_occupancy_update");
}
