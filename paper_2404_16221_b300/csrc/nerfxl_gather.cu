// Level-grouped gather of the tensor-core forward, for fields whose hash
// tables outgrow what L2 keeps for these random gathers.
//
// The tensor-core forward sweeps the regions one at a time, so a region's
// whole table (every level) is the working set of the gather. Random 4- or
// 8-byte gathers keep their L2 hit rate only while that set stays small
// (measured on the street/city shapes: 95 % at 27 MB, 44 % at 50 MB, 27 % at
// the 96 MB of a region with 2^21-entry levels, where the forward then reads
// 214x the tables' bytes from HBM). This pass instead sweeps (region, group
// of levels) pairs: for every tile of the region, the features of one group
// of levels, then the next group. It writes each row's 16-bit features as
// level-major words (whole sectors: 512 contiguous bytes per level and tile),
// and the tensor-core forward then reads the features from there instead of
// gathering. The features equal the fused gather's bit for bit (same
// per-level arithmetic, same rounding to the MLP's 16-bit type). A first pass
// over the window's rows (k_gather_coords) stores each row's region
// coordinates once, so the group passes do not repeat the ray, segment and
// sample arithmetic. Each group is still one more pass over the region's
// samples (coordinates, launch, feature words), so the groups are as large as
// still pays: two groups of a 96 MB table beat three to eleven smaller ones.
//
// Work items are (region, group, tile) in that order over a window of tiles;
// the persistent CTAs take consecutive items, so the GPU works on one
// (region, group) at a time. Two items per CTA of 256 threads, one row per
// thread.

#include <cuda_runtime.h>

#include "nerfxl_field.cuh"
#include "nerfxl_half.cuh"
#include "nerfxl_host.h"

namespace nerfxl {
namespace {

constexpr int kGThreads = 256;
constexpr int kGRows = 128;  // one 4-chunk tile

struct GatherGroupsParams {
  const float* rays_o;
  const float* rays_d;
  const float* boxes;
  const void* tables;  // [K][E] of float2 or half2
  LevelParams lp;
  SampParams sp;
  int K;
  const RayHdr* hdr;
  const SegDesc* segs;
  const int32_t* base;
  const Slot* chunks;
  const int32_t* n_tiles;
  uint32_t* feat;  // level-major words: level l, tile t, row r at feat[(l * window + t - w0) * 128 + r]
  int64_t window;  // tiles per level in feat
  int64_t w0, w1;  // the window of 4-chunk tiles (w1 - w0 <= window)
  int n_groups;
  int32_t g_lo[kMaxLevels + 1];  // group g holds levels g_lo[g] .. g_lo[g + 1] - 1
};

// The window's rows once: each row's sample position in its region's box, as
// the tensor-core forward computes it (the same arithmetic, so the groups'
// features equal the one-pass gather's), stored after the feature words for
// every group pass to read instead of repeating the ray, segment and sample
// arithmetic per group.
__global__ void __launch_bounds__(kGThreads) k_gather_coords(GatherGroupsParams p) {
  const int64_t n_sub = (int64_t)*p.n_tiles * (kChunksPerTile / 4);
  const int64_t wa = p.w0, wb = p.w1 < n_sub ? p.w1 : n_sub;
  const size_t cstride = (size_t)p.window * kGRows;
  uint32_t* cw0 = p.feat + (size_t)p.lp.L * cstride;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < (wb - wa) * kGRows;
       gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = wa + gi / kGRows;
    const uint32_t row = (uint32_t)(gi % kGRows);
    const int q = (int)(row / kWarp), lane = (int)(row % kWarp);
    const SlotLane sl = slot_lane(p.chunks[t * 4 + q], lane);
    bool valid = false;
    float u[3] = {0.0f, 0.0f, 0.0f};
    if (sl.has) {
      const int k = region_of_chunk(p.base, p.K, (int)(t * 4));
      const uint32_t ray = sl.ref.x;
      const int seg = sl.ref.y >> 16;
      const int c = sl.ref.y & 0xFFFF;
      const RayHdr h = p.hdr[ray];
      const SegDesc sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
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
        float x[3];
        sample_point(o, d, tbar, x);
        region_coord(p.boxes + 6 * k, x, u);
      }
    }
    uint32_t* cw = cw0 + (size_t)(t - wa) * kGRows + row;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) cw[ax * cstride] = __float_as_uint(u[ax]);
    cw[3 * cstride] = valid ? 1u : 0u;
  }
}

template <bool kF16Table, bool kBF16>
__global__ void __launch_bounds__(kGThreads, 4) k_gather_groups(GatherGroupsParams p) {
  using TabT = typename TableOf<kF16Table>::T;
  extern __shared__ int32_t s_i[];
  const int K = p.K;
  int32_t* s_pre = s_i;            // [K + 1] first item of each region
  int32_t* s_start = s_i + K + 1;  // [K] first tile of the region inside the window
  int32_t* s_cnt = s_start + K;    // [K] tiles of the region inside the window
  const int64_t n_sub = (int64_t)*p.n_tiles * (kChunksPerTile / 4);
  const int64_t wa = p.w0, wb = p.w1 < n_sub ? p.w1 : n_sub;
  if (wa >= wb) return;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int64_t tb = p.base[k] / 4, te = p.base[k + 1] / 4;
    const int64_t lo = tb > wa ? tb : wa, hi = te < wb ? te : wb;
    s_start[k] = (int32_t)lo;
    s_cnt[k] = hi > lo ? (int32_t)(hi - lo) : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_pre[0] = 0;
    for (int k = 0; k < K; ++k) s_pre[k + 1] = s_pre[k] + s_cnt[k] * p.n_groups;
  }
  __syncthreads();
  const int total = s_pre[K];
  const int sub = threadIdx.x / kGRows;
  const uint32_t row = threadIdx.x % kGRows;
  for (int it = blockIdx.x * 2 + sub; it < total; it += gridDim.x * 2) {
    int lo = 0, hi = K - 1;  // region k: s_pre[k] <= it < s_pre[k + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const int k = lo;
    const int rem = it - s_pre[k];
    const int g = rem / s_cnt[k];
    const int64_t t = s_start[k] + rem % s_cnt[k];
    // the row's region coordinates, from the window's coordinate words
    const uint32_t* cw = p.feat + ((size_t)p.lp.L * p.window + (size_t)(t - wa)) * kGRows + row;
    const size_t cstride = (size_t)p.window * kGRows;
    const bool valid = __ldcs(cw + 3 * cstride) != 0u;
    float u[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) u[ax] = __uint_as_float(__ldcs(cw + ax * cstride));
    const TabT* table = static_cast<const TabT*>(p.tables) + (size_t)k * p.lp.E;
    // level-major words: the 128 rows of a tile write 512 contiguous bytes per
    // level, whole sectors (a partly written sector would cost L2 a read
    // from HBM to merge)
    uint32_t* dst = p.feat + (size_t)(t - wa) * kGRows + row;
    const int l_end = p.g_lo[g + 1];
    for (int l = p.g_lo[g]; l < l_end; ++l) {
      const float2 v = valid ? gather1<TabT>(p.lp, table, u, l) : make_float2(0.0f, 0.0f);
      __stcs(dst + (size_t)l * p.window * kGRows, Half2Of<kBF16>::pack(v.x, v.y));
    }
  }
}

size_t g_group_min = kGroupMinBytes;
size_t g_group_bytes = kGroupBytes;
int64_t g_window = kGatherWindowTiles;
int64_t g_group_samples = kGroupMinRegionSamples;

}  // namespace

size_t group_min_bytes() { return g_group_min; }
int64_t gather_window_tiles() { return g_window; }

bool grouped_gather(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R) {
  if (f->mlp_dtype != NERFXL_BF16 && f->mlp_dtype != NERFXL_F16) return false;
  const int64_t E = nerfxl_table_entries(f->level_res, f->L, f->log2_T);
  const int64_t bytes = E * f->F * (f->table_dtype == NERFXL_F16 ? 2 : 4);
  return (size_t)bytes > g_group_min && R * (int64_t)s->n_samples >= g_group_samples * (int64_t)f->K;
}

int gather_groups(const nerfxl_field* f, const LevelParams& lp, int32_t* g_lo) {
  const size_t eb = (size_t)f->F * (f->table_dtype == NERFXL_F16 ? 2 : 4);
  int n = 0;
  size_t acc = 0;
  g_lo[0] = 0;
  for (int l = 0; l < lp.L; ++l) {
    const size_t bytes = (size_t)((l + 1 < lp.L ? lp.off[l + 1] : lp.E) - lp.off[l]) * eb;
    if (l > 0 && acc + bytes > g_group_bytes) {
      g_lo[++n] = l;
      acc = 0;
    }
    acc += bytes;
  }
  g_lo[++n] = lp.L;
  return n;
}

nerfxl_status launch_gather_groups(const nerfxl_field* f, const SampParams& sp, const LevelParams& lp,
                                   const float* rays_o, const float* rays_d, char* ws, const Layout& L, uint32_t* feat,
                                   int64_t window, int64_t w0, int64_t w1, cudaStream_t stream) {
  GatherGroupsParams p;
  p.rays_o = rays_o;
  p.rays_d = rays_d;
  p.boxes = f->boxes;
  p.tables = f->tables;
  p.lp = lp;
  p.sp = sp;
  p.K = f->K;
  p.hdr = reinterpret_cast<const RayHdr*>(ws + L.ray_hdr);
  p.segs = reinterpret_cast<const SegDesc*>(ws + L.segs);
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.chunks = reinterpret_cast<const Slot*>(ws + L.chunks);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.feat = feat;
  p.window = window;
  p.w0 = w0;
  p.w1 = w1;
  p.n_groups = gather_groups(f, lp, p.g_lo);
  const bool f16tab = f->table_dtype == NERFXL_F16, bf = f->mlp_dtype == NERFXL_BF16;
  void (*kern)(GatherGroupsParams) = f16tab ? (bf ? k_gather_groups<true, true> : k_gather_groups<true, false>)
                                            : (bf ? k_gather_groups<false, true> : k_gather_groups<false, false>);
  k_gather_coords<<<fwd_grid(((w1 - w0) * kGRows + kGThreads - 1) / kGThreads, 8), kGThreads, 0, stream>>>(p);
  nerfxl_status st = kernel_launched("k_gather_coords");
  if (st != NERFXL_OK) return st;
  const size_t smem = sizeof(int32_t) * (3 * (size_t)f->K + 1);
  const int64_t items = (w1 - w0) * p.n_groups;  // upper bound: the window's tiles times the groups
  const int grid = fwd_grid((items + 1) / 2, 4);
  kern<<<grid, kGThreads, smem, stream>>>(p);
  return kernel_launched("k_gather_groups");
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_set_gather_groups(size_t min_table_bytes, size_t group_bytes, int64_t window_tiles,
                                                  int64_t min_region_samples) {
  if (window_tiles < 0 || min_region_samples < 0)
    return set_error(NERFXL_E_INVALID, "window_tiles and min_region_samples must be >= 0");
  g_group_min = min_table_bytes ? min_table_bytes : kGroupMinBytes;
  g_group_bytes = group_bytes ? group_bytes : kGroupBytes;
  g_window = window_tiles ? window_tiles : kGatherWindowTiles;
  g_group_samples = min_region_samples ? min_region_samples : kGroupMinRegionSamples;
  return NERFXL_OK;
}
