// Forward pass of the one-GPU NeRF-XL hot path (arXiv 2404.16221) and the
// C-ABI entry points declared in include/nerfxl.h.
//
// Work decomposition. A ray's samples are grouped into CHUNKS of at most 32
// consecutive intervals that all lie in one region segment. Each chunk is
// reduced by one warp to a 7-float partial (optical depth, colour, opacity,
// depth, distortion), exactly the per-segment partial of Sec. 4.3: because
// the composition of Eq. 3-8 is associative, chunks are just finer segments,
// so chunks never need each other's state. Chunks are bucketed by region
// (padded to whole tiles of kChunksPerTile) so that every CTA tile evaluates a
// single region's MLP and can keep its weights in shared memory. A final
// per-ray kernel composites the chunk partials in ray order (Algorithm 1, 2).
//
// Kernels (one forward call):
//   k_segments     per ray: slab tests, sorted segments, interval counts;
//                  per-region chunk histogram (block-aggregated atomics)
//   k_region_scan  1 thread: padded exclusive scan of the histogram -> bases
//   k_fill_chunks  per ray: chunk references into the region buckets
//   k_field_fwd    persistent CTAs over tiles: hash gather + MLP + local render
//   k_composite    per ray: exclusive prefix product over chunk partials

#include <cuda_runtime.h>

#include <atomic>
#include <stdio.h>

#include <algorithm>
#include <string>

#include "nerfxl_device.cuh"
#include "nerfxl_split.cuh"
#include "nerfxl_tile.cuh"
#include "nerfxl_host.h"

namespace nerfxl {

// ---------------------------------------------------------------------------
// k_segments

__global__ void __launch_bounds__(256) k_segments(const float* __restrict__ rays_o, const float* __restrict__ rays_d,
                                                  int64_t R, const float* __restrict__ boxes, int K, SampParams sp,
                                                  RayHdr* __restrict__ hdr, SegDesc* __restrict__ segs,
                                                  int32_t* __restrict__ counts, int32_t* __restrict__ err) {
  extern __shared__ float s_mem[];
  float* s_boxes = s_mem;                                 // [K][6]
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_mem + 6 * K);  // [3][K]: chunks, of them width 16, width 8
  __shared__ unsigned long long s_samples, s_chunks;
  for (int i = threadIdx.x; i < 6 * K; i += blockDim.x) s_boxes[i] = boxes[i];
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) s_cnt[i] = 0;
  if (threadIdx.x == 0) s_samples = s_chunks = 0ull;
  __syncthreads();

  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) {
    float o[3], d[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      o[ax] = rays_o[3 * r + ax];
      d[ax] = rays_d[3 * r + ax];
    }
    float st0[kMaxSeg], st1[kMaxSeg];
    int sreg[kMaxSeg];
    const int hits = ray_segments(o, d, s_boxes, K, sp.t_min, sp.max_seg, st0, st1, sreg);
    if (hits > sp.max_seg) atomicOr(err, kErrOverflow);
    const int nseg = min(hits, sp.max_seg);
    RayHdr h;
    h.nseg = nseg;
    h.tn = nseg ? st0[0] : 0.0f;
    h.delta = nseg ? __fdiv_rn(__fsub_rn(st1[nseg - 1], st0[0]), (float)sp.S) : 0.0f;
    int cbase = 0, n_samples = 0;
    for (int k = 0; k < nseg; ++k) {
      const int jlo = first_edge_above(h.tn, h.delta, sp.S, st0[k]);
      const int jend = first_edge_at_or_above(h.tn, h.delta, sp.S, st1[k]);
      const int n = 1 + max(0, jend - jlo);
      SegDesc s;
      s.t0 = st0[k];
      s.t1 = st1[k];
      s.jlo_n = (jlo & 0xFFFF) | (n << 16);
      s.reg_cb = (sreg[k] & 0xFFFF) | (cbase << 16);
      segs[r * sp.max_seg + k] = s;
      const int nch = seg_chunks(n);
      if (counts) {
        atomicAdd(&s_cnt[sreg[k]], nch);
        const int tw = seg_tail_width(n);
        if (tw < kWarp) atomicAdd(&s_cnt[(tw == 16 ? K : 2 * K) + sreg[k]], 1);
      }
      cbase += nch;
      n_samples += n;
    }
    h.nchunk = cbase;
    hdr[r] = h;
    atomicAdd(&s_samples, (unsigned long long)n_samples);
    atomicAdd(&s_chunks, (unsigned long long)cbase);
  }
  __syncthreads();
  if (!counts) return;  // the occupancy pass buckets the kept samples
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&counts[i], s_cnt[i]);
  if (threadIdx.x == 0) {
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(err + 2);
    atomicAdd(stats + 0, s_samples);
    atomicAdd(stats + 1, s_chunks);
  }
}

// ---------------------------------------------------------------------------
// k_skip_empty: occupancy-grid skipping, one warp per ray. The ray's
// intervals are numbered in ray order (segment by segment) and tested 32 at a
// time, lane j of a group taking flat interval 32 gi + j. Lane k holds
// segment k and its first flat index; a lane finds its segment from the
// group's segment-start mask (an OR-reduction over the lanes), computes the
// interval's sample point with the same FP32 operations as the field kernels
// (the reciprocal box extents come from a per-CTA table, computed once with
// the same IEEE division), and loads the word holding the bit of its region
// cell min(floor(u G), G - 1). The loads of up to kSkipBatch groups are in
// flight together; then a ballot per group compacts the kept interval
// indices, in order, into the ray's list. Lane k counts its segment's kept
// samples; warp scans give each segment its list start and chunk base, and
// the ray's chunk count, the per-region chunk histogram and the sample /
// chunk counters become those of the kept samples (an emptied segment has no
// chunk).

constexpr int kSkipBatch = 4;

__global__ void __launch_bounds__(256) k_skip_empty(const float* __restrict__ rays_o, const float* __restrict__ rays_d,
                                                    int64_t R, const float* __restrict__ boxes, int K, SampParams sp,
                                                    const uint32_t* __restrict__ occ, int G, RayHdr* __restrict__ hdr,
                                                    SegDesc* __restrict__ segs, int32_t* __restrict__ seg_keep,
                                                    uint16_t* __restrict__ kept, int32_t* __restrict__ counts,
                                                    int32_t* __restrict__ err) {
  extern __shared__ float s_mem[];
  float* s_boxes = s_mem;                                      // [K][6]
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_mem + 6 * K);  // [3][K]: chunks, of them width 16, width 8
  float* s_inv = s_mem + 9 * K;                                // [K][3] 1 / box extent
  __shared__ unsigned long long s_samples, s_chunks;
  for (int i = threadIdx.x; i < 6 * K; i += blockDim.x) s_boxes[i] = boxes[i];
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) {
    const int k = i / 3, ax = i % 3;
    s_inv[i] = __fdiv_rn(1.0f, __fsub_rn(boxes[6 * k + 3 + ax], boxes[6 * k + ax]));
  }
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) s_cnt[i] = 0;
  if (threadIdx.x == 0) s_samples = s_chunks = 0ull;
  __syncthreads();

  const unsigned kFull = 0xFFFFFFFFu;
  const int lane = threadIdx.x % kWarp;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  if (r < R) {  // warp-uniform
    const RayHdr h = hdr[r];
    const int nseg = h.nseg;
    float o[3], d[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      o[ax] = rays_o[3 * r + ax];
      d[ax] = rays_d[3 * r + ax];
    }
    // lane k < nseg: segment k and its first flat interval index
    SegDesc my = {0.0f, 0.0f, 0, 0};
    if (lane < nseg) my = segs[r * sp.max_seg + lane];
    const int my_n = lane < nseg ? seg_n(my) : 0;
    int incl = my_n;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += v;
    }
    const int my_start = incl - my_n;
    const int my_end = incl;
    const int total = __shfl_sync(kFull, incl, kWarp - 1);
    const size_t words = ((size_t)G * G * G + 31) / 32;
    int kept_before = 0;  // kept samples of the ray so far (flat order)
    int my_count = 0;     // lane k: kept samples of segment k
    for (int base = 0; base < total; base += kSkipBatch * kWarp) {
      uint32_t word[kSkipBatch];
      int bit[kSkipBatch], iv[kSkipBatch];
#pragma unroll
      for (int gi = 0; gi < kSkipBatch; ++gi) {
        word[gi] = 0u;
        bit[gi] = 0;
        iv[gi] = 0;
        const int gbase = base + gi * kWarp;
        if (gbase >= total) continue;  // warp-uniform
        const int j = gbase + lane;
        // segment of j: the last segment starting at or before j (every
        // segment has >= 1 interval, so the starts strictly increase)
        const bool mine = lane < nseg;
        const unsigned heads = __reduce_or_sync(
            kFull, (mine && my_start >= gbase && my_start < gbase + kWarp) ? 1u << (my_start - gbase) : 0u);
        const int before = __popc(__ballot_sync(kFull, mine && my_start < gbase));
        const int k = before + __popc(heads & (lane == 31 ? kFull : ((2u << lane) - 1u))) - 1;
        SegDesc sd;
        sd.t0 = __shfl_sync(kFull, my.t0, k);
        sd.t1 = __shfl_sync(kFull, my.t1, k);
        sd.jlo_n = __shfl_sync(kFull, my.jlo_n, k);
        sd.reg_cb = __shfl_sync(kFull, my.reg_cb, k);
        const int i = j - __shfl_sync(kFull, my_start, k);
        iv[gi] = i;
        if (j < total) {
          float a, b;
          segment_interval(sd, h.tn, h.delta, i, a, b);
          const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
          float x[3], u[3];
          sample_point(o, d, tbar, x);
          const int reg = seg_region(sd);
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {  // region_coord with the CTA's reciprocal extents
            const float v = __fmul_rn(__fsub_rn(x[ax], s_boxes[6 * reg + ax]), s_inv[3 * reg + ax]);
            u[ax] = fminf(fmaxf(v, 0.0f), 1.0f);
          }
          int c[3];
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            float fr;
            level_cell(u[ax], G, c[ax], fr);
          }
          const uint32_t cell = (uint32_t)c[0] + (uint32_t)G * ((uint32_t)c[1] + (uint32_t)G * (uint32_t)c[2]);
          word[gi] = __ldg(occ + (size_t)reg * words + (cell >> 5));
          bit[gi] = (int)(cell & 31u);
        }
      }
#pragma unroll
      for (int gi = 0; gi < kSkipBatch; ++gi) {
        const int gbase = base + gi * kWarp;
        if (gbase >= total) break;  // warp-uniform
        const int j = gbase + lane;
        const bool keep = j < total && ((word[gi] >> bit[gi]) & 1u);
        const unsigned m = __ballot_sync(kFull, keep);
        if (keep) kept[r * sp.max_int + kept_before + __popc(m & ((1u << lane) - 1u))] = (uint16_t)iv[gi];
        kept_before += __popc(m);
        // lane k: the part of this group inside segment k's flat range
        const int lo = min(max(my_start - gbase, 0), kWarp), hi = min(max(my_end - gbase, 0), kWarp);
        const unsigned below_hi = hi >= kWarp ? kFull : ((1u << hi) - 1u);
        const unsigned below_lo = lo >= kWarp ? kFull : ((1u << lo) - 1u);
        my_count += __popc(m & below_hi & ~below_lo);
      }
    }
    // per segment: list start and chunk base (exclusive scans over the lanes)
    const int my_nch = seg_chunks(my_count);
    int inc_c = my_count, inc_h = my_nch;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
      const int vc = __shfl_up_sync(kFull, inc_c, off);
      const int vh = __shfl_up_sync(kFull, inc_h, off);
      if (lane >= off) {
        inc_c += vc;
        inc_h += vh;
      }
    }
    if (lane < nseg) {
      const int reg = seg_region(my);
      const int cbase = inc_h - my_nch;
      seg_keep[r * sp.max_seg + lane] = my_count | ((inc_c - my_count) << 16);
      segs[r * sp.max_seg + lane].reg_cb = (reg & 0xFFFF) | (cbase << 16);
      if (my_nch) atomicAdd(&s_cnt[reg], my_nch);
      if (my_nch && seg_tail_width(my_count) < kWarp)
        atomicAdd(&s_cnt[(seg_tail_width(my_count) == 16 ? K : 2 * K) + reg], 1);
    }
    const int nchunk = __shfl_sync(kFull, inc_h, kWarp - 1);
    if (lane == 0) {
      hdr[r].nchunk = nchunk;
      atomicAdd(&s_samples, (unsigned long long)kept_before);
      atomicAdd(&s_chunks, (unsigned long long)nchunk);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&counts[i], s_cnt[i]);
  if (threadIdx.x == 0) {
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(err + 2);
    atomicAdd(stats + 0, s_samples);
    atomicAdd(stats + 1, s_chunks);
  }
}

// ---------------------------------------------------------------------------
// k_region_scan: region k holds counts[k] chunks, counts[K + k] of them of
// width 16 (at most 16 samples) and counts[2K + k] of width 8 (at most 8); its
// slots are one per wider chunk, then one per pair of width-16 chunks, then
// one per four of width 8: full_k + ceil(h_k / 2) + ceil(q_k / 4).
// base[k] = sum_{k' < k} round_up(slots_k', tile); padding slots get the
// empty marker, the free parts of the last pair / quad the unused marker;
// header word 1 = total tiles.

__device__ __forceinline__ void set_ref(uint2* chunks, int64_t slot, int part, uint32_t x) {
  chunks[4 * slot + part] = make_uint2(x, 0u);
}

__global__ void k_region_scan(const int32_t* __restrict__ counts, int K, int chunks_per_tile,
                              int32_t* __restrict__ base, uint2* __restrict__ chunks, int32_t* __restrict__ n_tiles) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t acc = 0;
  for (int k = 0; k < K; ++k) {
    base[k] = acc;
    const int h = counts[K + k], qn = counts[2 * K + k];
    const int full = counts[k] - h - qn, hs = (h + 1) / 2, qs = (qn + 3) / 4;
    const int slots = full + hs + qs;
    const int padded = (slots + chunks_per_tile - 1) / chunks_per_tile * chunks_per_tile;
    if (h & 1) set_ref(chunks, acc + full + hs - 1, 1, kUnusedPart);
    for (int p = qn & 3; p > 0 && p < 4; ++p) set_ref(chunks, acc + full + hs + qs - 1, p, kUnusedPart);
    for (int i = slots; i < padded; ++i)
      for (int p = 0; p < 4; ++p) set_ref(chunks, acc + i, p, kEmptyChunk);
    acc += padded;
  }
  base[K] = acc;
  *n_tiles = acc / chunks_per_tile;
}

// ---------------------------------------------------------------------------
// k_fill_chunks: chunk references {ray, seg << 16 | chunk-in-segment} into
// the region's slots (chunks = uint2 [slots][4]): a chunk of more than 16
// samples fills a slot alone; a segment's last chunk of at most 16 (8) takes
// the next free half (quarter) of the region's width-16 (width-8) slots.

__global__ void __launch_bounds__(256) k_fill_chunks(int64_t R, int K, SampParams sp, const RayHdr* __restrict__ hdr,
                                                     const SegDesc* __restrict__ segs,
                                                     const int32_t* __restrict__ counts,
                                                     const int32_t* __restrict__ base, int32_t* __restrict__ cursor,
                                                     uint2* __restrict__ chunks) {
  extern __shared__ int32_t s_i[];
  int32_t* s_cnt = s_i;           // [3][K]: this block's whole-slot, width-16 and width-8 chunks
  int32_t* s_base = s_i + 3 * K;  // [3][K]: their first index in the region
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int nseg = 0;
  int off[kMaxSeg], toff[kMaxSeg];
  if (r < R) {
    nseg = hdr[r].nseg;
    for (int k = 0; k < nseg; ++k) {
      const SegDesc s = segs[r * sp.max_seg + k];
      const int n = seg_samples(sp, s, r, k).n;
      const int tw = seg_tail_width(n);
      off[k] = atomicAdd(&s_cnt[seg_region(s)], seg_chunks(n) - (tw < kWarp ? 1 : 0));
      toff[k] = tw < kWarp ? atomicAdd(&s_cnt[(tw == 16 ? K : 2 * K) + seg_region(s)], 1) : 0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) s_base[i] = s_cnt[i] ? atomicAdd(&cursor[i], s_cnt[i]) : 0;
  __syncthreads();
  for (int k = 0; k < nseg; ++k) {
    const SegDesc s = segs[r * sp.max_seg + k];
    const int reg = seg_region(s);
    const int n = seg_samples(sp, s, r, k).n;
    const int nch = seg_chunks(n);
    const int tw = seg_tail_width(n);
    const int nfull = nch - (tw < kWarp ? 1 : 0);
    const int dst = base[reg] + s_base[reg] + off[k];
    for (int c = 0; c < nfull; ++c) {
      chunks[4 * (int64_t)(dst + c)] = make_uint2((uint32_t)r, (uint32_t)((k << 16) | c));
      for (int p = 1; p < 4; ++p) set_ref(chunks, dst + c, p, kEmptyChunk);
    }
    if (tw < kWarp) {
      const int h = counts[K + reg], qn = counts[2 * K + reg];
      const int full = counts[reg] - h - qn;
      const uint2 ref = make_uint2((uint32_t)r, (uint32_t)((k << 16) | (nch - 1)));
      if (tw == 16) {
        const int i = s_base[K + reg] + toff[k];  // index among the region's width-16 chunks
        const int64_t slot = base[reg] + full + (i >> 1);
        chunks[4 * slot + (i & 1)] = ref;
        if ((i & 1) == 0) {  // a width-16 slot's references 2, 3 stay empty
          set_ref(chunks, slot, 2, kEmptyChunk);
          set_ref(chunks, slot, 3, kEmptyChunk);
        }
      } else {
        const int i = s_base[2 * K + reg] + toff[k];  // index among the region's width-8 chunks
        const int64_t slot = base[reg] + full + (h + 1) / 2 + (i >> 2);
        chunks[4 * slot + (i & 3)] = ref;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// k_field_fwd_f32: the fused FP32 field on CUDA cores. Persistent CTAs of 256
// threads take 128-row sub-tiles (4 chunk slots, half of a 256-row tile; both
// halves of a tile belong to one region) interleaved across the grid, two
// CTAs per SM so that one gathers while the other multiplies. Per sub-tile:
//   gather    thread (h, s) encodes levels 8 h .. 8 h + 7 of sample s into
//             rows 16 h .. 16 h + 15 of the unit-major feature buffer (and the
//             FP32 records for the backward, when asked for)
//   MLP       register-tiled products over the 128 samples (a thread owns 8
//             samples x 4 units; weights staged row-major per region), unit-
//             major activations in two buffers of 64 rows
//   render    thread s (warps 0-3, one chunk slot each): raw outputs, sigma,
//             rgb, the chunk's partial (or the sample-level values)
// Each output accumulates over its inputs in order with fused multiply-adds
// from zero, as a per-sample dot product would, and the backward's recompute
// does the same.

constexpr int kFwdRows = 128;                    // samples per sub-tile
constexpr int kFwdThreads = 2 * kFwdRows;        // two threads per sample in the gather
constexpr int kFPitch = kFwdRows + 4;            // unit-major row pitch
constexpr int kFwdSubPerTile = kChunksPerTile / 4;

struct FwdParams {
  const float* rays_o;
  const float* rays_d;
  FieldPtrs fp;
  LevelParams lp;
  SampParams sp;
  int K;
  const RayHdr* hdr;
  const SegDesc* segs;
  const int32_t* base;     // [K+1]
  const Slot* chunks;      // slots
  const int32_t* n_tiles;
  float4* partials;        // [R][max_chunk][2]
  float4* smp4;            // per sample slot: sigma, rgb (sample-level composition), or NULL
  float2* smp2;            // per sample slot: tbar - tn, delta
  float* rec32;            // the backward's FP32 feature records [tiles][32][256], or NULL
};

// Weights in shared memory, row-major as stored: W1 [32][64], W2 [64][64], W3 [64][4].
__global__ void __launch_bounds__(kFwdThreads, 2) k_field_fwd_f32(FwdParams p) {
  extern __shared__ __align__(16) float s_dyn[];
  constexpr int kWFloats = kMlpParams;
  float* s_w = s_dyn;
  float* s_A = s_w + kWFloats;       // [64][kFPitch]
  float* s_B = s_A + kWidth * kFPitch;  // [64][kFPitch]
  int32_t* s_base = reinterpret_cast<int32_t*>(s_B + kWidth * kFPitch);  // [K+1]
  const int tid = threadIdx.x, warp = tid / kWarp, lane = tid % kWarp;
  const int h = tid / kFwdRows;            // gather half: levels 8 h .. 8 h + 7
  const int srow = tid % kFwdRows;         // the thread's sample row
  const int q = warp & 3;                  // its chunk slot within the sub-tile
  const int sb = tid & 15, ub = tid >> 4;  // products: samples 4 sb.., 64 + 4 sb..; units of block ub
  for (int i = tid; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  __syncthreads();
  const int n_sub = *p.n_tiles * kFwdSubPerTile;
  int region = -1;
  const float2* table = nullptr;
  // The two activation buffers alternate roles by sub-tile: features and h2
  // in s_F, h1 in s_H, swapped on the next sub-tile. So the render of a
  // sub-tile (warps 0-3, reading h2) overlaps the next sub-tile's gather
  // (warps 4-7 start it at once; its features go to the other buffer), and no
  // barrier closes a sub-tile: the next layer 1, which overwrites this h2, runs
  // after the barrier that ends the next gather.
  int it = 0;
  for (int t = blockIdx.x; t < n_sub; t += gridDim.x, ++it) {
    const int k = region_of_chunk(s_base, p.K, t * 4);
    float* s_F = (it & 1) ? s_B : s_A;
    float* s_H = (it & 1) ? s_A : s_B;
    if (k != region) {
      __syncthreads();  // the render warps are done with the previous weights
      for (int i = tid; i < kMlpParams; i += blockDim.x) s_w[i] = p.fp.mlp[(size_t)k * kMlpParams + i];
      region = k;
      table = reinterpret_cast<const float2*>(p.fp.tables) + (size_t)k * p.lp.E;
    }
    // ---- per sample (both gather halves): slot, geometry, 8 levels of features
    const SlotLane sl = slot_lane(p.chunks[t * 4 + q], lane);
    const uint2 ref = sl.ref;
    const uint32_t ray = sl.has ? ref.x : 0u;
    const int seg = ref.y >> 16, c = ref.y & 0xFFFF;
    RayHdr hd = {0.0f, 0.0f, 0, 0};
    SegDesc sd = {0.0f, 0.0f, 0, 0};
    float d[3] = {0.0f, 0.0f, 0.0f};
    bool valid = false;
    float tbar = 0.0f, dl = 0.0f;
    float feat[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) feat[j] = 0.0f;
    if (sl.has) {
      hd = p.hdr[ray];
      sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) d[ax] = p.rays_d[3 * (size_t)ray + ax];
      const SegSamples ss = seg_samples(p.sp, sd, ray, seg);
      const int i = c * kWarp + sl.sl;
      valid = i < ss.n;
      if (valid) {
        float o[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) o[ax] = p.rays_o[3 * (size_t)ray + ax];
        float a, b;
        segment_interval(sd, hd.tn, hd.delta, sample_interval(p.sp, ss, i), a, b);
        tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
        dl = __fsub_rn(b, a);
        float x[3], u[3];
        sample_point(o, d, tbar, x);
        region_coord(p.fp.boxes + 6 * k, x, u);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int l = 8 * h + j;
          if (l < p.lp.L) {
            const float2 v = encode_level_f32(p.lp, table, u, l);
            feat[2 * j] = v.x;
            feat[2 * j + 1] = v.y;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) s_F[(16 * h + j) * kFPitch + srow] = feat[j];
    if (p.rec32 && valid) {  // records for the backward: feature 16 h + j of tile row (t % 2) * 128 + srow
      float* rec = p.rec32 + (size_t)(t / kFwdSubPerTile) * kIn * (kWarp * kChunksPerTile) +
                   (t % kFwdSubPerTile) * kFwdRows + srow;
#pragma unroll
      for (int j = 0; j < 16; ++j) __stcs(rec + (16 * h + j) * (kWarp * kChunksPerTile), feat[j]);
    }
    __syncthreads();
    float acc[8][4];
    {
      const float* W1 = s_w;
      const float* W2 = s_w + kIn * kWidth;
      // h1 = relu(F W1) -> H; h2 = relu(h1 W2) -> F
      tile_ab<kFPitch, kFwdRows / 2, kIn, 4, kWidth>(s_F, W1, sb, 4 * ub, acc);
      tile_relu<8, 4>(acc);
      tile_st<kFPitch, kFwdRows / 2, 4>(s_H, sb, 4 * ub, acc);
      __syncthreads();
      tile_ab<kFPitch, kFwdRows / 2, kWidth, 4, kWidth>(s_H, W2, sb, 4 * ub, acc);
      tile_relu<8, 4>(acc);
      tile_st<kFPitch, kFwdRows / 2, 4>(s_F, sb, 4 * ub, acc);  // the features' reads ended before h1's store
    }
    __syncthreads();
    // ---- render (warps 0-3: thread = sample srow of slot q)
    if (h == 0 && sl.slot_ok) {  // warp-uniform; lanes of an unused part of a narrow slot are empty samples
      const float* W3 = s_w + kIn * kWidth + kWidth * kWidth;
      float raw[kOut] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
      for (int n = 0; n < kWidth; ++n) {
        const float hv = s_F[n * kFPitch + srow];  // h2
        const float4 w3 = *reinterpret_cast<const float4*>(W3 + 4 * n);
        raw[0] = fmaf(hv, w3.x, raw[0]);
        raw[1] = fmaf(hv, w3.y, raw[1]);
        raw[2] = fmaf(hv, w3.z, raw[2]);
        raw[3] = fmaf(hv, w3.w, raw[3]);
      }
      float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
      if (valid) {
        sigma = expf(raw[0]);
#pragma unroll
        for (int j = 0; j < 3; ++j) rgb[j] = 1.0f / (1.0f + expf(-raw[1 + j]));
      }
      const float tr = valid ? __fsub_rn(tbar, hd.tn) : 0.0f;
      const size_t slot = (size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c;
      if (p.smp4) {  // sample-level composition: every sample leaves the kernel
        if (sl.has) {
          p.smp4[slot * kWarp + sl.sl] = make_float4(sigma, rgb[0], rgb[1], rgb[2]);
          p.smp2[slot * kWarp + sl.sl] = make_float2(tr, dl);
          for (int j = sl.width + sl.sl; j < kWarp; j += sl.width) {  // a narrow chunk's other sample slots
            p.smp4[slot * kWarp + j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            p.smp2[slot * kWarp + j] = make_float2(0.0f, 0.0f);
          }
        }
      } else {
        const Partial pt = render_chunk(sigma, rgb, tr, dl, sl.sl, nullptr, 0, sl.width);
        if (sl.has && sl.sl == 0) {
          float4* dst = p.partials + 2 * slot;
          dst[0] = make_float4(pt.tau, pt.c0, pt.c1, pt.c2);
          dst[1] = make_float4(pt.A, pt.D, pt.L, 0.0f);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// k_field_fwd_persample_f32: the FP32 field with one sample per thread
// (256-row tiles, warp w on chunk slot w), weights read from shared memory as
// broadcasts. It serves the split representation (per-region density MLP,
// the shared colour MLP staged once per CTA after the density block), whose
// five-layer MLP measured slower as tiled products over 128-row sub-tiles
// (29.9 against 24.3 ms per grid8 step: seven barriers per sub-tile and a
// 16-output layer), and the fused MLP when a region's table outgrows what L2
// keeps for random gathers (city32: 196 ms against 263 ms tiled, whose
// gather and product phases alternate with the HBM latency exposed).
constexpr int kPerSampleThreads = kChunksPerTile * kWarp;

template <bool kSplit>
__global__ void __launch_bounds__(kPerSampleThreads, 2) k_field_fwd_persample_f32(FwdParams p) {
  extern __shared__ __align__(16) float s_dyn[];
  constexpr int kWFloats = kSplit ? kSplitSmemFloats : kMlpParams;
  float* s_w = s_dyn;                                              // kWFloats floats
  int32_t* s_base = reinterpret_cast<int32_t*>(s_dyn + kWFloats);  // [K+1]
  for (int i = threadIdx.x; i <= p.K; i += blockDim.x) s_base[i] = p.base[i];
  if (kSplit) load_color_f32(p.fp.mlp + (size_t)p.K * kDensityParams, s_w + kDensityParams);
  __syncthreads();
  const int n_tiles = *p.n_tiles;
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  int region = -1;
  const float2* table = nullptr;
  // Interleaved tiles: at any moment the whole GPU works on neighbouring
  // tiles of the region-major list, i.e. on one region whose tables then stay
  // resident in L2; a CTA switches region (and reloads weights) about K times.
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int chunk = t * kChunksPerTile + warp;
    const int k = region_of_chunk(s_base, p.K, t * kChunksPerTile);
    if (k != region) {
      __syncthreads();
      if (kSplit) load_density_f32(p.fp.mlp + (size_t)k * kDensityParams, s_w);
      else load_mlp_f32(p.fp.mlp + (size_t)k * kMlpParams, s_w);
      __syncthreads();
      region = k;
      table = reinterpret_cast<const float2*>(p.fp.tables) + (size_t)k * p.lp.E;
    }
    const SlotLane sl = slot_lane(p.chunks[chunk], lane);
    if (!sl.slot_ok) continue;  // warp-uniform (padding)
    // lanes of an unused part of a narrow slot take part in the scans as empty samples
    const uint2 ref = sl.ref;
    const uint32_t ray = sl.has ? ref.x : 0u;
    const int seg = ref.y >> 16, c = ref.y & 0xFFFF;
    RayHdr h = {0.0f, 0.0f, 0, 0};
    SegDesc sd = {0.0f, 0.0f, 0, 0};
    float o[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 0.0f};
    bool valid = false;
    int i = 0;
    SegSamples ss = {0, 0};
    if (sl.has) {
      h = p.hdr[ray];
      sd = p.segs[(size_t)ray * p.sp.max_seg + seg];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        o[ax] = p.rays_o[3 * (size_t)ray + ax];
        d[ax] = p.rays_d[3 * (size_t)ray + ax];
      }
      ss = seg_samples(p.sp, sd, ray, seg);
      i = c * kWarp + sl.sl;
      valid = i < ss.n;
    }
    float feat[kIn];
    float tbar = 0.0f, dl = 0.0f;
    if (valid) {
      float a, b;
      segment_interval(sd, h.tn, h.delta, sample_interval(p.sp, ss, i), a, b);
      tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
      dl = __fsub_rn(b, a);
      float x[3], u[3];
      sample_point(o, d, tbar, x);
      region_coord(p.fp.boxes + 6 * k, x, u);
      encode_f32(p.lp, table, u, feat);
    } else {
#pragma unroll
      for (int q = 0; q < kIn; ++q) feat[q] = 0.0f;
    }
    if (p.rec32) {  // records for the backward: feature j of sample (warp, lane), unit-major
      float* rec = p.rec32 + (size_t)t * kIn * (kWarp * kChunksPerTile) + warp * kWarp + lane;
#pragma unroll
      for (int q = 0; q < kIn; ++q) __stcs(rec + q * (kWarp * kChunksPerTile), feat[q]);
    }
    float raw[kOut];
    if (kSplit) {
      float sh[kSh];
      sh4_f32(d, sh);  // the lane's ray
      split_f32_smem(s_w, s_w + kDensityParams, feat, sh, raw);
    } else {
      mlp_f32_smem(s_w, feat, raw);
    }
    float sigma = 0.0f, rgb[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
      sigma = expf(raw[0]);
#pragma unroll
      for (int q = 0; q < 3; ++q) rgb[q] = 1.0f / (1.0f + expf(-raw[1 + q]));
    }
    const float tr = valid ? __fsub_rn(tbar, h.tn) : 0.0f;
    const size_t slot = (size_t)ray * p.sp.max_chunk + seg_chunk_base(sd) + c;
    if (p.smp4) {  // sample-level composition: every sample leaves the kernel
      if (sl.has) {
        p.smp4[slot * kWarp + sl.sl] = make_float4(sigma, rgb[0], rgb[1], rgb[2]);
        p.smp2[slot * kWarp + sl.sl] = make_float2(tr, dl);
        for (int j = sl.width + sl.sl; j < kWarp; j += sl.width) {  // a narrow chunk's other sample slots
          p.smp4[slot * kWarp + j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          p.smp2[slot * kWarp + j] = make_float2(0.0f, 0.0f);
        }
      }
      continue;
    }
    const Partial pt = render_chunk(sigma, rgb, tr, dl, sl.sl, nullptr, 0, sl.width);
    if (sl.has && sl.sl == 0) {
      float4* dst = p.partials + 2 * slot;
      dst[0] = make_float4(pt.tau, pt.c0, pt.c1, pt.c2);
      dst[1] = make_float4(pt.A, pt.D, pt.L, 0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// k_composite_samples: sample-level composition, one warp per ray. The ray's
// sample slots are visited in ray order (chunks of segments sorted along the
// ray), 32 at a time; within a step the lanes scan their optical depth and
// weights, across steps the prefix optical depth (log space, compensated), the
// accumulated C, A, D and the weight sums W, WT of the distortion's prefix form
// carry over:
//   T_i = exp(-sum_{j<i} tau_j), w_i = T_i (1 - exp(-tau_i)),
//   L = sum_i 2 w_i (t_i W_<i - WT_<i) + w_i^2 delta_i / 3.

__global__ void __launch_bounds__(256) k_composite_samples(int64_t R, SampParams sp, const RayHdr* __restrict__ hdr,
                                                           const float4* __restrict__ smp4,
                                                           const float2* __restrict__ smp2, float* __restrict__ rgb,
                                                           float* __restrict__ depth, float* __restrict__ opacity,
                                                           float* __restrict__ dist, const int64_t* __restrict__ out_index) {
  const int lane = threadIdx.x % kWarp;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  if (r >= R) return;  // warp-uniform
  const int64_t o = out_index ? out_index[r] : r;
  if (o < 0) return;
  const RayHdr h = hdr[r];
  float tau = 0.0f, comp = 0.0f;  // prefix optical depth before this step
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f, D = 0.0f, L = 0.0f, W = 0.0f, WT = 0.0f;
  for (int c = 0; c < h.nchunk; ++c) {
    const size_t at = ((size_t)r * sp.max_chunk + c) * kWarp + lane;
    const float4 a = smp4[at];
    const float2 b = smp2[at];
    const float t_i = a.x * b.y;  // optical depth of the sample
    const float incl = warp_inclusive_scan(t_i, lane);
    const float excl = warp_exclusive_from_inclusive(incl, lane);
    const float T = expf(-(tau + excl));
    const float w = T * -expm1f(-t_i);
    const float wt = w * b.x;
    const float W_lt = W + warp_exclusive_from_inclusive(warp_inclusive_scan(w, lane), lane);
    const float WT_lt = WT + warp_exclusive_from_inclusive(warp_inclusive_scan(wt, lane), lane);
    const float l = 2.0f * w * (b.x * W_lt - WT_lt) + w * w * b.y * (1.0f / 3.0f);
    C0 += warp_sum(w * a.y);
    C1 += warp_sum(w * a.z);
    C2 += warp_sum(w * a.w);
    const float ws = warp_sum(w), wts = warp_sum(wt);
    A += ws;
    D += wts;
    W += ws;
    WT += wts;
    L += warp_sum(l);
    const float y = __shfl_sync(0xFFFFFFFFu, incl, kWarp - 1) - comp;
    const float s = tau + y;
    comp = (s - tau) - y;
    tau = s;
  }
  if (lane == 0) {
    rgb[3 * o + 0] = C0;
    rgb[3 * o + 1] = C1;
    rgb[3 * o + 2] = C2;
    depth[o] = D + A * h.tn;
    opacity[o] = A;
    if (dist) dist[o] = L;
  }
}

// ---------------------------------------------------------------------------
// k_composite: Algorithm 1 + 2 over the chunk partials of one ray, with the
// prefix optical depth accumulated in log space (Kahan-compensated):
//   L += T^2 L_c + 2 T (D_c A - A_c D);  C += T C_c;  A += T A_c;  D += T D_c;
//   tau += tau_c;  T = exp(-tau).

__global__ void __launch_bounds__(256) k_composite(int64_t R, SampParams sp, const RayHdr* __restrict__ hdr,
                                                   const float4* __restrict__ partials, float* __restrict__ rgb,
                                                   float* __restrict__ depth, float* __restrict__ opacity,
                                                   float* __restrict__ dist, const int64_t* __restrict__ out_index) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int64_t o = out_index ? out_index[r] : r;  // output slot of this ray
  if (o < 0) return;
  const RayHdr h = hdr[r];
  float T = 1.0f, tau = 0.0f, comp = 0.0f;
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, A = 0.0f, D = 0.0f, L = 0.0f;
  const float4* src = partials + 2 * (size_t)r * sp.max_chunk;
  for (int c = 0; c < h.nchunk; ++c) {
    const float4 q0 = src[2 * c], q1 = src[2 * c + 1];
    const float S = q1.y * A - q1.x * D;
    L += T * T * q1.z + 2.0f * T * S;
    C0 += T * q0.y;
    C1 += T * q0.z;
    C2 += T * q0.w;
    A += T * q1.x;
    D += T * q1.y;
    const float y = q0.x - comp;
    const float s = tau + y;
    comp = (s - tau) - y;
    tau = s;
    T = expf(-tau);
  }
  rgb[3 * o + 0] = C0;
  rgb[3 * o + 1] = C1;
  rgb[3 * o + 2] = C2;
  depth[o] = D + A * h.tn;
  opacity[o] = A;
  if (dist) dist[o] = L;
}

// ---------------------------------------------------------------------------
// Host side.

namespace {

thread_local std::string g_last_error;

nerfxl_status fail(nerfxl_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int g_num_sms = 0;

}  // namespace

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    g_num_sms = n;
  }
  return g_num_sms;
}

const char* last_error() { return g_last_error.c_str(); }
nerfxl_status set_error(nerfxl_status st, const std::string& msg) { return fail(st, msg); }

int effective_max_seg(const nerfxl_field* f, const nerfxl_sampling* s) {
  int ms = s->max_segments > 0 ? s->max_segments : std::min(f->K, (int)kMaxSeg);
  return ms;
}

int max_chunks(int S, int max_seg) { return max_seg + (S - 1) / kWarp; }

RecordOut record_out(char* ws, const Layout& L) {
  RecordOut r = {nullptr, nullptr, nullptr, nullptr, 0};
  if (L.rec_tiles == 0) return r;
  r.feat = reinterpret_cast<uint4*>(ws + L.rec_feat);
  r.geom = reinterpret_cast<float*>(ws + L.rec_geom);
  r.pos = reinterpret_cast<int32_t*>(ws + L.rec_pos);
  r.gfeat = L.gfeat_tiles ? reinterpret_cast<uint32_t*>(ws + L.gfeat) : nullptr;
  r.gfeat_tiles = L.gfeat_tiles;
  return r;
}

Layout layout(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R, int for_backward) {
  Layout L;
  const int ms = effective_max_seg(f, s);
  const int mc = max_chunks(s->n_samples, ms);
  const int K = f->K;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  L.hdr = take(sizeof(int32_t) * 16);
  L.counts = take(sizeof(int32_t) * 3 * K);  // chunks per region, then those of width 16, width 8
  L.cursor = take(sizeof(int32_t) * 3 * K);
  L.zero_end = off;
  L.base = take(sizeof(int32_t) * (K + 1));
  L.ray_hdr = take(sizeof(RayHdr) * R);
  L.segs = take(sizeof(SegDesc) * R * ms);
  L.max_int = s->n_samples + ms - 1;
  L.seg_keep = L.kept = 0;
  if (f->occupancy) {  // before the backward-only regions: forward and backward layouts agree
    L.seg_keep = take(sizeof(int32_t) * R * ms);
    L.kept = take(sizeof(uint16_t) * R * L.max_int);
  }
  L.chunk_cap = (int64_t)R * mc + (int64_t)kChunksPerTile * K;
  L.chunks = take(sizeof(Slot) * L.chunk_cap);  // slots (at most one per chunk)
  L.partials = take(sizeof(float4) * 2 * R * mc);
  L.dpartials = for_backward ? take(sizeof(float4) * 2 * R * mc) : 0;
  L.rec_feat = L.rec_geom = L.rec_dpart = L.rec_pos = 0;
  L.rec_tiles = 0;
  if (for_backward && (f->mlp_dtype == NERFXL_BF16 || f->mlp_dtype == NERFXL_F16)) {
    L.rec_tiles = (L.chunk_cap + 3) / 4;
    L.rec_feat = take(kRecFeatBytes * L.rec_tiles);
    L.rec_geom = take(sizeof(float) * kGeomFloats * L.rec_tiles);
    L.rec_dpart = take(sizeof(float4) * 2 * 16 * L.rec_tiles);
    L.rec_pos = take(sizeof(int32_t) * R * mc);
  }
  L.rec32 = 0;
  if (for_backward && f->mlp_dtype == NERFXL_F32)
    L.rec32 = take(sizeof(float) * kIn * kWarp * kChunksPerTile * (size_t)((L.chunk_cap + kChunksPerTile - 1) / kChunksPerTile));
  L.smp4 = L.smp2 = 0;
  if (s->flags & NERFXL_SAMPLE_COMPOSITE) {
    L.smp4 = take(sizeof(float4) * (size_t)R * mc * kWarp);
    L.smp2 = take(sizeof(float2) * (size_t)R * mc * kWarp);
  }
  // last, so that the regions before it agree between forward and backward
  // layouts
  L.gfeat = 0;
  L.gfeat_tiles = 0;
  if (grouped_gather(f, s, R)) {
    L.gfeat_tiles = std::min<int64_t>((L.chunk_cap + 3) / 4, gather_window_tiles());
    L.gfeat = take(sizeof(uint32_t) * 128 * (size_t)(f->L + kGatherCoordWords) * (size_t)L.gfeat_tiles);
  }
  L.total = off;
  L.max_seg = ms;
  L.max_chunk = mc;
  return L;
}

nerfxl_status validate(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R) {
  if (!f || !s) return fail(NERFXL_E_INVALID, "null field or sampling");
  if (f->K < 1 || f->K > NERFXL_MAX_REGIONS) return fail(NERFXL_E_INVALID, "K out of range");
  if (f->L < 1 || f->L > NERFXL_MAX_LEVELS) return fail(NERFXL_E_INVALID, "L out of range");
  if (f->log2_T < 1 || f->log2_T > 24) return fail(NERFXL_E_INVALID, "log2_T out of range");
  if (f->F != 2 || f->mlp_in != kIn || f->mlp_width != kWidth || f->L * f->F > kIn)
    return fail(NERFXL_E_UNSUPPORTED, "only F=2, mlp_in=32, width=64, L*F<=32 are built");
  for (int l = 0; l < f->L; ++l)
    if (f->level_res[l] < 1 || f->level_res[l] > (1 << 20)) return fail(NERFXL_E_INVALID, "level_res out of range");
  if (s->n_samples < 1 || s->n_samples > 16384) return fail(NERFXL_E_INVALID, "n_samples out of range");
  const int ms = effective_max_seg(f, s);
  if (ms < 1 || ms > kMaxSeg) return fail(NERFXL_E_UNSUPPORTED, "max_segments must be in [1, 32]");
  if (max_chunks(s->n_samples, ms) > 0xFFFF) return fail(NERFXL_E_UNSUPPORTED, "too many chunks per ray");
  if (R < 0 || R > (int64_t)0x7FFFFFFF) return fail(NERFXL_E_INVALID, "n_rays out of range");
  if (!f->boxes || !f->tables || !f->mlp) return fail(NERFXL_E_INVALID, "null field pointer");
  if (f->occupancy && (f->occ_res < 1 || f->occ_res > 1024))
    return fail(NERFXL_E_INVALID, "occupancy grid resolution must be in [1, 1024]");
  if (f->arch != NERFXL_ARCH_FUSED && f->arch != NERFXL_ARCH_SPLIT) return fail(NERFXL_E_INVALID, "unknown arch");
  if (f->arch == NERFXL_ARCH_SPLIT && f->mlp_dtype == NERFXL_E4M3)
    return fail(NERFXL_E_UNSUPPORTED, "the split representation is built for FP32, BF16 and FP16 MLPs");
  return NERFXL_OK;
}

LevelParams level_params(const nerfxl_field* f) {
  LevelParams lp;
  const int64_t T = int64_t(1) << f->log2_T;
  int64_t off = 0;
  lp.dense_mask = 0;
  for (int l = 0; l < kMaxLevels; ++l) {
    lp.N[l] = 1;
    lp.off[l] = 0;
  }
  for (int l = 0; l < f->L; ++l) {
    const int64_t side = (int64_t)f->level_res[l] + 1;
    const int64_t verts = side * side * side;
    const bool dense = verts <= T;
    lp.N[l] = f->level_res[l];
    lp.off[l] = (uint32_t)off;
    if (dense) lp.dense_mask |= 1u << l;
    off += dense ? (verts + 7) / 8 * 8 : T;
  }
  lp.hash_mask = (uint32_t)(T - 1);
  lp.L = f->L;
  lp.E = (uint32_t)off;
  return lp;
}

SampParams samp_params(const nerfxl_field* f, const nerfxl_sampling* s) {
  SampParams sp;
  sp.S = s->n_samples;
  sp.max_seg = effective_max_seg(f, s);
  sp.max_chunk = max_chunks(s->n_samples, sp.max_seg);
  sp.t_min = s->t_min;
  sp.seg_keep = nullptr;
  sp.kept = nullptr;
  sp.max_int = s->n_samples + sp.max_seg - 1;
  return sp;
}

SampParams samp_params(const nerfxl_field* f, const nerfxl_sampling* s, char* ws, const Layout& L) {
  SampParams sp = samp_params(f, s);
  if (f->occupancy) {
    sp.seg_keep = reinterpret_cast<const int32_t*>(ws + L.seg_keep);
    sp.kept = reinterpret_cast<const uint16_t*>(ws + L.kept);
  }
  return sp;
}

nerfxl_status launch_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NERFXL_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return NERFXL_OK;
}

// Process-wide count of the kernels this library has launched.
std::atomic<int64_t> g_launches(0);

nerfxl_status kernel_launched(const char* name) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return launch_check(name);
}

// Steps (a) and bucketing, shared by forward, backward and debug calls.
nerfxl_status run_sampling(const nerfxl_field* f, const SampParams& sp, int64_t R, const float* rays_o,
                           const float* rays_d, char* ws, const Layout& L, cudaStream_t stream) {
  const int K = f->K;
  if (cudaMemsetAsync(ws, 0, L.zero_end, stream) != cudaSuccess) return launch_check("workspace clear");
  int32_t* hdr_words = reinterpret_cast<int32_t*>(ws + L.hdr);
  const int threads = 256;
  const int blocks = (int)((R + threads - 1) / threads);
  if (R > 0) {
    const size_t smem = sizeof(float) * 6 * K + sizeof(int32_t) * 3 * K;
    int32_t* counts = reinterpret_cast<int32_t*>(ws + L.counts);
    k_segments<<<blocks, threads, smem, stream>>>(rays_o, rays_d, R, f->boxes, K, sp,
                                                  reinterpret_cast<RayHdr*>(ws + L.ray_hdr),
                                                  reinterpret_cast<SegDesc*>(ws + L.segs),
                                                  f->occupancy ? nullptr : counts, hdr_words + 0);
    nerfxl_status st = kernel_launched("k_segments");
    if (st != NERFXL_OK) return st;
    if (f->occupancy) {
      if (!sp.seg_keep) return set_error(NERFXL_E_INVALID, "occupancy lists not attached to the sampling");
      const int64_t warps_per_block = threads / kWarp;
      k_skip_empty<<<(int)((R + warps_per_block - 1) / warps_per_block), threads, smem + sizeof(float) * 3 * K,
                     stream>>>(
          rays_o, rays_d, R, f->boxes, K, sp, f->occupancy, f->occ_res, reinterpret_cast<RayHdr*>(ws + L.ray_hdr),
          reinterpret_cast<SegDesc*>(ws + L.segs), reinterpret_cast<int32_t*>(ws + L.seg_keep),
          reinterpret_cast<uint16_t*>(ws + L.kept), counts, hdr_words + 0);
      st = kernel_launched("k_skip_empty");
      if (st != NERFXL_OK) return st;
    }
  }
  k_region_scan<<<1, 32, 0, stream>>>(reinterpret_cast<int32_t*>(ws + L.counts), K, kChunksPerTile,
                                      reinterpret_cast<int32_t*>(ws + L.base), reinterpret_cast<uint2*>(ws + L.chunks),
                                      hdr_words + 1);
  nerfxl_status st = kernel_launched("k_region_scan");
  if (st != NERFXL_OK) return st;
  if (R > 0) {
    k_fill_chunks<<<blocks, threads, sizeof(int32_t) * 6 * K, stream>>>(
        R, K, sp, reinterpret_cast<RayHdr*>(ws + L.ray_hdr), reinterpret_cast<SegDesc*>(ws + L.segs),
        reinterpret_cast<int32_t*>(ws + L.counts), reinterpret_cast<int32_t*>(ws + L.base),
        reinterpret_cast<int32_t*>(ws + L.cursor), reinterpret_cast<uint2*>(ws + L.chunks));
    st = kernel_launched("k_fill_chunks");
    if (st != NERFXL_OK) return st;
  }
  return NERFXL_OK;
}

cudaEvent_t g_prof[2] = {nullptr, nullptr};

void profile_mark(int which, cudaStream_t stream) {
  if (g_prof[which]) cudaEventRecord(g_prof[which], stream);
}

int fwd_grid(int64_t max_tiles, int ctas_per_sm) {
  const int64_t g = (int64_t)num_sms() * ctas_per_sm;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, max_tiles));
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" {

int64_t nerfxl_table_entries(const int32_t* level_res, int32_t L, int32_t log2_T) {
  if (!level_res || L < 1 || L > NERFXL_MAX_LEVELS || log2_T < 1 || log2_T > 24) return -1;
  const int64_t T = int64_t(1) << log2_T;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    if (level_res[l] < 1) return -1;
    const int64_t side = (int64_t)level_res[l] + 1;
    const int64_t verts = side * side * side;
    off += verts <= T ? (verts + 7) / 8 * 8 : T;
  }
  return off;
}

int64_t nerfxl_mlp_params(int32_t mlp_in, int32_t width) {
  return (int64_t)mlp_in * width + (int64_t)width * width + (int64_t)width * 4;
}

int64_t nerfxl_field_mlp_params(const nerfxl_field* f) {
  if (!f || f->K < 1 || f->mlp_in < 1 || f->mlp_width < 1) return -1;
  const int64_t W = f->mlp_width;
  if (f->arch == NERFXL_ARCH_SPLIT)
    return (int64_t)f->K * (f->mlp_in * W + W * kGeo) + (kColorIn * W + W * W + W * kOut);
  if (f->arch != NERFXL_ARCH_FUSED) return -1;
  return (int64_t)f->K * nerfxl_mlp_params(f->mlp_in, f->mlp_width);
}

int32_t nerfxl_max_chunks(const nerfxl_sampling* s, int32_t K) {
  if (!s) return -1;
  const int ms = s->max_segments > 0 ? s->max_segments : std::min<int>(K, kMaxSeg);
  return max_chunks(s->n_samples, ms);
}

size_t nerfxl_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, int32_t for_backward) {
  if (validate(f, s, n_rays) != NERFXL_OK) return 0;
  return layout(f, s, n_rays, for_backward).total;
}

nerfxl_status nerfxl_render_fwd(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                const float* rays_o, const float* rays_d, float* rgb, float* depth, float* opacity,
                                float* dist, void* workspace, size_t ws_bytes, cudaStream_t stream) {
  return render_fwd_impl(f, s, n_rays, rays_o, rays_d, rgb, depth, opacity, dist, nullptr, workspace, ws_bytes,
                         stream);
}

}  // extern "C"

namespace nerfxl {

nerfxl_status render_fwd_impl(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, const float* rays_o,
                              const float* rays_d, float* rgb, float* depth, float* opacity, float* dist,
                              const int64_t* out_index, void* workspace, size_t ws_bytes, cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  const bool tab_ok = f->table_dtype == NERFXL_F32 || f->table_dtype == NERFXL_F16;
  const bool tc_mlp = f->mlp_dtype == NERFXL_BF16 || f->mlp_dtype == NERFXL_F16 || f->mlp_dtype == NERFXL_E4M3;
  if (!tab_ok || !(tc_mlp || f->mlp_dtype == NERFXL_F32) || (f->mlp_dtype == NERFXL_F32 && f->table_dtype != NERFXL_F32))
    return set_error(NERFXL_E_UNSUPPORTED, "supported: FP32 tables + FP32 MLP, or FP32/FP16 tables + BF16/FP16/E4M3 MLP");
  if (n_rays > 0 && (!rays_o || !rays_d || !rgb || !depth || !opacity))
    return set_error(NERFXL_E_INVALID, "null ray or output pointer");
  const Layout L = layout(f, s, n_rays, 0);
  if (!workspace || ws_bytes < L.total) return set_error(NERFXL_E_WORKSPACE, "workspace too small");
  char* ws = static_cast<char*>(workspace);
  const SampParams sp = samp_params(f, s, ws, L);
  st = run_sampling(f, sp, n_rays, rays_o, rays_d, ws, L, stream);
  if (st != NERFXL_OK) return st;
  if (n_rays == 0) return NERFXL_OK;
  if (tc_mlp && (s->flags & NERFXL_SAMPLE_COMPOSITE))
    return set_error(NERFXL_E_UNSUPPORTED, "sample-level composition is built for the FP32 MLP only");
  if (tc_mlp) {
    RecordOut rec = {nullptr, nullptr, nullptr, nullptr, 0};
    if (s->flags & NERFXL_SAVE_FEATURES) {
      if (f->mlp_dtype == NERFXL_E4M3) return set_error(NERFXL_E_UNSUPPORTED, "E4M3 is forward-only");
      const Layout LB = layout(f, s, n_rays, 1);
      if (ws_bytes < LB.total) return set_error(NERFXL_E_WORKSPACE, "NERFXL_SAVE_FEATURES needs a backward workspace");
      rec = record_out(ws, LB);
    }
    st = launch_field_fwd_tc(f, sp, level_params(f), rays_o, rays_d, ws, L, rec, stream);
    if (st != NERFXL_OK) return st;
    k_composite<<<(int)((n_rays + 255) / 256), 256, 0, stream>>>(
        n_rays, sp, reinterpret_cast<const RayHdr*>(ws + L.ray_hdr), reinterpret_cast<const float4*>(ws + L.partials),
        rgb, depth, opacity, dist, out_index);
    return kernel_launched("k_composite");
  }

  FwdParams p;
  p.rays_o = rays_o;
  p.rays_d = rays_d;
  p.fp.boxes = f->boxes;
  p.fp.tables = static_cast<const float*>(f->tables);
  p.fp.mlp = static_cast<const float*>(f->mlp);
  p.lp = level_params(f);
  p.sp = sp;
  p.K = f->K;
  p.hdr = reinterpret_cast<const RayHdr*>(ws + L.ray_hdr);
  p.segs = reinterpret_cast<const SegDesc*>(ws + L.segs);
  p.base = reinterpret_cast<const int32_t*>(ws + L.base);
  p.chunks = reinterpret_cast<const Slot*>(ws + L.chunks);
  p.n_tiles = reinterpret_cast<const int32_t*>(ws + L.hdr) + 1;
  p.partials = reinterpret_cast<float4*>(ws + L.partials);
  const bool per_sample = (s->flags & NERFXL_SAMPLE_COMPOSITE) != 0;
  p.smp4 = per_sample ? reinterpret_cast<float4*>(ws + L.smp4) : nullptr;
  p.smp2 = per_sample ? reinterpret_cast<float2*>(ws + L.smp2) : nullptr;
  const bool split = f->arch == NERFXL_ARCH_SPLIT;
  p.rec32 = nullptr;
  if (s->flags & NERFXL_SAVE_FEATURES) {
    const Layout LB = layout(f, s, n_rays, 1);
    if (ws_bytes < LB.total) return set_error(NERFXL_E_WORKSPACE, "NERFXL_SAVE_FEATURES needs a backward workspace");
    p.rec32 = reinterpret_cast<float*>(ws + LB.rec32);
  }
  // one sample per thread (256-row tiles): the split MLP, or a fused one whose region table is beyond
  // what L2 keeps for random gathers (the threshold of the level-grouped gather)
  const size_t table_bytes = (size_t)nerfxl_table_entries(f->level_res, f->L, f->log2_T) * f->F * sizeof(float);
  if (split || table_bytes > group_min_bytes()) {
    const size_t smem = sizeof(float) * (split ? kSplitSmemFloats : kMlpParams) + sizeof(int32_t) * (f->K + 1);
    const int grid = fwd_grid(L.chunk_cap / kChunksPerTile, 2);
    void (*kern)(FwdParams) = split ? k_field_fwd_persample_f32<true> : k_field_fwd_persample_f32<false>;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                                 cudaSuccess)
      return launch_check("k_field_fwd_persample_f32 smem attribute");
    profile_mark(0, stream);
    kern<<<grid, kPerSampleThreads, smem, stream>>>(p);
    profile_mark(1, stream);
    st = kernel_launched("k_field_fwd_persample_f32");
  } else {  // tiled products over 128-row sub-tiles
    const size_t smem = sizeof(float) * (kMlpParams + 2 * kWidth * kFPitch) + sizeof(int32_t) * (f->K + 1);
    if (smem > 232448 / 2 - 1024)
      return set_error(NERFXL_E_UNSUPPORTED, "too many regions for the forward's shared memory");
    const int grid = fwd_grid(L.chunk_cap / 4, 2);
    if (cudaFuncSetAttribute(k_field_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return launch_check("k_field_fwd_f32 smem attribute");
    profile_mark(0, stream);
    k_field_fwd_f32<<<grid, kFwdThreads, smem, stream>>>(p);
    profile_mark(1, stream);
    st = kernel_launched("k_field_fwd_f32");
  }
  if (st != NERFXL_OK) return st;
  if (per_sample) {
    const int64_t threads = n_rays * kWarp;
    k_composite_samples<<<(int)((threads + 255) / 256), 256, 0, stream>>>(n_rays, sp, p.hdr, p.smp4, p.smp2, rgb,
                                                                           depth, opacity, dist, out_index);
    return kernel_launched("k_composite_samples");
  }
  k_composite<<<(int)((n_rays + 255) / 256), 256, 0, stream>>>(n_rays, sp, p.hdr, p.partials, rgb, depth, opacity,
                                                                dist, out_index);
  return kernel_launched("k_composite");
}

}  // namespace nerfxl

extern "C" {

int64_t nerfxl_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

nerfxl_status nerfxl_check(const void* workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!workspace || ws_bytes < 64) return set_error(NERFXL_E_WORKSPACE, "no workspace");
  int32_t flags = 0;
  if (cudaMemcpyAsync(&flags, workspace, sizeof(flags), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return launch_check("nerfxl_check");
  if (flags & kErrTimeout) return set_error(NERFXL_E_TIMEOUT, "a bounded wait on the tensor-core pipeline expired");
  if (flags & kErrOverflow) return set_error(NERFXL_E_OVERFLOW, "a ray crossed more regions than max_segments");
  return NERFXL_OK;
}

nerfxl_status nerfxl_workspace_stats(const void* workspace, size_t ws_bytes, int64_t* n_samples, int64_t* n_chunks,
                                     cudaStream_t stream) {
  if (!workspace || ws_bytes < 64) return set_error(NERFXL_E_WORKSPACE, "no workspace");
  int64_t v[2] = {0, 0};
  if (cudaMemcpyAsync(v, static_cast<const char*>(workspace) + 8, sizeof(v), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return launch_check("nerfxl_workspace_stats");
  if (n_samples) *n_samples = v[0];
  if (n_chunks) *n_chunks = v[1];
  return NERFXL_OK;
}

nerfxl_status nerfxl_region_chunks(const void* workspace, size_t ws_bytes, int32_t K, int32_t* counts,
                                   cudaStream_t stream) {
  if (!workspace || !counts || K < 1 || K > NERFXL_MAX_REGIONS) return set_error(NERFXL_E_INVALID, "bad arguments");
  // the counts follow the 256-byte header block (see layout())
  const size_t off = align_up(sizeof(int32_t) * 16, 256);
  if (ws_bytes < off + sizeof(int32_t) * (size_t)K) return set_error(NERFXL_E_WORKSPACE, "workspace too small");
  if (cudaMemcpyAsync(counts, static_cast<const char*>(workspace) + off, sizeof(int32_t) * (size_t)K,
                      cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return launch_check("nerfxl_region_chunks");
  return NERFXL_OK;
}

nerfxl_status nerfxl_set_profile_events(cudaEvent_t start, cudaEvent_t stop) {
  if ((start == nullptr) != (stop == nullptr)) return set_error(NERFXL_E_INVALID, "give both events or neither");
  g_prof[0] = start;
  g_prof[1] = stop;
  return NERFXL_OK;
}

const char* nerfxl_last_error(void) { return last_error(); }

}  // extern "C"
