// Device-side building blocks of the NeRF-XL hot path (arXiv 2404.16221).
//
// Geometry (Sec. 4.2) and the hash index (App. A.1, Instant-NGP encoding)
// are written with explicit round-to-nearest intrinsics so that nvcc cannot
// contract them into fused multiply-adds: region assignment, interval edges
// and table indices are then identical to any IEEE FP32 evaluation in the
// same operation order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nerfxl.h"

namespace nerfxl {

constexpr int kWarp = 32;
constexpr int kMaxSeg = NERFXL_MAX_SEGMENTS;
constexpr int kMaxLevels = NERFXL_MAX_LEVELS;
constexpr uint32_t kEmptyChunk = 0xFFFFFFFFu;
constexpr uint32_t kHashPrime2 = 2654435761u;  // Instant-NGP spatial hash primes (pi_1 = 1)
constexpr uint32_t kHashPrime3 = 805459861u;

// Fixed-size MLP the kernels are specialised for: 32 -> 64 -> 64 -> 4.
constexpr int kIn = 32;
constexpr int kWidth = 64;
constexpr int kOut = 4;
constexpr int kMlpParams = kIn * kWidth + kWidth * kWidth + kWidth * kOut;

// Chunk slots per CTA tile (one warp per slot); region buckets are padded to it.
constexpr int kChunksPerTile = 8;

// A chunk is up to 32 consecutive samples of one ray segment, the unit of the
// local render. A slot is the 32 rows (one warp) chunks are evaluated in: one
// chunk (width 32, lane = sample), two chunks of at most 16 samples (width 16:
// lanes 0-15 and 16-31) or four of at most 8 (width 8) - segment tails and
// short segments. A slot is four references {ray, seg << 16 | chunk}; the
// unused references of a narrow slot hold kUnusedPart, a padding slot holds
// kEmptyChunk everywhere, and a slot's width is 8 if its third reference is
// not kEmptyChunk, else 16 if its second is not, else 32.
constexpr uint32_t kUnusedPart = 0xFFFFFFFEu;

struct Slot {
  uint4 a, b;  // references 0, 1 and 2, 3
};

struct SlotLane {
  uint2 ref;     // the lane's chunk {ray, seg << 16 | chunk}
  bool slot_ok;  // the slot is not padding (warp-uniform)
  bool has;      // the lane's part of the slot holds a chunk
  int width;     // lanes per chunk in this slot: 32, 16 or 8
  int sl;        // the lane's sample index within its chunk
  int part;      // which chunk of the slot: lane / width
};

__device__ __forceinline__ SlotLane slot_lane(const Slot& s, int lane) {
  SlotLane o;
  o.width = s.b.x != kEmptyChunk ? 8 : (s.a.z != kEmptyChunk ? 16 : 32);
  o.part = lane / o.width;
  o.sl = lane % o.width;
  o.ref = o.part == 0 ? make_uint2(s.a.x, s.a.y)
                      : (o.part == 1 ? make_uint2(s.a.z, s.a.w) : (o.part == 2 ? make_uint2(s.b.x, s.b.y)
                                                                             : make_uint2(s.b.z, s.b.w)));
  o.slot_ok = s.a.x != kEmptyChunk;
  o.has = o.ref.x < kUnusedPart;
  return o;
}

// A slot's sample counts as the tensor-core records keep them (one int32:
// 6 bits per chunk, chunk p at bit 6 p, the width code at bit 24: 0 for 32,
// 1 for 16, 2 for 8), resolved for a lane: its chunk's count, width, index
// in it and part. 0 is an empty slot.
struct SlotCount {
  int n, width, sl, part;
};

__device__ __forceinline__ int32_t slot_count_word(int width, const int n[4]) {
  const int code = width == 32 ? 0 : (width == 16 ? 1 : 2);
  return n[0] | (n[1] << 6) | (n[2] << 12) | (n[3] << 18) | (code << 24);
}

__device__ __forceinline__ SlotCount slot_count(int32_t word, int lane) {
  SlotCount o;
  o.width = 32 >> ((word >> 24) & 3);
  o.part = lane / o.width;
  o.sl = lane % o.width;
  o.n = (word >> (6 * o.part)) & 63;
  return o;
}

// Chunks of a segment of n samples, and the width its last chunk takes in a
// slot: 8 for at most 8 samples, 16 for at most 16, else 32 (also for an
// emptied segment, which has no chunk).
__device__ __forceinline__ int seg_chunks(int n) { return (n + 31) / 32; }
__device__ __forceinline__ int seg_tail_width(int n) {
  if (n <= 0) return 32;
  const int tail = n - 32 * ((n - 1) / 32);
  return tail <= 8 ? 8 : (tail <= 16 ? 16 : 32);
}

// Error flags written into the workspace header.
constexpr int kErrOverflow = 1;
constexpr int kErrTimeout = 2;  // a bounded wait on the tensor-core pipeline expired

// Per-level layout of a region table, passed by value in kernel parameters.
struct LevelParams {
  int32_t N[kMaxLevels];       // cells per axis
  uint32_t off[kMaxLevels];    // first entry of the level
  uint32_t dense_mask;         // bit l set: level l stored densely
  uint32_t hash_mask;          // 2^log2_T - 1
  int32_t L;
  uint32_t E;                  // entries per region
};

// Sampling description shared by the kernels. With an occupancy grid the
// samples of a segment are the intervals whose cell is occupied: seg_keep
// holds, per segment, their count (low 16 bits) and the first slot of their
// list in kept (high 16 bits); kept lists, per ray, interval indices within
// their segment in increasing order. Without a grid seg_keep is NULL and
// sample i of a segment is its interval i.
struct SampParams {
  int32_t S;          // grid intervals over [tn, tf]
  int32_t max_seg;    // segments per ray bound (<= kMaxSeg)
  int32_t max_chunk;  // chunks per ray bound
  float t_min;
  const int32_t* seg_keep;  // [R][max_seg], or NULL
  const uint16_t* kept;     // [R][max_int]
  int32_t max_int;          // list slots per ray (intervals per ray bound)
};

// One ray's sampling header.
struct __align__(16) RayHdr {
  float tn;       // first segment start
  float delta;    // (tf - tn) / S
  int32_t nseg;
  int32_t nchunk;
};

// One segment: [t0, t1] inside region; first interior grid edge j_lo and
// interval count n; chunk_base = index of its first chunk within the ray.
struct __align__(16) SegDesc {
  float t0, t1;
  int32_t jlo_n;      // j_lo (low 16 bits) | n (high 16 bits)
  int32_t reg_cb;     // region (low 16 bits) | chunk_base (high 16 bits)
};

__device__ __forceinline__ int seg_jlo(const SegDesc& s) { return s.jlo_n & 0xFFFF; }
__device__ __forceinline__ int seg_n(const SegDesc& s) { return (s.jlo_n >> 16) & 0xFFFF; }
__device__ __forceinline__ int seg_region(const SegDesc& s) { return s.reg_cb & 0xFFFF; }
__device__ __forceinline__ int seg_chunk_base(const SegDesc& s) { return (s.reg_cb >> 16) & 0xFFFF; }

// Samples of one segment: their count and where their interval list starts
// (list < 0: sample i is interval i).
struct SegSamples {
  int n;
  int64_t list;
};

__device__ __forceinline__ SegSamples seg_samples(const SampParams& sp, const SegDesc& sd, size_t ray, int seg) {
  if (!sp.seg_keep) return {seg_n(sd), -1};
  const int kp = sp.seg_keep[ray * sp.max_seg + seg];
  return {kp & 0xFFFF, (int64_t)ray * sp.max_int + ((kp >> 16) & 0xFFFF)};
}

// Interval index of sample i (< n) of a segment.
__device__ __forceinline__ int sample_interval(const SampParams& sp, const SegSamples& ss, int i) {
  return ss.list < 0 ? i : (int)sp.kept[ss.list + i];
}

// ---------------------------------------------------------------------------
// Geometry (Sec. 4.2).

// Slab test: t0 = max(t_min, max_axis min(ta, tb)), t1 = min_axis max(ta, tb),
// ta = (bmin - o) * (1/d), tb = (bmax - o) * (1/d); fminf/fmaxf ignore NaN.
__device__ __forceinline__ bool slab(const float o[3], const float inv_d[3], const float* box, float t_min,
                                     float& t0, float& t1) {
  float tn = -INFINITY, tf = INFINITY;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float ta = __fmul_rn(__fsub_rn(box[ax], o[ax]), inv_d[ax]);
    const float tb = __fmul_rn(__fsub_rn(box[3 + ax], o[ax]), inv_d[ax]);
    tn = fmaxf(tn, fminf(ta, tb));
    tf = fminf(tf, fmaxf(ta, tb));
  }
  tn = fmaxf(tn, t_min);
  t0 = tn;
  t1 = tf;
  return tf > tn;
}

// Grid edge e_j = tn + j * delta, two roundings.
__device__ __forceinline__ float grid_edge(float tn, float delta, int j) {
  return __fadd_rn(tn, __fmul_rn((float)j, delta));
}

// First j in [1, S] with e_j > t (S if none): estimate, then walk to the exact
// boundary of the monotone sequence e_j (each walk is bounded by S steps).
__device__ __forceinline__ int first_edge_above(float tn, float delta, int S, float t) {
  float est = __fdiv_rn(__fsub_rn(t, tn), delta);
  est = fminf(fmaxf(est, 0.0f), (float)S);
  int j = max(1, (int)est);
  for (int it = 0; it <= S && j > 1 && grid_edge(tn, delta, j - 1) > t; ++it) --j;
  for (int it = 0; it <= S && j < S && !(grid_edge(tn, delta, j) > t); ++it) ++j;
  return j;
}

// First j in [1, S] with e_j >= t (S if none).
__device__ __forceinline__ int first_edge_at_or_above(float tn, float delta, int S, float t) {
  float est = __fdiv_rn(__fsub_rn(t, tn), delta);
  est = fminf(fmaxf(est, 0.0f), (float)S);
  int j = max(1, (int)est);
  for (int it = 0; it <= S && j > 1 && grid_edge(tn, delta, j - 1) >= t; ++it) --j;
  for (int it = 0; it <= S && j < S && !(grid_edge(tn, delta, j) >= t); ++it) ++j;
  return j;
}

// Segments of one ray, sorted by (t0, region). Returns the number of hits
// (possibly > max_seg: only the first max_seg in sort order are kept and the
// caller flags an overflow).
__device__ __forceinline__ int ray_segments(const float o[3], const float d[3], const float* boxes, int K,
                                            float t_min, int max_seg, float* st0, float* st1, int* sreg) {
  float inv_d[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) inv_d[ax] = __fdiv_rn(1.0f, d[ax]);
  int n = 0, hits = 0;
  for (int k = 0; k < K; ++k) {
    float t0, t1;
    if (!slab(o, inv_d, boxes + 6 * k, t_min, t0, t1)) continue;
    ++hits;
    // insertion into the sorted prefix (K is scanned in increasing order, so
    // equal t0 keeps the lower region id first)
    int pos = n;
    while (pos > 0 && st0[pos - 1] > t0) --pos;
    if (pos >= max_seg) continue;
    const int last = min(n, max_seg - 1);
    for (int q = last; q > pos; --q) {
      st0[q] = st0[q - 1];
      st1[q] = st1[q - 1];
      sreg[q] = sreg[q - 1];
    }
    st0[pos] = t0;
    st1[pos] = t1;
    sreg[pos] = k;
    n = min(n + 1, max_seg);
  }
  return hits;
}

// Interval i of a segment: [a, b].
__device__ __forceinline__ void segment_interval(const SegDesc& sd, float tn, float delta, int i, float& a,
                                                 float& b) {
  const int jlo = seg_jlo(sd), n = seg_n(sd);
  a = (i == 0) ? sd.t0 : grid_edge(tn, delta, jlo + i - 1);
  b = (i == n - 1) ? sd.t1 : grid_edge(tn, delta, jlo + i);
}

// Sample point x = o + tbar * d, two roundings per axis.
__device__ __forceinline__ void sample_point(const float o[3], const float d[3], float tbar, float x[3]) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) x[ax] = __fadd_rn(o[ax], __fmul_rn(tbar, d[ax]));
}

// Region-local coordinate u = clamp((x - bmin) * (1 / (bmax - bmin)), 0, 1).
__device__ __forceinline__ void region_coord(const float* box, const float x[3], float u[3]) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float inv_ext = __fdiv_rn(1.0f, __fsub_rn(box[3 + ax], box[ax]));
    const float v = __fmul_rn(__fsub_rn(x[ax], box[ax]), inv_ext);
    u[ax] = fminf(fmaxf(v, 0.0f), 1.0f);
  }
}

// Cell of level resolution N: c = min(floor(u * N), N - 1), f = u * N - c.
__device__ __forceinline__ void level_cell(float u, int N, int& c, float& f) {
  const float p = __fmul_rn(u, (float)N);
  int ci = (int)floorf(p);
  ci = min(max(ci, 0), N - 1);
  c = ci;
  f = __fsub_rn(p, (float)ci);
}

// Index within level l of vertex (x, y, z).
__device__ __forceinline__ uint32_t vertex_index(const LevelParams& lp, int l, uint32_t x, uint32_t y, uint32_t z) {
  if ((lp.dense_mask >> l) & 1u) {
    const uint32_t side = (uint32_t)lp.N[l] + 1u;
    return x + y * side + z * side * side;
  }
  return (x ^ (y * kHashPrime2) ^ (z * kHashPrime3)) & lp.hash_mask;
}

// Region owning chunk slot `chunk`: the largest k with base[k] <= chunk.
__device__ __forceinline__ int region_of_chunk(const int32_t* base, int K, int chunk) {
  int lo = 0, hi = K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= chunk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Warp scans and reductions.

// Sums and scans over segments of `width` lanes (32, 16 or 8; every lane of
// the warp takes part); `lane` is the index within the segment. With a width
// below 32 the segments are independent, and a chunk's results equal those
// over 32 lanes with zeros after it, bit for bit (the extra steps add zeros).
__device__ __forceinline__ float warp_sum(float v, int width = 32) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if (o < width) v += __shfl_xor_sync(0xFFFFFFFFu, v, o, width);
  return v;
}

__device__ __forceinline__ float warp_inclusive_scan(float v, int lane, int width = 32) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= width) break;
    const float t = __shfl_up_sync(0xFFFFFFFFu, v, o, width);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ float warp_exclusive_from_inclusive(float incl, int lane, int width = 32) {
  const float t = __shfl_up_sync(0xFFFFFFFFu, incl, 1, width);
  return lane == 0 ? 0.0f : t;
}

// Suffix sum (sum over lanes >= lane of the segment).
__device__ __forceinline__ float warp_suffix_scan(float v, int lane, int width = 32) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= width) break;
    const float t = __shfl_down_sync(0xFFFFFFFFu, v, o, width);
    if (lane + o < width) v += t;
  }
  return v;
}

}  // namespace nerfxl
