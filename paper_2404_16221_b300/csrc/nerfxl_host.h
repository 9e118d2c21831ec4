// Host-side helpers shared by the translation units of libnerfxl.
#pragma once

#include <stdint.h>

#include <string>

#include "nerfxl_device.cuh"

namespace nerfxl {

// Byte offsets of the workspace regions (each 256-byte aligned).
struct Layout {
  size_t hdr;        // int32[16]: [0] error flags, [1] tile count, [2..5] int64 samples, chunks
  size_t counts;     // int32[K] chunks per region
  size_t cursor;     // int32[K] fill cursors
  size_t zero_end;   // [0, zero_end) is cleared at the start of each call
  size_t base;       // int32[K+1] first chunk slot of each region bucket
  size_t ray_hdr;    // RayHdr[R]
  size_t segs;       // SegDesc[R][max_seg]
  // Occupancy skipping (fields with an occupancy grid; 0 otherwise):
  size_t seg_keep;   // int32[R][max_seg]: kept samples | first list slot << 16
  size_t kept;       // uint16[R][max_int]: kept interval indices within their segment
  size_t chunks;     // Slot[chunk_cap]: chunk slots (one, two or four chunks each; see slot_lane)
  size_t partials;   // float4[R][max_chunk][2]
  size_t dpartials;  // float4[R][max_chunk][2] (backward workspaces only)
  // Per-tile records of the tensor-core backward (backward workspaces with a
  // 16-bit MLP only; 0 otherwise). A tile is 4 chunks = 128 sample rows.
  size_t rec_feat;   // [tiles][128 rows][64 B]: 16-bit features, 64-byte-swizzled MMA tile
  size_t rec_geom;   // float[tiles][kGeomFloats]: per row u0 u1 u2 tr dl, then Tn w pair sigma rgb
                     // (fused) or the ray direction d0 d1 d2 (split); chunk counts
  size_t rec_dpart;  // float4[tiles * 16][2]: chunk adjoints in tile order (4 positions per slot)
  size_t rec_pos;    // int32[R][max_chunk]: tile-order position of each chunk
  // FP32 records (backward workspaces of the fused FP32 MLP): the forward's
  // features per 256-row tile, unit-major [tiles][32][256] float.
  size_t rec32;
  // Sample-level composition (NERFXL_SAMPLE_COMPOSITE; 0 otherwise):
  size_t smp4;       // float4[R][max_chunk][32]: sigma, r, g, b per sample slot
  size_t smp2;       // float2[R][max_chunk][32]: tbar - tn, delta per sample slot
  // Level-grouped gather (fields whose region table exceeds kGroupMinBytes):
  // a window of gfeat_tiles tiles of level-major feature words,
  // [L][gfeat_tiles][128] uint32 (two 16-bit features per word), followed by
  // the rows' region coordinates and sample flags, [4][gfeat_tiles][128]
  // (u0, u1, u2 as float bits, then 1 for a sample, 0 for an empty row).
  size_t gfeat;
  int64_t gfeat_tiles;
  size_t total;
  int64_t rec_tiles; // tiles the record regions hold
  int64_t chunk_cap;
  int max_seg, max_chunk, max_int;
};

const char* last_error();
nerfxl_status set_error(nerfxl_status st, const std::string& msg);
nerfxl_status launch_check(const char* what);
// launch_check after a kernel launch, counting the launch (nerfxl_launch_count).
nerfxl_status kernel_launched(const char* name);
nerfxl_status validate(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R);
int effective_max_seg(const nerfxl_field* f, const nerfxl_sampling* s);
int max_chunks(int S, int max_seg);
Layout layout(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R, int for_backward);
LevelParams level_params(const nerfxl_field* f);
// Sampling parameters; the second form also points the kernels at the
// workspace's occupancy lists when the field has an occupancy grid.
SampParams samp_params(const nerfxl_field* f, const nerfxl_sampling* s);
SampParams samp_params(const nerfxl_field* f, const nerfxl_sampling* s, char* ws, const Layout& L);
nerfxl_status run_sampling(const nerfxl_field* f, const SampParams& sp, int64_t R, const float* rays_o,
                           const float* rays_d, char* ws, const Layout& L, cudaStream_t stream);
// Records the instrumentation event `which` (0 = before, 1 = after the
// dominant kernel) if the caller installed one.
void profile_mark(int which, cudaStream_t stream);
int fwd_grid(int64_t max_tiles, int ctas_per_sm);
// SMs of the current device (cached on first use).
int num_sms();
// Forward render; out_index (device [R], may be NULL) gives each ray's output slot.
nerfxl_status render_fwd_impl(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, const float* rays_o,
                              const float* rays_d, float* rgb, float* depth, float* opacity, float* dist,
                              const int64_t* out_index, void* workspace, size_t ws_bytes, cudaStream_t stream);
// Records of one 128-row tile for the tensor-core backward.
//   features  row r's 32 16-bit features as the K-major A operand of the first
//             MMA in the 64-byte swizzle: 16-byte chunk c of row r at byte
//             64 r + 16 (c ^ ((r / 2) % 4)).
//   geometry  128 floats each of u0, u1, u2 (region coordinates), tr (tbar - tn),
//             dl (interval length), Tn (transmittance after the sample within its
//             chunk), w (chunk-local weight), pair (sum over the chunk of
//             w_j |tr_i - tr_j|), sigma, r, g, b (the MLP outputs after exp /
//             sigmoid); then per slot (int32) the sample counts of its chunks and
//             its width (slot_count_word). The
//             split representation's backward recomputes its two MLPs and the
//             render quantities; its rows 5..7 hold the ray direction instead
//             (the colour MLP's SH input) and rows 8..11 are unused.
constexpr int kRecRows = 128;
constexpr int kGeomRowFields = 12;
constexpr int kGeomFloats = kGeomRowFields * kRecRows + 4;  // 6160 bytes, a multiple of 16
constexpr size_t kRecFeatBytes = (size_t)kRecRows * 64;     // 8192 bytes per tile

// Where the tensor-core forward writes the backward's records (all NULL for a
// plain forward).
struct RecordOut {
  uint4* feat;
  float* geom;
  int32_t* pos;
  uint32_t* gfeat;  // the backward layout's level-grouped gather window (or NULL)
  int64_t gfeat_tiles;
};
RecordOut record_out(char* ws, const Layout& L);

// Level-grouped gather of the tensor-core forward. A region table of more than
// kGroupMinBytes is gathered one group of levels at a time (groups of at most
// kGroupBytes, at least one level), over windows of at most
// kGatherWindowTiles 4-chunk tiles, into feature tiles the forward then reads.
constexpr size_t kGroupMinBytes = size_t(64) << 20;
constexpr size_t kGroupBytes = size_t(64) << 20;
constexpr int64_t kGatherWindowTiles = 65536;
constexpr int kGatherCoordWords = 4;  // per row after the feature words: u0, u1, u2, sample flag
// The values in force (nerfxl_set_gather_groups may change them).
size_t group_min_bytes();
int64_t gather_window_tiles();
// A batch of R rays gathers by groups when the region table exceeds the
// size threshold and the batch brings at least kGroupMinRegionSamples samples
// per region (R * n_samples / K): each group is one more pass over the
// samples, which only pays when a region's samples reuse its table lines.
constexpr int64_t kGroupMinRegionSamples = int64_t(1) << 21;
bool grouped_gather(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R);
int gather_groups(const nerfxl_field* f, const LevelParams& lp, int32_t* g_lo);
nerfxl_status launch_gather_groups(const nerfxl_field* f, const SampParams& sp, const LevelParams& lp,
                                   const float* rays_o, const float* rays_d, char* ws, const Layout& L, uint32_t* feat,
                                   int64_t window, int64_t w0, int64_t w1, cudaStream_t stream);

// Tensor-core field backward (16-bit MLP), from the per-tile records.
nerfxl_status launch_field_bwd_tc(const nerfxl_field* f, const LevelParams& lp, char* ws, const Layout& L,
                                  float* grad_tables, float* grad_mlp, cudaStream_t stream);
// Tensor-core backward of the split representation (BF16/FP16 MLPs; FP32 or
// FP16 tables), recomputing the field from the tables; dpart = chunk adjoints.
nerfxl_status launch_field_bwd_split_tc(const nerfxl_field* f, const LevelParams& lp, char* ws, const Layout& L,
                                        float* grad_tables, float* grad_mlp, cudaStream_t stream);
// Tensor-core field forward (BF16/FP16 MLP; FP32 or FP16 tables).
nerfxl_status launch_field_fwd_tc(const nerfxl_field* f, const SampParams& sp, const LevelParams& lp,
                                  const float* rays_o, const float* rays_d, char* ws, const Layout& L,
                                  const RecordOut& rec, cudaStream_t stream);

}  // namespace nerfxl
