/*
 * nerfxl.h -- C ABI of the one-GPU NeRF-XL hot path (arXiv 2404.16221).
 *
 * The scene is split into K disjoint axis-aligned regions (Sec. 4.2). Each
 * region owns its own multiresolution hash grid and small MLP (App. A.1).
 * Every ray is (a) cut into per-region segments and sampled without any
 * interval crossing a region face (Sec. 4.2), (b) evaluated through each
 * region's hash grid and MLP, (c) rendered region-locally into per-segment
 * partials (transmittance, colour, opacity, depth, distortion; Eq. 3-8), and
 * (d) composited across regions by an exclusive prefix product in ray order
 * (Algorithm 1, Algorithm 2), which equals single-pass rendering.
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE memory owned by the caller unless a
 *    comment says "host". The library never allocates device memory: scratch
 *    comes from a caller-provided workspace sized by nerfxl_workspace_bytes().
 *  - Calls are asynchronous on the given stream. Arguments are validated on
 *    the host before anything is launched; a bad argument returns
 *    NERFXL_E_INVALID / NERFXL_E_UNSUPPORTED / NERFXL_E_WORKSPACE and launches
 *    nothing. A launch failure returns NERFXL_E_CUDA. Conditions only the
 *    device can see (more segments on a ray than max_segments) set a flag in
 *    the workspace that nerfxl_check() reports.
 *  - No C++ exception crosses this boundary. nerfxl_last_error() returns a
 *    thread-local description of the last non-OK status.
 *  - Rays: rays_o, rays_d are [R][3] float32, d of unit length. A ray that
 *    misses every region renders rgb = 0, depth = 0, opacity = 0, dist = 0
 *    (black background).
 *  - Geometry and hash indices are computed in FP32 with a fixed operation
 *    order (IEEE division, no fused multiply-add), so region assignment,
 *    interval edges and hash indices are reproducible bit for bit.
 */
#ifndef NERFXL_H_
#define NERFXL_H_

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NERFXL_MAX_LEVELS 32
#define NERFXL_MAX_SEGMENTS 32
#define NERFXL_MAX_REGIONS 1024

typedef enum {
  NERFXL_OK = 0,
  NERFXL_E_INVALID = 1,     /* malformed argument */
  NERFXL_E_WORKSPACE = 2,   /* workspace missing or too small */
  NERFXL_E_CUDA = 3,        /* a CUDA call or launch failed */
  NERFXL_E_TIMEOUT = 4,     /* a bounded device wait gave up */
  NERFXL_E_UNSUPPORTED = 5, /* valid but not implemented (sizes, dtypes) */
  NERFXL_E_OVERFLOW = 6     /* a ray crossed more regions than max_segments */
} nerfxl_status;

typedef enum { NERFXL_F32 = 0, NERFXL_F16 = 1, NERFXL_BF16 = 2, NERFXL_E4M3 = 3 } nerfxl_dtype;

/* Field representations (nerfxl_field.arch). */
#define NERFXL_ARCH_FUSED 0 /* one MLP per region: feat -> W -> W -> 4 */
#define NERFXL_ARCH_SPLIT 1 /* per-region density MLP + one shared, view-dependent colour MLP */

/*
 * The partitioned field: K regions, each with a hash grid of L levels of F
 * features and an MLP mlp_in -> W -> W -> 4 (ReLU, no biases; density =
 * exp(o0), colour = sigmoid(o1..o3)).
 *
 * Level l has resolution level_res[l] (N_l cells per axis, (N_l+1)^3
 * vertices). It is stored densely when (N_l+1)^3 <= 2^log2_T (the vertex
 * count rounded up to a multiple of 8 entries), else as 2^log2_T hashed
 * entries with the Instant-NGP spatial hash. E = nerfxl_table_entries() is the
 * sum of the level sizes; a region's table is [E][F], levels back to back.
 *
 * tables: [K][E][F] of table_dtype (F32 or F16).
 * mlp:    [K][P] of mlp_dtype, P = nerfxl_mlp_params(); each block is
 *         W1 [mlp_in][W], W2 [W][W], W3 [W][4], row-major. Features beyond L*F
 *         are zero, so only the first L*F rows of W1 matter.
 * Currently supported: F = 2, mlp_in = 32, W = 64, L*F <= 32; dtypes FP32
 * tables with an FP32 MLP (CUDA cores), or FP32/FP16 tables with a BF16/FP16
 * MLP (tensor cores, FP32 accumulation). Hash features are interpolated in
 * FP32 and rounded to the MLP's 16-bit type.
 */
typedef struct nerfxl_field {
  int32_t K, L, F, log2_T, mlp_in, mlp_width;
  int32_t level_res[NERFXL_MAX_LEVELS]; /* host values, copied into launches */
  const float* boxes;                   /* [K][6]: min xyz, max xyz; disjoint */
  const void* tables;                   /* [K][E][F] of table_dtype */
  const void* mlp;                      /* [K][P] of mlp_dtype */
  int32_t table_dtype, mlp_dtype;       /* nerfxl_dtype */
  const float* mlp_scales;              /* [K][3] dequantisation scales for E4M3, else NULL */
  /*
   * Occupancy grid (optional; NULL = every sample is evaluated). The
   * spatial-skipping structure of the paper's experimental system (Sec. 5.1,
   * the grid of the cited Instant-NGP paper): per region G^3 cells over the
   * region box (G = occ_res), cell (x, y, z) = x + G (y + G z) holding bit
   * c % 32 of word c / 32 of the region's ceil(G^3 / 32) words. A sample whose
   * point lies in a region-coordinate cell min(floor(u G), G - 1) with a clear
   * bit is empty space: it is not evaluated and renders with density 0, so
   * the result equals rendering it with sigma = 0 (no gradient reaches it).
   */
  const uint32_t* occupancy;            /* [K][ceil(G^3/32)], or NULL */
  int32_t occ_res;                      /* G in [1, 1024] when occupancy is set */
  /*
   * Representation. NERFXL_ARCH_FUSED: as above. NERFXL_ARCH_SPLIT, the
   * representation the paper trains (App. A.1, after Instant-NGP): region k's
   * block is a density MLP Wd1 [mlp_in][W], Wd2 [W][16] (ReLU, no biases; its
   * 16 outputs g, density = exp(g0)); one colour MLP shared by all regions
   * follows the K density blocks in the same array: Wc1 [32][W], Wc2 [W][W],
   * Wc3 [W][4] on [g, SH(d)] -> ReLU -> ReLU -> colour = sigmoid of the first
   * three outputs (column 3 of Wc3 is unused). SH(d) is the 16 real spherical
   * harmonics of degrees 0..3 of the ray's unit direction (Condon-Shortley
   * phase; order Y_0^0, Y_1^-1, Y_1^0, Y_1^1, Y_2^-2, ..., Y_3^3). mlp then
   * holds K * (mlp_in W + 16 W) + (32 W + W W + 4 W) values
   * (nerfxl_field_mlp_params). Built: FP32 tables and MLP (forward, backward,
   * training step, grid refresh); FP32/FP16 tables with a BF16/FP16 MLP:
   * forward and backward on the tensor cores (the backward reads the forward's
   * NERFXL_SAVE_FEATURES records and recomputes both MLPs). E4M3:
   * E_UNSUPPORTED.
   */
  int32_t arch;
} nerfxl_field;

/*
 * Sampling (Sec. 4.2): the ray's segments [t0_k, t1_k] are sorted by t0; a
 * uniform grid of n_samples intervals is laid over [first t0, last t1]
 * (edges e_j = tn + j * ((tf - tn) / n_samples)), and each segment is cut at
 * its own ends: segment k owns {t0_k} U {e_j : t0_k < e_j < t1_k} U {t1_k}.
 * A ray therefore has at most n_samples + max_segments - 1 intervals.
 * max_segments bounds the segments of one ray (0 means min(K, 32)).
 */
typedef struct nerfxl_sampling {
  int32_t n_samples;
  int32_t max_segments;
  float t_min;   /* near clamp of every t0 (0 for cameras outside the scene) */
  int32_t flags; /* NERFXL_SAVE_FEATURES | NERFXL_SAMPLE_COMPOSITE, or 0 */
} nerfxl_sampling;

/*
 * Training: the forward keeps per-sample records for the backward in a
 * backward-sized workspace, so that the backward does not gather the tables
 * again. With a 16-bit MLP these are the tensor-core backward's per-tile
 * records (the 16-bit encoded features, sample geometry and the chunk-render
 * values its adjoint reuses: about 116 bytes per sample row); without the flag
 * nerfxl_render_bwd rebuilds them with one more forward pass first. With an
 * FP32 MLP they are the FP32 features (128 bytes per sample row); without the
 * flag the backward encodes again (the split representation's backward then
 * writes the records itself, as it reads the features twice). The flag must
 * be the same on the forward and the backward call.
 */
#define NERFXL_SAVE_FEATURES 1

/*
 * Sample-level composition (the naive scheme of Sec. 4.2 that the paper's
 * segment-level composition replaces): the FP32 forward writes every sample's
 * sigma, rgb, tbar - tn and delta (24 bytes per sample slot) instead of one
 * partial per 32-sample chunk, and the composite renders each ray in a single
 * pass over its samples (Eq. 1-2, 5-6 and the distortion loss directly). Same
 * outputs within FP32 rounding; kept to measure what the segment-level scheme
 * saves (bytes between the field kernel and the composite). FP32 MLP only
 * (E_UNSUPPORTED otherwise); forward only.
 */
#define NERFXL_SAMPLE_COMPOSITE 2

/* Entries per region table (sum of level sizes), or -1 on bad input. */
int64_t nerfxl_table_entries(const int32_t* level_res /* host [L] */, int32_t L, int32_t log2_T);
/* Parameters per region MLP block: mlp_in*W + W*W + 4*W. */
int64_t nerfxl_mlp_params(int32_t mlp_in, int32_t width);
/* Elements of f->mlp for its representation (K * P fused; K density blocks + the colour block split), or -1. */
int64_t nerfxl_field_mlp_params(const nerfxl_field* f);
/* Largest number of 32-sample chunks one ray can produce. */
int32_t nerfxl_max_chunks(const nerfxl_sampling* s, int32_t K);

/*
 * Workspace for R rays. With for_backward != 0 it also holds what
 * nerfxl_render_bwd needs; a forward call on such a workspace keeps the
 * per-chunk partials for the backward call that follows.
 */
size_t nerfxl_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, int32_t for_backward);

/*
 * Forward render (steps a-d above). Outputs: rgb [R][3], depth [R]
 * (unnormalised expected distance, Eq. 6), opacity [R] (accumulated weight,
 * Eq. 5), dist [R] (distortion loss of the ray, Eq. 7; may be NULL).
 */
nerfxl_status nerfxl_render_fwd(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                const float* rays_o, const float* rays_d, float* rgb, float* depth, float* opacity,
                                float* dist, void* workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * Backward (adjoint) render. Given dL/d(output) per ray (any of d_rgb [R][3],
 * d_depth, d_opacity, d_dist [R] may be NULL, meaning zero), ACCUMULATES the
 * gradient into grad_tables [K][E][F] and grad_mlp [K][P] (FP32, caller
 * zeroes them). The workspace must be the one of the immediately preceding
 * nerfxl_render_fwd on the same field and rays, sized with for_backward=1 and
 * unmodified since. Per-sample activations are recomputed, not stored.
 * Gradient accumulation order is unspecified (FP32 atomics), so results vary
 * in the last bits between runs. Loss gradients reach each region's
 * parameters only through that region's own samples (Sec. 4.2).
 */
nerfxl_status nerfxl_render_bwd(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                const float* rays_o, const float* rays_d, const float* d_rgb, const float* d_depth,
                                const float* d_opacity, const float* d_dist, float* grad_tables, float* grad_mlp,
                                void* workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * Loss L = mean_{r,c} (rgb - target)^2 + lambda * mean_r dist (Sec. 4.1:
 * photometric L2 plus the distortion regulariser of Eq. 2). Writes
 * loss_out[3] = {L, photometric term, mean distortion} and, where non-NULL,
 * the output adjoints d_rgb [R][3] and d_dist [R]. scratch holds
 * ceil(R/256) float2 block sums. Deterministic (fixed reduction order).
 */
nerfxl_status nerfxl_loss(int64_t n_rays, const float* rgb, const float* dist, const float* target_rgb,
                          float lambda_dist, float* d_rgb, float* d_dist, float* loss_out, void* scratch,
                          size_t scratch_bytes, cudaStream_t stream);

/* Adam hyper-parameters of one update; step is 1-based. */
typedef struct nerfxl_adam {
  float lr, beta1, beta2, eps;
  int64_t step;
} nerfxl_adam;

/*
 * One Adam step (Kingma & Ba, bias-corrected) over n FP32 parameters, in
 * place. If copy_dtype is NERFXL_F16 or NERFXL_BF16 the updated values are
 * also written, rounded, to compute_copy (the reduced-precision parameters
 * the render kernels read).
 */
nerfxl_status nerfxl_adam_update(int64_t n, float* params, const float* grads, float* m, float* v,
                                 const nerfxl_adam* opt, void* compute_copy, int32_t copy_dtype, cudaStream_t stream);

/*
 * E4M3 weights of fused MLP blocks for the FP8 precision form (the MLP
 * precision sweep; forward only). mlp [K][P] FP32 blocks W1 [mlp_in][width],
 * W2 [width][width], W3 [width][4] (P = nerfxl_mlp_params); per region k and
 * layer li: scales[k][li] = max(max |W|, 1e-30) / 448 (FP32, IEEE division),
 * q = E4M3(W / scale) rounded to nearest even and saturated to +-448, so W ~=
 * scale q. Outputs q [K][P] bytes and scales [K][3] (device), the
 * field's mlp and mlp_scales for mlp_dtype NERFXL_E4M3.
 */
nerfxl_status nerfxl_quantize_e4m3(int32_t K, int32_t mlp_in, int32_t width, const float* mlp, uint8_t* q,
                                   float* scales, cudaStream_t stream);

/* FP32 master parameters, their gradients and Adam moments (all [K][E][F] / [K][P]). */
typedef struct nerfxl_train_state {
  float* tables;
  float* mlp;
  float* grad_tables;
  float* grad_mlp;
  float* m_tables;
  float* v_tables;
  float* m_mlp;
  float* v_mlp;
} nerfxl_train_state;

/*
 * Workspace of nerfxl_step for R rays in one pass. A smaller workspace runs
 * the step in ray sub-batches (below); nerfxl_step_sub_batch returns the
 * sub-batch a workspace of ws_bytes gives: R itself when the one-pass
 * workspace fits, else the largest multiple of 256 rays that fits, 0 if none
 * does (-1 on invalid arguments).
 */
size_t nerfxl_step_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays);
int64_t nerfxl_step_sub_batch(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, size_t ws_bytes);

/*
 * One training step of the partitioned field (Sec. 4.1: the photometric L2
 * loss plus lambda_dist times the distortion loss of Eq. 2, normalised as
 * mean over rays and channels and mean over rays; gradients reach each
 * region's parameters only through its own samples, Sec. 4.2-4.3; then one
 * Adam step, Kingma & Ba, with bias correction): clear the gradients, forward
 * render, loss, backward, Adam on tables and MLP. loss_out[3] as nerfxl_loss
 * (the loss of the parameters before the update). For the FP32 path the field
 * must point at the masters (f->tables == st->tables, f->mlp == st->mlp).
 *
 * Bounded memory: the per-sample state the backward needs grows with the
 * batch (about 116 bytes per sample with a 16-bit MLP). When ws_bytes is below
 * nerfxl_step_workspace_bytes(f, s, n_rays), the rays are processed in
 * sub-batches of nerfxl_step_sub_batch(...) rays: forward, loss adjoints
 * (normalised by all n_rays) and backward per sub-batch, gradients summed,
 * then one Adam step. The result equals the one-pass step up to the order of
 * the FP32 gradient sums; the loss is the same fixed-order sum.
 * E_WORKSPACE if not even 256 rays fit.
 */
nerfxl_status nerfxl_step(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, const float* rays_o,
                          const float* rays_d, const float* target_rgb, float lambda_dist,
                          const nerfxl_train_state* st, const nerfxl_adam* opt, float* loss_out, void* workspace,
                          size_t ws_bytes, cudaStream_t stream);

/* A pinhole camera (row-major pixels, pixel centres, vertical field of view). */
typedef struct nerfxl_camera {
  float origin[3];
  float right[3], up[3], forward[3]; /* orthonormal camera frame */
  float tan_half_fov;                /* tan of half the vertical field of view */
  int32_t width, height;
  int32_t reserved;
} nerfxl_camera;

/* One contiguous range of one camera's pixels inside a rendering batch. */
typedef struct nerfxl_ray_item {
  int64_t batch_offset; /* first ray of the item in the batch (items sorted, contiguous from 0) */
  int64_t first_pixel;  /* row-major index of its first pixel in the camera image */
  int64_t out_offset;   /* output slot of its first pixel */
  int32_t camera;       /* index into cams */
  int32_t count;        /* number of pixels */
} nerfxl_ray_item;

/* Workspace of nerfxl_render_cameras for batches of up to max_rays rays. */
size_t nerfxl_render_cameras_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t max_rays);

/*
 * Render a batch of pixel ranges from many cameras in one pass (the device
 * side of the serving loop; the paper renders novel views of the partitioned
 * field by Algorithm 1 on each pixel's camera ray, Sec. 4.3). items [n_items] and cams [n_cams] are DEVICE arrays; the
 * batch has n_rays = sum of item counts rays, generated on the device from
 * the cameras. Pixel p of item it is written to rgb [(out_offset + p) * 3],
 * depth and opacity [out_offset + p]. A ray's result does not depend on the
 * rest of the batch, so a request renders identically alone or mixed. A ray
 * that falls outside its item, its image or the camera list is skipped (no
 * output written).
 */
nerfxl_status nerfxl_render_cameras(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, int32_t n_items,
                                    const nerfxl_ray_item* items, const nerfxl_camera* cams, int32_t n_cams,
                                    float* rgb, float* depth, float* opacity, void* workspace, size_t ws_bytes,
                                    cudaStream_t stream);

/*
 * Pixel p = i W + j (row i from the top) of a camera generates the ray
 *   aspect = W / H,  x = ((((j + 0.5) / W) * 2 - 1) * tan_half_fov) * aspect,
 *   y = (1 - ((i + 0.5) / H) * 2) * tan_half_fov,
 *   v = (x right + y up) + forward,  d = v / sqrt((v0 v0 + v1 v1) + v2 v2),
 *   o = origin,
 * each operation one IEEE FP32 rounding, no fused multiply-add, evaluated in
 * the order written; the rays are therefore reproducible bit for bit.
 * nerfxl_debug_camera_rays writes the rays nerfxl_render_cameras renders for
 * the same items and cameras (device arrays rays_o, rays_d [n_rays][3]; a ray
 * outside its item, image or camera list gets origin 3e30 and direction +x).
 */
nerfxl_status nerfxl_debug_camera_rays(int64_t n_rays, int32_t n_items, const nerfxl_ray_item* items,
                                       const nerfxl_camera* cams, int32_t n_cams, float* rays_o, float* rays_d,
                                       cudaStream_t stream);

/*
 * Occupancy-grid refresh (keeps the grid of nerfxl_field.occupancy current
 * during training; Sec. 5.1 with the cited Instant-NGP grid). For every cell c
 * = (cx, cy, cz) of every region k, one point is drawn in the cell in region
 * coordinates, u = ((float)c + xi) / G (FP32), with xi_axis = (word_axis >> 8)
 * * 2^-24 from the first three words of Philox4x32-10 (Salmon et al., SC 2011)
 * at counter {c, k, step lo, step hi} and key {seed lo, seed hi}; then
 *   density[k][c] = max(decay * density[k][c], sigma_k(u)),
 *   bit c of bits[k] = density[k][c] > threshold   (unused tail bits 0).
 * Readings where the paper is silent: every cell is refreshed on each call
 * (the caller chooses how often), the threshold is fixed (no mean-density
 * rule), and a grid starts with density 0 and every bit set.
 * The field must have FP32 tables and an FP32 MLP (pass the training
 * masters); its own occupancy pointer is not read. density [K][G^3] float
 * (device, in/out), bits [K][ceil(G^3/32)] uint32 (device, out; may be the
 * grid the field renders with, not while a render on it is in flight).
 * G in [1, 1024] with K * G^3 < 2^31; decay in [0, 1]; E_INVALID otherwise.
 */
nerfxl_status nerfxl_occupancy_update(const nerfxl_field* f, int32_t G, int64_t step, uint64_t seed, float decay,
                                      float threshold, float* density, uint32_t* bits, cudaStream_t stream);

/*
 * Spatial partitioning (Sec. 4.4 "Spatial Partitioning" and its appendix
 * figure): split the root box [6] (min xyz, max xyz) recursively, `levels`
 * times, at the plane where the CDF of the points inside the box along one
 * axis is 0.5, choosing the axis whose two halves are closest to cubic; the
 * result is 2^levels disjoint boxes with balanced point counts, written to
 * boxes [2^levels][6] in depth-first order (lower half first), and the number
 * of points in each to counts [2^levels] (may be NULL). points [n_points][3]
 * is the scene content: an SfM point cloud, or samples of training rays when
 * there is none. Readings where the paper is silent: the CDF = 0.5 plane of
 * m points is their median 0.5 (s[(m-1)/2] + s[m/2]) along the axis (FP32); a
 * point goes below the plane if its coordinate < plane; a plane that is not
 * strictly inside the box falls back to the midplane; aspect ratio = longest
 * side / shortest side, a split scored by the worse of its two boxes, ties to
 * the lowest axis; points outside the root are ignored. HOST pointers; runs
 * on the CPU (once per scene). levels in 0..10; E_INVALID on bad arguments.
 */
nerfxl_status nerfxl_partition(const float* points, int64_t n_points, const float* root, int32_t levels, float* boxes,
                               int64_t* counts);

/*
 * Per-region chunk counts of the last sampling in a workspace (a chunk is up
 * to 32 samples of one ray segment): copies K int32 to the HOST array counts
 * (synchronises the stream). The measure of how evenly a partition spreads
 * the samples over the regions. The paper has no counterpart.
 */
nerfxl_status nerfxl_region_chunks(const void* workspace, size_t ws_bytes, int32_t K, int32_t* counts,
                                   cudaStream_t stream);

/*
 * Forward render without a caller workspace (the paper has no counterpart:
 * this serves callers that cannot allocate device memory, such as plain C
 * programs or plug-ins without an allocator, hosts that own the whole device
 * memory pool, or frame loops where cudaMalloc would stall). Same inputs,
 * outputs and results as nerfxl_render_fwd; the scratch comes from a fixed
 * 32 MiB array in the library's device image, reserved on every GPU that
 * loads the library until exit. Batches needing more scratch are refused
 * with NERFXL_E_WORKSPACE (grid8-sized rays: roughly 60 thousand per call).
 * Each call looks up the array's address on the current device (no caching,
 * so a cudaDeviceReset leaves nothing stale); the first call on a device also
 * loads the library's device code there, so make it before any stream
 * capture. Calls share the array: calls that overlap on the GPU race, so
 * order them on one stream. Allocates nothing.
 */
nerfxl_status nerfxl_render_fwd_static(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                       const float* rays_o, const float* rays_d, float* rgb, float* depth,
                                       float* opacity, float* dist, cudaStream_t stream);

/*
 * Device-side status of the last nerfxl_render_fwd_static call on the current
 * device (synchronises the stream), as nerfxl_check reports it for a caller
 * workspace: NERFXL_OK, NERFXL_E_OVERFLOW (a ray crossed more regions than
 * max_segments; its segments beyond that were dropped) or NERFXL_E_TIMEOUT
 * (the tensor-core forward gave up a bounded wait; that call's outputs are
 * invalid). Allocates nothing.
 */
nerfxl_status nerfxl_static_check(cudaStream_t stream);

/*
 * Status of device-side checks of the last call made with this workspace
 * (synchronises the stream): NERFXL_OK, NERFXL_E_OVERFLOW, or NERFXL_E_TIMEOUT (a
 * bounded wait of the tensor-core pipeline expired; the kernel stopped early
 * and released its tensor memory, the outputs of that call are invalid).
 */
nerfxl_status nerfxl_check(const void* workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * Counters of the last call made with this workspace (synchronises the
 * stream): samples evaluated (all intervals, or those in occupied cells when
 * the field has an occupancy grid) and non-empty 32-sample chunks.
 */
nerfxl_status nerfxl_workspace_stats(const void* workspace, size_t ws_bytes, int64_t* n_samples, int64_t* n_chunks,
                                     cudaStream_t stream);

/*
 * Instrumentation: while set (non-NULL), every following call records
 * `start` right before and `stop` right after its dominant kernel (the fused
 * field kernel of the forward or backward pass), on the call's stream, so a
 * caller can time that kernel with CUDA events. Pass NULL, NULL to stop.
 * Process-wide setting; not for concurrent use from several threads.
 */
nerfxl_status nerfxl_set_profile_events(cudaEvent_t start, cudaEvent_t stop);

/*
 * Level-grouped gather of the tensor-core forward (BF16/FP16 MLP). The
 * forward sweeps the regions one at a time, so one region's table is the
 * working set of its random gathers; beyond some 30-40 MB (measured on B300)
 * the L2 stops holding it and the gather reads the table many times from HBM.
 * A batch whose field has a region table above min_table_bytes, and which
 * brings at least min_region_samples samples per region (n_rays x n_samples /
 * K; each group is one more pass over the samples, which pays only when a
 * region's samples reuse its table lines: a city training sub-batch of 62 K
 * rays ran slower grouped), is therefore gathered
 * one group of levels (at most group_bytes of table, at least one level) at a
 * time over all of a region's samples, into level-major feature words (4
 * bytes per level per sample row), which the MLP and render then read
 * (results bit for bit those of the one-pass gather). Workspaces of such
 * fields hold a window of window_tiles tiles of 128 rows (L x 512 bytes
 * each). Process-wide; pass 0 for a default (64 MiB, 64 MiB, 65536
 * tiles, 2^21 samples: on the street/city field, 2 groups of a 96 MB FP16 region table ran
 * faster than 3 to 11 smaller ones, whose extra passes cost more than their
 * fewer L2 misses save); set it before sizing workspaces. The paper has no
 * counterpart (its GPUs each hold one region).
 */
nerfxl_status nerfxl_set_gather_groups(size_t min_table_bytes, size_t group_bytes, int64_t window_tiles,
                                       int64_t min_region_samples);

/*
 * Instrumentation: the number of kernels this library has launched in this
 * process (all entry points, all devices and streams), for counting the
 * launches of a timed region. The paper has no counterpart.
 */
int64_t nerfxl_launch_count(void);

/*
 * Failure-path probe: one thread waits on an mbarrier with the same bounded
 * poll loop the tensor-core kernels use (at most `spins` polls; <= 2^26).
 * With arrive != 0 the barrier completes and the call returns NERFXL_OK;
 * with arrive == 0 nothing ever arrives, the wait gives up, and the call
 * returns NERFXL_E_TIMEOUT with the context still usable. status is one
 * device int32 (1 = completed, 0 = timed out). Synchronises the stream.
 */
nerfxl_status nerfxl_debug_wait_probe(int32_t* status, uint32_t spins, int32_t arrive, cudaStream_t stream);

/*
 * Reduction-rate probe: the measured ceiling of the backward kernels' table
 * scatter. Launches (asynchronously on `stream`) 4 CTAs of 256 threads per
 * SM; each thread issues `iters` 16-byte FP32 vector reductions
 * (red.global.add.v4.f32, evict-last L2 hint, as the scatter issues them)
 * adding 1.0 to float4 slots of `buf` chosen by a mixing hash, all inside
 * [buf, buf + bytes). `buf`: caller-owned device memory, 16-byte aligned,
 * contents overwritten; bytes / 16 < 2^32. *ops (host) receives the number
 * of reductions launched; the caller times the launch with its own events.
 * E_INVALID on bad arguments. The paper has no counterpart (measurement).
 */
nerfxl_status nerfxl_probe_reduction_rate(void* buf, size_t bytes, int32_t iters, int64_t* ops, cudaStream_t stream);

/*
 * Load-rate probe: the measured ceiling of the forward's table gather.
 * Launches (asynchronously on `stream`) 4 CTAs of 256 threads per SM; each
 * thread issues `iters` x 16 independent 8-byte loads from slots of `buf`
 * chosen by a mixing hash, all inside [buf, buf + bytes). `buf`: caller-owned
 * device memory, 8-byte aligned, only read; bytes / 8 < 2^32. *ops (host)
 * receives the number of loads launched; the caller times the launch with its
 * own events. E_INVALID on bad arguments. The paper has no counterpart
 * (measurement).
 */
nerfxl_status nerfxl_probe_load_rate(const void* buf, size_t bytes, int32_t iters, int64_t* ops, cudaStream_t stream);

/* Thread-local text for the last non-OK status. */
const char* nerfxl_last_error(void);

/*
 * Debug views of the forward pass, computed by the same device functions as
 * nerfxl_render_fwd, for bit-exact checks.
 *
 * nerfxl_debug_segments: nseg [R]; region, t0, t1, n_intervals [R][max_seg].
 * nerfxl_debug_samples: per ray count [R]; per interval a, b [R][max_int]
 *   (float32) and region [R][max_int]; optionally hash indices within the
 *   level idx [R][max_int][L][8] (uint32, may be NULL), features
 *   feat [R][max_int][mlp_in] (float32, may be NULL) and raw MLP outputs
 *   raw [R][max_int][4] (float32, may be NULL). Slots past count are untouched.
 */
nerfxl_status nerfxl_debug_segments(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                    const float* rays_o, const float* rays_d, int32_t max_seg, int32_t* nseg,
                                    int32_t* region, float* t0, float* t1, int32_t* n_intervals, void* workspace,
                                    size_t ws_bytes, cudaStream_t stream);
nerfxl_status nerfxl_debug_samples(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                   const float* rays_o, const float* rays_d, int32_t max_int, int32_t* count,
                                   float* a, float* b, int32_t* region, uint32_t* idx, float* feat, float* raw,
                                   cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* NERFXL_H_ */
