// Debug views of the forward pass: the same device functions as the fused
// kernels, written out per ray / per interval for bit-exact checks of region
// assignment, interval edges and hash indices.

#include <cuda_runtime.h>

#include "nerfxl_field.cuh"
#include "nerfxl_host.h"

namespace nerfxl {

__global__ void k_debug_seg_out(int64_t R, int max_seg_ws, int max_seg_out, const RayHdr* __restrict__ hdr,
                                const SegDesc* __restrict__ segs, int32_t* nseg, int32_t* region, float* t0, float* t1,
                                int32_t* nint) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const RayHdr h = hdr[r];
  nseg[r] = h.nseg;
  for (int k = 0; k < h.nseg && k < max_seg_out; ++k) {
    const SegDesc s = segs[r * max_seg_ws + k];
    region[r * max_seg_out + k] = seg_region(s);
    t0[r * max_seg_out + k] = s.t0;
    t1[r * max_seg_out + k] = s.t1;
    nint[r * max_seg_out + k] = seg_n(s);
  }
}

// One thread per ray: segments, intervals, and per interval optionally the
// level indices, the encoded features and the raw MLP outputs.
__global__ void k_debug_samples(int64_t R, const float* __restrict__ rays_o, const float* __restrict__ rays_d,
                                FieldPtrs fp, int K, LevelParams lp, SampParams sp, int max_int, int32_t* count,
                                float* a_out, float* b_out, int32_t* reg_out, uint32_t* idx_out, float* feat_out,
                                float* raw_out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  float o[3], d[3];
  for (int ax = 0; ax < 3; ++ax) {
    o[ax] = rays_o[3 * r + ax];
    d[ax] = rays_d[3 * r + ax];
  }
  float st0[kMaxSeg], st1[kMaxSeg];
  int sreg[kMaxSeg];
  const int hits = ray_segments(o, d, fp.boxes, K, sp.t_min, sp.max_seg, st0, st1, sreg);
  const int nseg = min(hits, sp.max_seg);
  const float tn = nseg ? st0[0] : 0.0f;
  const float delta = nseg ? __fdiv_rn(__fsub_rn(st1[nseg - 1], st0[0]), (float)sp.S) : 0.0f;
  int out = 0;
  for (int k = 0; k < nseg; ++k) {
    const int jlo = first_edge_above(tn, delta, sp.S, st0[k]);
    const int jend = first_edge_at_or_above(tn, delta, sp.S, st1[k]);
    const int n = 1 + max(0, jend - jlo);
    SegDesc sd;
    sd.t0 = st0[k];
    sd.t1 = st1[k];
    sd.jlo_n = (jlo & 0xFFFF) | (n << 16);
    sd.reg_cb = sreg[k];
    for (int i = 0; i < n; ++i, ++out) {
      if (out >= max_int) continue;
      float a, b;
      segment_interval(sd, tn, delta, i, a, b);
      const size_t slot = (size_t)r * max_int + out;
      a_out[slot] = a;
      b_out[slot] = b;
      reg_out[slot] = sreg[k];
      if (!idx_out && !feat_out && !raw_out) continue;
      const float tbar = __fmul_rn(0.5f, __fadd_rn(a, b));
      float x[3], u[3];
      sample_point(o, d, tbar, x);
      region_coord(fp.boxes + 6 * sreg[k], x, u);
      if (idx_out) {
        for (int l = 0; l < lp.L; ++l) {
          int c[3];
          float f[3];
          for (int ax = 0; ax < 3; ++ax) level_cell(u[ax], lp.N[l], c[ax], f[ax]);
          for (int e = 0; e < 8; ++e)
            idx_out[(slot * lp.L + l) * 8 + e] =
                vertex_index(lp, l, c[0] + (e & 1), c[1] + ((e >> 1) & 1), c[2] + ((e >> 2) & 1));
        }
      }
      if (feat_out || raw_out) {
        float feat[kIn];
        encode_f32(lp, reinterpret_cast<const float2*>(fp.tables) + (size_t)sreg[k] * lp.E, u, feat);
        if (feat_out)
          for (int q = 0; q < kIn; ++q) feat_out[slot * kIn + q] = feat[q];
        if (raw_out) {
          float raw[kOut];
          mlp_f32_global(fp.mlp + (size_t)sreg[k] * kMlpParams, feat, raw);
          for (int q = 0; q < kOut; ++q) raw_out[slot * kOut + q] = raw[q];
        }
      }
    }
  }
  count[r] = out;
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" {

nerfxl_status nerfxl_debug_segments(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                    const float* rays_o, const float* rays_d, int32_t max_seg, int32_t* nseg,
                                    int32_t* region, float* t0, float* t1, int32_t* n_intervals, void* workspace,
                                    size_t ws_bytes, cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  const Layout L = layout(f, s, n_rays, 0);
  if (!workspace || ws_bytes < L.total) return set_error(NERFXL_E_WORKSPACE, "workspace too small");
  if (max_seg < 1) return set_error(NERFXL_E_INVALID, "max_seg < 1");
  char* ws = static_cast<char*>(workspace);
  const SampParams sp = samp_params(f, s, ws, L);
  st = run_sampling(f, sp, n_rays, rays_o, rays_d, ws, L, stream);
  if (st != NERFXL_OK || n_rays == 0) return st;
  k_debug_seg_out<<<(int)((n_rays + 127) / 128), 128, 0, stream>>>(
      n_rays, L.max_seg, max_seg, reinterpret_cast<const RayHdr*>(ws + L.ray_hdr),
      reinterpret_cast<const SegDesc*>(ws + L.segs), nseg, region, t0, t1, n_intervals);
  return kernel_launched("k_debug_seg_out");
}

nerfxl_status nerfxl_debug_samples(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                   const float* rays_o, const float* rays_d, int32_t max_int, int32_t* count,
                                   float* a, float* b, int32_t* region, uint32_t* idx, float* feat, float* raw,
                                   cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  if (f->table_dtype != NERFXL_F32 || f->mlp_dtype != NERFXL_F32)
    return set_error(NERFXL_E_UNSUPPORTED, "debug views read FP32 parameters");
  if (raw && f->arch != NERFXL_ARCH_FUSED)
    return set_error(NERFXL_E_UNSUPPORTED, "raw MLP outputs are built for the fused representation");
  if (max_int < 1 || !count || !a || !b || !region) return set_error(NERFXL_E_INVALID, "bad debug outputs");
  if (n_rays == 0) return NERFXL_OK;
  FieldPtrs fp;
  fp.boxes = f->boxes;
  fp.tables = static_cast<const float*>(f->tables);
  fp.mlp = static_cast<const float*>(f->mlp);
  k_debug_samples<<<(int)((n_rays + 63) / 64), 64, 0, stream>>>(n_rays, rays_o, rays_d, fp, f->K, level_params(f),
                                                                samp_params(f, s), max_int, count, a, b, region, idx,
                                                                feat, raw);
  return kernel_launched("k_debug_samples");
}

}  // extern "C"
