// Batched rendering of pixel ranges from many cameras in one pass: the
// device side of the serving loop. A batch is a list of work items, each a
// contiguous range of one request's pixels; rays are generated on the device
// from the request's pinhole camera, the batch runs through the same
// persistent pipeline as nerfxl_render_fwd, and the composite writes each
// ray's result straight into its request's image. A ray's result depends only
// on the ray (its chunks are reduced independently and composited per ray),
// so a request renders identically alone or mixed with others.

#include <cuda_runtime.h>

#include <string>

#include "nerfxl_device.cuh"
#include "nerfxl_host.h"

namespace nerfxl {

// Pixel p = i W + j (row i from the top, column j) of camera c, in a
// prescribed FP32 operation sequence with one IEEE rounding per operation and
// no fused multiply-add, so that any implementation of the same sequence gives
// the same rays bit for bit:
//   aspect = W / H
//   x = ((((j + 0.5) / W) * 2 - 1) * tan) * aspect
//   y = (1 - ((i + 0.5) / H) * 2) * tan
//   v_a = (x right_a + y up_a) + forward_a
//   n = sqrt((v_0 v_0 + v_1 v_1) + v_2 v_2),   d_a = v_a / n,   o = origin.
// A ray outside its item, its camera's image, or the camera list is rendered
// as a miss and gets output slot -1 (the composite skips it).
__global__ void __launch_bounds__(256) k_gen_rays(int64_t R, int n_items, const nerfxl_ray_item* __restrict__ items,
                                                  const nerfxl_camera* __restrict__ cams, int n_cams,
                                                  float* __restrict__ rays_o, float* __restrict__ rays_d,
                                                  int64_t* __restrict__ out_index) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int lo = 0, hi = n_items - 1;  // last item with batch_offset <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].batch_offset <= r) lo = mid;
    else hi = mid - 1;
  }
  const nerfxl_ray_item it = items[lo];
  const int64_t local = r - it.batch_offset;
  const bool item_ok = it.camera >= 0 && it.camera < n_cams && local >= 0 && local < it.count;
  const nerfxl_camera cam = cams[item_ok ? it.camera : 0];
  const int64_t pix = it.first_pixel + local;
  if (!item_ok || cam.width < 1 || cam.height < 1 || pix < 0 || pix >= (int64_t)cam.width * cam.height) {
    const float miss_o[3] = {3.0e30f, 3.0e30f, 3.0e30f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rays_o[3 * r + a] = miss_o[a];
      rays_d[3 * r + a] = a == 0 ? 1.0f : 0.0f;
    }
    if (out_index) out_index[r] = -1;
    return;
  }
  const int i = (int)(pix / cam.width), j = (int)(pix % cam.width);
  const float Wf = (float)cam.width, Hf = (float)cam.height, tanh_ = cam.tan_half_fov;
  const float aspect = __fdiv_rn(Wf, Hf);
  const float x =
      __fmul_rn(__fmul_rn(__fsub_rn(__fmul_rn(__fdiv_rn(__fadd_rn((float)j, 0.5f), Wf), 2.0f), 1.0f), tanh_), aspect);
  const float y = __fmul_rn(__fsub_rn(1.0f, __fmul_rn(__fdiv_rn(__fadd_rn((float)i, 0.5f), Hf), 2.0f)), tanh_);
  float v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    v[a] = __fadd_rn(__fadd_rn(__fmul_rn(x, cam.right[a]), __fmul_rn(y, cam.up[a])), cam.forward[a]);
  const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rays_o[3 * r + a] = cam.origin[a];
    rays_d[3 * r + a] = __fdiv_rn(v[a], n);
  }
  if (out_index) out_index[r] = it.out_offset + local;
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" {

size_t nerfxl_render_cameras_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t max_rays) {
  if (validate(f, s, max_rays) != NERFXL_OK) return 0;
  const size_t rays = ((size_t)max_rays * (6 * sizeof(float) + sizeof(int64_t)) + 255) / 256 * 256;
  return layout(f, s, max_rays, 0).total + rays + 256;
}

nerfxl_status nerfxl_render_cameras(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, int32_t n_items,
                                    const nerfxl_ray_item* items, const nerfxl_camera* cams, int32_t n_cams, float* rgb,
                                    float* depth, float* opacity, void* workspace, size_t ws_bytes,
                                    cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  if (n_rays > 0 && (n_items < 1 || n_cams < 1 || !items || !cams || !rgb || !depth || !opacity))
    return set_error(NERFXL_E_INVALID, "bad camera batch arguments");
  const size_t need = nerfxl_render_cameras_workspace_bytes(f, s, n_rays);
  if (!workspace || ws_bytes < need) return set_error(NERFXL_E_WORKSPACE, "camera batch workspace too small");
  if (n_rays == 0) return NERFXL_OK;
  const Layout L = layout(f, s, n_rays, 0);
  char* ws = static_cast<char*>(workspace);
  char* extra = ws + (L.total + 255) / 256 * 256;
  float* rays_o = reinterpret_cast<float*>(extra);
  float* rays_d = rays_o + 3 * (size_t)n_rays;
  // 6R floats = 24R bytes, so the index array that follows stays 8-byte aligned
  int64_t* out_index = reinterpret_cast<int64_t*>(rays_d + 3 * (size_t)n_rays);
  k_gen_rays<<<(int)((n_rays + 255) / 256), 256, 0, stream>>>(n_rays, n_items, items, cams, n_cams, rays_o, rays_d,
                                                              out_index);
  st = kernel_launched("k_gen_rays");
  if (st != NERFXL_OK) return st;
  return render_fwd_impl(f, s, n_rays, rays_o, rays_d, rgb, depth, opacity, nullptr, out_index, workspace, L.total,
                         stream);
}

nerfxl_status nerfxl_debug_camera_rays(int64_t n_rays, int32_t n_items, const nerfxl_ray_item* items,
                                       const nerfxl_camera* cams, int32_t n_cams, float* rays_o, float* rays_d,
                                       cudaStream_t stream) {
  if (n_rays < 0 || (n_rays > 0 && (n_items < 1 || n_cams < 1 || !items || !cams || !rays_o || !rays_d)))
    return set_error(NERFXL_E_INVALID, "bad camera ray arguments");
  if (n_rays == 0) return NERFXL_OK;
  k_gen_rays<<<(int)((n_rays + 255) / 256), 256, 0, stream>>>(n_rays, n_items, items, cams, n_cams, rays_o, rays_d,
                                                              nullptr);
  return kernel_launched("k_gen_rays");
}

}  // extern "C"
