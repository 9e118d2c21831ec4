// Loss, optimiser and the fused training step of the one-GPU NeRF-XL path.
//
// Loss (photometric L2 plus the distortion regulariser of Sec. 4.1, Eq. 2):
//   L = mean_{r,c} (C_rc - C*_rc)^2 + lambda * mean_r L_dist,r
// Its output adjoints are dL/dC = 2 (C - C*) / (3R), dL/dL_dist = lambda / R.
// Adam (Kingma & Ba) with bias correction updates the FP32 master parameters.

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "nerfxl_host.h"

namespace nerfxl {

constexpr int kLossThreads = 256;

// Kahan-compensated block sums of the two loss terms; per-ray adjoints.
__global__ void __launch_bounds__(kLossThreads) k_loss(int64_t R, const float* __restrict__ rgb,
                                                       const float* __restrict__ dist,
                                                       const float* __restrict__ target, float lambda,
                                                       float* __restrict__ d_rgb, float* __restrict__ d_dist,
                                                       float2* __restrict__ block_sums) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float photo = 0.0f, dd = 0.0f;
  if (r < R) {
    const float inv = 1.0f / (3.0f * (float)R);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float e = rgb[3 * r + c] - target[3 * r + c];
      photo += e * e;
      if (d_rgb) d_rgb[3 * r + c] = 2.0f * e * inv;
    }
    dd = dist ? dist[r] : 0.0f;
    if (d_dist) d_dist[r] = lambda / (float)R;
  }
  // fixed-order tree reduction within the block
  __shared__ float s_p[kLossThreads], s_d[kLossThreads];
  s_p[threadIdx.x] = photo;
  s_d[threadIdx.x] = dd;
  __syncthreads();
  for (int o = kLossThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_p[threadIdx.x] += s_p[threadIdx.x + o];
      s_d[threadIdx.x] += s_d[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = make_float2(s_p[0], s_d[0]);
}

// Sums the block partials in a fixed order (Kahan) -> loss_out = {total, photo, dist}.
// Final reduction of the per-block sums: FP64 partial sums per thread, then a
// fixed-order tree in shared memory (deterministic, error far below FP32).
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) k_loss_final(const float2* __restrict__ block_sums, int nb, int64_t R,
                                                              float lambda, float* __restrict__ loss_out) {
  __shared__ double s_p[kFinalThreads], s_d[kFinalThreads];
  double sp = 0.0, sd = 0.0;
  for (int b = threadIdx.x; b < nb; b += kFinalThreads) {
    const float2 v = block_sums[b];
    sp += (double)v.x;
    sd += (double)v.y;
  }
  s_p[threadIdx.x] = sp;
  s_d[threadIdx.x] = sd;
  __syncthreads();
  for (int o = kFinalThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_p[threadIdx.x] += s_p[threadIdx.x + o];
      s_d[threadIdx.x] += s_d[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const float photo = R > 0 ? (float)(s_p[0] / (3.0 * (double)R)) : 0.0f;
  const float dmean = R > 0 ? (float)(s_d[0] / (double)R) : 0.0f;
  loss_out[0] = photo + lambda * dmean;
  loss_out[1] = photo;
  loss_out[2] = dmean;
}

// One Adam step over n FP32 parameters; optionally refreshes a reduced-
// precision compute copy (dtype 1 = fp16, 2 = bf16).
__global__ void __launch_bounds__(256) k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                              float b2, float eps, float inv_c1, float inv_sqrt_c2,
                                              void* __restrict__ copy, int copy_dtype) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    // lr * mhat / (sqrt(vhat) + eps), mhat = m / c1, vhat = v / c2
    const float pi = p[i] - lr * (mi * inv_c1) / (sqrtf(vi) * inv_sqrt_c2 + eps);
    p[i] = pi;
    if (copy_dtype == 1) reinterpret_cast<__half*>(copy)[i] = __float2half_rn(pi);
    else if (copy_dtype == 2) reinterpret_cast<__nv_bfloat16*>(copy)[i] = __float2bfloat16_rn(pi);
  }
}

nerfxl_status launch_adam(int64_t n, float* p, const float* g, float* m, float* v, const nerfxl_adam* opt,
                          void* copy, int copy_dtype, cudaStream_t stream) {
  if (n <= 0) return NERFXL_OK;
  const double c1 = 1.0 - std::pow((double)opt->beta1, (double)opt->step);
  const double c2 = 1.0 - std::pow((double)opt->beta2, (double)opt->step);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_adam<<<blocks, 256, 0, stream>>>(n, p, g, m, v, opt->lr, opt->beta1, opt->beta2, opt->eps, (float)(1.0 / c1),
                                     (float)(1.0 / std::sqrt(c2)), copy, copy_dtype);
  return kernel_launched("k_adam");
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" {

nerfxl_status nerfxl_loss(int64_t n_rays, const float* rgb, const float* dist, const float* target_rgb,
                          float lambda_dist, float* d_rgb, float* d_dist, float* loss_out, void* scratch,
                          size_t scratch_bytes, cudaStream_t stream) {
  if (n_rays < 0 || (n_rays > 0 && (!rgb || !target_rgb)) || !loss_out)
    return set_error(NERFXL_E_INVALID, "bad loss arguments");
  const int nb = (int)((n_rays + kLossThreads - 1) / kLossThreads);
  if (!scratch || scratch_bytes < sizeof(float2) * (size_t)std::max(nb, 1))
    return set_error(NERFXL_E_WORKSPACE, "loss scratch too small");
  float2* sums = static_cast<float2*>(scratch);
  if (nb > 0) {
    k_loss<<<nb, kLossThreads, 0, stream>>>(n_rays, rgb, dist, target_rgb, lambda_dist, d_rgb, d_dist, sums);
    nerfxl_status st = kernel_launched("k_loss");
    if (st != NERFXL_OK) return st;
  }
  k_loss_final<<<1, kFinalThreads, 0, stream>>>(sums, nb, n_rays, lambda_dist, loss_out);
  return kernel_launched("k_loss_final");
}

nerfxl_status nerfxl_adam_update(int64_t n, float* params, const float* grads, float* m, float* v,
                                 const nerfxl_adam* opt, void* compute_copy, int32_t copy_dtype,
                                 cudaStream_t stream) {
  if (!opt || n < 0 || (n > 0 && (!params || !grads || !m || !v)) || opt->step < 1)
    return set_error(NERFXL_E_INVALID, "bad Adam arguments");
  if (copy_dtype != NERFXL_F32 && copy_dtype != NERFXL_F16 && copy_dtype != NERFXL_BF16)
    return set_error(NERFXL_E_UNSUPPORTED, "compute copy must be fp16 or bf16");
  if (copy_dtype != NERFXL_F32 && !compute_copy) return set_error(NERFXL_E_INVALID, "null compute copy");
  return launch_adam(n, params, grads, m, v, opt, compute_copy, copy_dtype == NERFXL_F32 ? 0 : copy_dtype, stream);
}

size_t nerfxl_step_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays) {
  if (validate(f, s, n_rays) != NERFXL_OK) return 0;
  const size_t nb = (size_t)std::max<int64_t>(1, (n_rays + kLossThreads - 1) / kLossThreads);
  const size_t extra = ((size_t)n_rays * (3 + 3 + 1 + 1 + 1 + 1) * sizeof(float) + nb * sizeof(float2) + 1023) /
                       256 * 256 + 1024;
  return layout(f, s, n_rays, 1).total + extra;
}

nerfxl_status nerfxl_step(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, const float* rays_o,
                          const float* rays_d, const float* target_rgb, float lambda_dist,
                          const nerfxl_train_state* st, const nerfxl_adam* opt, float* loss_out, void* workspace,
                          size_t ws_bytes, cudaStream_t stream) {
  nerfxl_status rc = validate(f, s, n_rays);
  if (rc != NERFXL_OK) return rc;
  if (!st || !opt || !loss_out) return set_error(NERFXL_E_INVALID, "null train state, optimiser or loss output");
  if (!st->tables || !st->mlp || !st->grad_tables || !st->grad_mlp || !st->m_tables || !st->v_tables ||
      !st->m_mlp || !st->v_mlp)
    return set_error(NERFXL_E_INVALID, "null train-state pointer");
  const bool tab32 = f->table_dtype == NERFXL_F32, mlp32 = f->mlp_dtype == NERFXL_F32;
  if ((tab32 && st->tables != f->tables) || (mlp32 && st->mlp != f->mlp))
    return set_error(NERFXL_E_INVALID, "an FP32 field block must be the master itself");
  if ((!tab32 && f->table_dtype != NERFXL_F16) || (!mlp32 && f->mlp_dtype != NERFXL_BF16 && f->mlp_dtype != NERFXL_F16))
    return set_error(NERFXL_E_UNSUPPORTED, "compute copies must be FP16 tables and BF16/FP16 MLP");
  const size_t need = nerfxl_step_workspace_bytes(f, s, n_rays);
  if (!workspace || ws_bytes < need) return set_error(NERFXL_E_WORKSPACE, "step workspace too small");
  const Layout L = layout(f, s, n_rays, 1);
  char* ws = static_cast<char*>(workspace);
  char* ex = ws + (L.total + 255) / 256 * 256;
  const size_t R = (size_t)n_rays;
  float* rgb = reinterpret_cast<float*>(ex);
  float* d_rgb = rgb + 3 * R;
  float* depth = d_rgb + 3 * R;
  float* opacity = depth + R;
  float* dist = opacity + R;
  float* d_dist = dist + R;
  float2* sums = reinterpret_cast<float2*>(ex + ((6 * R + 4 * R) * sizeof(float) + 255) / 256 * 256);
  const int nb = (int)std::max<int64_t>(1, (n_rays + kLossThreads - 1) / kLossThreads);
  const int64_t n_tab = (int64_t)f->K * nerfxl_table_entries(f->level_res, f->L, f->log2_T) * f->F;
  const int64_t n_mlp = nerfxl_field_mlp_params(f);
  if (cudaMemsetAsync(st->grad_tables, 0, sizeof(float) * n_tab, stream) != cudaSuccess ||
      cudaMemsetAsync(st->grad_mlp, 0, sizeof(float) * n_mlp, stream) != cudaSuccess)
    return launch_check("gradient clear");
  rc = nerfxl_render_fwd(f, s, n_rays, rays_o, rays_d, rgb, depth, opacity, dist, workspace, L.total, stream);
  if (rc != NERFXL_OK) return rc;
  rc = nerfxl_loss(n_rays, rgb, dist, target_rgb, lambda_dist, d_rgb, d_dist, loss_out, sums, sizeof(float2) * nb,
                   stream);
  if (rc != NERFXL_OK) return rc;
  rc = nerfxl_render_bwd(f, s, n_rays, rays_o, rays_d, d_rgb, nullptr, nullptr, d_dist, st->grad_tables,
                         st->grad_mlp, workspace, L.total, stream);
  if (rc != NERFXL_OK) return rc;
  // masters updated in FP32; 16-bit compute copies refreshed from them
  rc = launch_adam(n_tab, st->tables, st->grad_tables, st->m_tables, st->v_tables, opt,
                   tab32 ? nullptr : const_cast<void*>(f->tables), tab32 ? 0 : 1, stream);
  if (rc != NERFXL_OK) return rc;
  return launch_adam(n_mlp, st->mlp, st->grad_mlp, st->m_mlp, st->v_mlp, opt, mlp32 ? nullptr : const_cast<void*>(f->mlp),
                     mlp32 ? 0 : (f->mlp_dtype == NERFXL_BF16 ? 2 : 1), stream);
}

}  // extern "C"
