// Loss, optimiser and the fused training step of the one-GPU NeRF-XL path.
//
// Loss (photometric L2 plus the distortion regulariser of Sec. 4.1, Eq. 2):
//   L = mean_{r,c} (C_rc - C*_rc)^2 + lambda * mean_r L_dist,r
// Its output adjoints are dL/dC = 2 (C - C*) / (3R), dL/dL_dist = lambda / R.
// Adam (Kingma & Ba) with bias correction updates the FP32 master parameters.

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "nerfxl_host.h"

namespace nerfxl {

constexpr int kLossThreads = 256;

// Kahan-compensated block sums of the two loss terms; per-ray adjoints.
// R rays of a batch whose loss is a mean over R_norm rays (R_norm > R when the
// batch is one sub-batch of a larger step).
__global__ void __launch_bounds__(kLossThreads) k_loss(int64_t R, int64_t R_norm, const float* __restrict__ rgb,
                                                       const float* __restrict__ dist,
                                                       const float* __restrict__ target, float lambda,
                                                       float* __restrict__ d_rgb, float* __restrict__ d_dist,
                                                       float2* __restrict__ block_sums) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float photo = 0.0f, dd = 0.0f;
  if (r < R) {
    const float inv = 1.0f / (3.0f * (float)R_norm);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float e = rgb[3 * r + c] - target[3 * r + c];
      photo += e * e;
      if (d_rgb) d_rgb[3 * r + c] = 2.0f * e * inv;
    }
    dd = dist ? dist[r] : 0.0f;
    if (d_dist) d_dist[r] = lambda / (float)R_norm;
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
// One parameter's update (the same arithmetic in the scalar and vector forms).
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1, float b2, float eps,
                                      float inv_c1, float inv_sqrt_c2) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  // lr * mhat / (sqrt(vhat) + eps), mhat = m / c1, vhat = v / c2
  p = p - lr * (m * inv_c1) / (sqrtf(v) * inv_sqrt_c2 + eps);
}

__device__ __forceinline__ void store_copy(void* copy, int copy_dtype, int64_t i, float p) {
  if (copy_dtype == 1) reinterpret_cast<__half*>(copy)[i] = __float2half_rn(p);
  else if (copy_dtype == 2) reinterpret_cast<__nv_bfloat16*>(copy)[i] = __float2bfloat16_rn(p);
}

// Scalar form (any alignment) over [i0, n).
__global__ void __launch_bounds__(256) k_adam(int64_t i0, int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                              float b2, float eps, float inv_c1, float inv_sqrt_c2,
                                              void* __restrict__ copy, int copy_dtype) {
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float pi = p[i], mi = m[i], vi = v[i];
    adam1(pi, g[i], mi, vi, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
    store_copy(copy, copy_dtype, i, pi);
  }
}

// Vector form: four parameters per thread and iteration (16-byte loads and
// stores of the FP32 arrays, 8 bytes of the 16-bit copy), for 16-byte-aligned
// arrays; n4 groups of four.
__global__ void __launch_bounds__(256) k_adam4(int64_t n4, float4* __restrict__ p, const float4* __restrict__ g,
                                               float4* __restrict__ m, float4* __restrict__ v, float lr, float b1,
                                               float b2, float eps, float inv_c1, float inv_sqrt_c2,
                                               void* __restrict__ copy, int copy_dtype) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 pi = p[i], mi = m[i], vi = v[i];
    const float4 gi = __ldcs(g + i);  // read once
    adam1(pi.x, gi.x, mi.x, vi.x, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam1(pi.y, gi.y, mi.y, vi.y, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam1(pi.z, gi.z, mi.z, vi.z, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam1(pi.w, gi.w, mi.w, vi.w, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
    if (copy_dtype == 1) {
      const __half2 a = __floats2half2_rn(pi.x, pi.y), b = __floats2half2_rn(pi.z, pi.w);
      reinterpret_cast<uint2*>(copy)[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                                                     *reinterpret_cast<const uint32_t*>(&b));
    } else if (copy_dtype == 2) {
      const __nv_bfloat162 a = __floats2bfloat162_rn(pi.x, pi.y), b = __floats2bfloat162_rn(pi.z, pi.w);
      reinterpret_cast<uint2*>(copy)[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                                                     *reinterpret_cast<const uint32_t*>(&b));
    }
  }
}

nerfxl_status launch_adam(int64_t n, float* p, const float* g, float* m, float* v, const nerfxl_adam* opt,
                          void* copy, int copy_dtype, cudaStream_t stream) {
  if (n <= 0) return NERFXL_OK;
  const double c1 = 1.0 - std::pow((double)opt->beta1, (double)opt->step);
  const double c2 = 1.0 - std::pow((double)opt->beta2, (double)opt->step);
  const float inv_c1 = (float)(1.0 / c1), inv_sqrt_c2 = (float)(1.0 / std::sqrt(c2));
  auto aligned = [](const void* q, uintptr_t a) { return (reinterpret_cast<uintptr_t>(q) & (a - 1)) == 0; };
  const bool vec = aligned(p, 16) && aligned(g, 16) && aligned(m, 16) && aligned(v, 16) &&
                   (copy_dtype == 0 || aligned(copy, 8));
  const int64_t n4 = vec ? n / 4 : 0;
  if (n4 > 0) {
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, (int64_t)num_sms() * 8);
    k_adam4<<<blocks, 256, 0, stream>>>(n4, reinterpret_cast<float4*>(p), reinterpret_cast<const float4*>(g),
                                        reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), opt->lr,
                                        opt->beta1, opt->beta2, opt->eps, inv_c1, inv_sqrt_c2, copy, copy_dtype);
    const nerfxl_status st = kernel_launched("k_adam4");
    if (st != NERFXL_OK) return st;
  }
  if (4 * n4 < n) {  // the tail (or everything, unaligned)
    const int64_t rest = n - 4 * n4;
    const int blocks = (int)std::min<int64_t>((rest + 255) / 256, (int64_t)num_sms() * 16);
    k_adam<<<blocks, 256, 0, stream>>>(4 * n4, n, p, g, m, v, opt->lr, opt->beta1, opt->beta2, opt->eps, inv_c1,
                                       inv_sqrt_c2, copy, copy_dtype);
    return kernel_launched("k_adam");
  }
  return NERFXL_OK;
}

// E4M3 weight quantisation of fused MLP blocks (the FP8 experiment of the
// precision forms). Per region k and layer li (W1, W2, W3 of the block):
//   scale[k][li] = max(max |W|, 1e-30) / 448   (448: the largest finite E4M3 value)
//   q = e4m3(W / scale), round to nearest even, saturating to +-448,
// so W ~= scale * q. One block per (region, layer) finds max |W| in a fixed
// order (exact: a maximum does not round).
constexpr int kQuantThreads = 256;
__global__ void __launch_bounds__(kQuantThreads) k_e4m3_scales(const float* __restrict__ mlp, int64_t P, int64_t n1,
                                                               int64_t n2, int64_t n3, float* __restrict__ scales) {
  const int k = blockIdx.x, li = blockIdx.y;
  const int64_t off = li == 0 ? 0 : (li == 1 ? n1 : n1 + n2);
  const int64_t n = li == 0 ? n1 : (li == 1 ? n2 : n3);
  const float* w = mlp + (int64_t)k * P + off;
  float a = 0.0f;
  for (int64_t i = threadIdx.x; i < n; i += kQuantThreads) a = fmaxf(a, fabsf(w[i]));
  __shared__ float s_a[kQuantThreads];
  s_a[threadIdx.x] = a;
  __syncthreads();
  for (int o = kQuantThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_a[threadIdx.x] = fmaxf(s_a[threadIdx.x], s_a[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scales[3 * k + li] = __fdiv_rn(fmaxf(s_a[0], 1e-30f), 448.0f);
}

__global__ void __launch_bounds__(kQuantThreads) k_e4m3_quantize(const float* __restrict__ mlp, int64_t P, int64_t K,
                                                                 int64_t n1, int64_t n2,
                                                                 const float* __restrict__ scales,
                                                                 uint8_t* __restrict__ q) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K * P; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / P, j = i % P;
    const int li = j < n1 ? 0 : (j < n1 + n2 ? 1 : 2);
    q[i] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(mlp[i], scales[3 * k + li]), __NV_SATFINITE, __NV_E4M3);
  }
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
    k_loss<<<nb, kLossThreads, 0, stream>>>(n_rays, n_rays, rgb, dist, target_rgb, lambda_dist, d_rgb, d_dist, sums);
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

nerfxl_status nerfxl_quantize_e4m3(int32_t K, int32_t mlp_in, int32_t width, const float* mlp, uint8_t* q,
                                   float* scales, cudaStream_t stream) {
  if (K < 1 || K > NERFXL_MAX_REGIONS || mlp_in < 1 || width < 1 || !mlp || !q || !scales)
    return set_error(NERFXL_E_INVALID, "bad E4M3 quantisation arguments");
  const int64_t n1 = (int64_t)mlp_in * width, n2 = (int64_t)width * width, n3 = (int64_t)width * 4;
  const int64_t P = n1 + n2 + n3;
  k_e4m3_scales<<<dim3((unsigned)K, 3), kQuantThreads, 0, stream>>>(mlp, P, n1, n2, n3, scales);
  nerfxl_status st = kernel_launched("k_e4m3_scales");
  if (st != NERFXL_OK) return st;
  const int blocks = (int)std::min<int64_t>((K * P + kQuantThreads - 1) / kQuantThreads, 148 * 8);
  k_e4m3_quantize<<<blocks, kQuantThreads, 0, stream>>>(mlp, P, K, n1, n2, scales, q);
  return kernel_launched("k_e4m3_quantize");
}

}  // extern "C"

namespace nerfxl {
namespace {

// Workspace of a training step over R rays run in sub-batches of Rb rays:
// the backward layout of Rb rays, Rb rays of outputs and adjoints
// (rgb, d_rgb [3], depth, opacity, dist, d_dist), and the loss's block sums
// of all R rays.
size_t step_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t Rb, int64_t R) {
  const size_t nb = (size_t)std::max<int64_t>(1, (R + kLossThreads - 1) / kLossThreads);
  const size_t per_ray = ((size_t)Rb * 10 * sizeof(float) + 255) / 256 * 256;
  return (layout(f, s, Rb, 1).total + 255) / 256 * 256 + per_ray + nb * sizeof(float2) + 256;
}

// Largest sub-batch (the whole batch, else a multiple of the loss block) whose
// step workspace fits in ws_bytes; 0 if none does.
int64_t step_sub_batch(const nerfxl_field* f, const nerfxl_sampling* s, int64_t R, size_t ws_bytes) {
  if (R == 0 || step_bytes(f, s, R, R) <= ws_bytes) return R;
  int64_t lo = 0, hi = (R - 1) / kLossThreads;  // in units of kLossThreads rays
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (step_bytes(f, s, mid * kLossThreads, R) <= ws_bytes) lo = mid;
    else hi = mid - 1;
  }
  return lo * kLossThreads;
}

}  // namespace
}  // namespace nerfxl

extern "C" {

size_t nerfxl_step_workspace_bytes(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays) {
  if (validate(f, s, n_rays) != NERFXL_OK) return 0;
  return step_bytes(f, s, n_rays, n_rays);
}

int64_t nerfxl_step_sub_batch(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays, size_t ws_bytes) {
  if (validate(f, s, n_rays) != NERFXL_OK) return -1;
  return step_sub_batch(f, s, n_rays, ws_bytes);
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
  const int64_t Rb = workspace ? step_sub_batch(f, s, n_rays, ws_bytes) : 0;
  if (n_rays > 0 && Rb == 0)
    return set_error(NERFXL_E_WORKSPACE, "step workspace too small even for a sub-batch of 256 rays");
  const Layout L = layout(f, s, Rb, 1);
  char* ws = static_cast<char*>(workspace);
  char* ex = ws + (L.total + 255) / 256 * 256;
  float* rgb = reinterpret_cast<float*>(ex);
  float* d_rgb = rgb + 3 * (size_t)Rb;
  float* depth = d_rgb + 3 * (size_t)Rb;
  float* opacity = depth + Rb;
  float* dist = opacity + Rb;
  float* d_dist = dist + Rb;
  float2* sums = reinterpret_cast<float2*>(ex + ((size_t)Rb * 10 * sizeof(float) + 255) / 256 * 256);
  const int nb = (int)std::max<int64_t>(1, (n_rays + kLossThreads - 1) / kLossThreads);
  const int64_t n_tab = (int64_t)f->K * nerfxl_table_entries(f->level_res, f->L, f->log2_T) * f->F;
  const int64_t n_mlp = nerfxl_field_mlp_params(f);
  if (cudaMemsetAsync(st->grad_tables, 0, sizeof(float) * n_tab, stream) != cudaSuccess ||
      cudaMemsetAsync(st->grad_mlp, 0, sizeof(float) * n_mlp, stream) != cudaSuccess)
    return launch_check("gradient clear");
  // Sub-batches: forward, per-ray loss adjoints (normalised by all n_rays) and
  // backward, the gradients accumulating over the sub-batches; the loss's
  // block sums land at each sub-batch's own blocks, so the loss is the same
  // fixed-order sum as in one pass.
  for (int64_t b0 = 0; b0 < n_rays; b0 += Rb) {
    const int64_t n = std::min<int64_t>(Rb, n_rays - b0);
    const float* o = rays_o + 3 * b0;
    const float* d = rays_d + 3 * b0;
    const size_t Ln = layout(f, s, n, 1).total;
    rc = nerfxl_render_fwd(f, s, n, o, d, rgb, depth, opacity, dist, workspace, Ln, stream);
    if (rc != NERFXL_OK) return rc;
    k_loss<<<(int)((n + kLossThreads - 1) / kLossThreads), kLossThreads, 0, stream>>>(
        n, n_rays, rgb, dist, target_rgb + 3 * b0, lambda_dist, d_rgb, d_dist, sums + b0 / kLossThreads);
    rc = kernel_launched("k_loss");
    if (rc != NERFXL_OK) return rc;
    rc = nerfxl_render_bwd(f, s, n, o, d, d_rgb, nullptr, nullptr, d_dist, st->grad_tables, st->grad_mlp, workspace,
                           Ln, stream);
    if (rc != NERFXL_OK) return rc;
  }
  k_loss_final<<<1, kFinalThreads, 0, stream>>>(sums, n_rays > 0 ? nb : 0, n_rays, lambda_dist, loss_out);
  rc = kernel_launched("k_loss_final");
  if (rc != NERFXL_OK) return rc;
  // masters updated in FP32; 16-bit compute copies refreshed from them
  rc = launch_adam(n_tab, st->tables, st->grad_tables, st->m_tables, st->v_tables, opt,
                   tab32 ? nullptr : const_cast<void*>(f->tables), tab32 ? 0 : 1, stream);
  if (rc != NERFXL_OK) return rc;
  return launch_adam(n_mlp, st->mlp, st->grad_mlp, st->m_mlp, st->v_mlp, opt, mlp32 ? nullptr : const_cast<void*>(f->mlp),
                     mlp32 ? 0 : (f->mlp_dtype == NERFXL_BF16 ? 2 : 1), stream);
}

}  // extern "C"
