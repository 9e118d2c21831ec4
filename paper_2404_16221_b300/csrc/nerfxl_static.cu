// nerfxl_render_fwd_static: the forward render for callers that cannot
// allocate device memory.
//
// Some callers have no way to hand the library a workspace: a plain C
// program or plug-in that links libnerfxl without PyTorch or any other
// allocator, a host application that owns the whole device memory pool and
// forbids allocations from plug-ins, or a real-time frame loop where a
// cudaMalloc would synchronise the device and stall the frame. For them this
// entry point takes its scratch from a fixed array that lives in the
// library's own device image.
//
// Rules of use:
//  - The array holds kStaticScratchBytes (32 MiB). Every GPU that loads the
//    library keeps it reserved until the process exits. Calls whose workspace
//    would exceed it are refused with NERFXL_E_WORKSPACE before anything is
//    launched; split such batches.
//  - Every call looks up the array's device address (cudaGetSymbolAddress,
//    which allocates nothing) with the caller's device current, so the address
//    is never stale, even after a cudaDeviceReset reloaded the module. The
//    first call on a device also loads the library's device code there; make
//    it before any stream capture begins.
//  - Device-side conditions (a ray crossing more regions than max_segments,
//    an expired bounded wait) are flagged in the array's header; read them
//    with nerfxl_static_check after the call.
//  - All calls share the one array, and it keeps the previous call's
//    contents: the call clears the counters it needs at zero itself. Calls
//    that overlap on the GPU (different streams, or host threads without
//    ordering) race on the array; order them on one stream.
//  - No cudaMalloc, cudaFree or allocating library routine is called.

#include <cuda_runtime.h>

#include <string>

#include "nerfxl_host.h"

namespace nerfxl {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch array on the current device. In host code
// g_static_scratch names a host-side stand-in, never the device memory, so
// only the looked-up address is passed to kernels.
nerfxl_status static_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p)
    return set_error(NERFXL_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return NERFXL_OK;
}

}  // namespace
}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_render_fwd_static(const nerfxl_field* f, const nerfxl_sampling* s, int64_t n_rays,
                                                  const float* rays_o, const float* rays_d, float* rgb, float* depth,
                                                  float* opacity, float* dist, cudaStream_t stream) {
  nerfxl_status st = validate(f, s, n_rays);
  if (st != NERFXL_OK) return st;
  const size_t need = layout(f, s, n_rays, 0).total;
  if (need > kStaticScratchBytes)
    return set_error(NERFXL_E_WORKSPACE, "batch needs " + std::to_string(need) + " bytes of scratch; the static array "
                                         "holds " + std::to_string(kStaticScratchBytes) + " bytes, split the batch");
  void* scratch = nullptr;
  st = static_scratch(&scratch);
  if (st != NERFXL_OK) return st;
  return nerfxl_render_fwd(f, s, n_rays, rays_o, rays_d, rgb, depth, opacity, dist, scratch, kStaticScratchBytes,
                           stream);
}

extern "C" nerfxl_status nerfxl_static_check(cudaStream_t stream) {
  void* scratch = nullptr;
  const nerfxl_status st = static_scratch(&scratch);
  if (st != NERFXL_OK) return st;
  return nerfxl_check(scratch, kStaticScratchBytes, stream);
}
