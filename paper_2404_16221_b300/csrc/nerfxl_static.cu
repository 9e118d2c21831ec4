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
//  - The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture begins.
//  - All calls share the one array, and it keeps the previous call's
//    contents: the call clears the counters it needs at zero itself. Calls
//    that overlap on the GPU (different streams, or host threads without
//    ordering) race on the array; order them on one stream.
//  - No cudaMalloc, cudaFree or allocating library routine is called.

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "nerfxl_host.h"

namespace nerfxl {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device. In host code g_static_scratch names a host-side stand-in, never
// the device memory, so only the looked-up address is passed to kernels.
nerfxl_status static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(NERFXL_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(NERFXL_E_UNSUPPORTED, "device index beyond 64");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(NERFXL_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
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
