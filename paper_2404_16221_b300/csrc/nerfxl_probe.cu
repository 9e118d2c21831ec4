// Probes.
// Bounded-wait probe: exercises the timeout path of the tensor-core kernels'
// mbarrier waits without faulting anything. A single thread initialises an
// mbarrier, arrives on it or not, and waits a bounded number of polls; the
// outcome is written to device memory and reported as NERFXL_OK or
// NERFXL_E_TIMEOUT by the host.
// Reduction-rate probe: the rate at which the GPU takes scattered 16-byte
// FP32 reductions (red.global.add.v4.f32 with the evict-last hint, as the
// backward's table scatter issues them) into a caller-owned buffer, the
// resource that bounds the backward kernels. Load-rate probe: the rate of
// scattered 8-byte loads (one sector each), the resource that bounds the
// forward's table gather.

#include <cuda_runtime.h>

#include "nerfxl_host.h"
#include "nerfxl_tc.cuh"

namespace nerfxl {

__global__ void k_wait_probe(int32_t* status, uint32_t spins, int arrive) {
  __shared__ uint64_t mbar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&mbar, 1);
  if (arrive) tc::mbar_arrive(&mbar);
  *status = tc::mbar_wait_bounded(&mbar, 0, spins) ? 1 : 0;
}

// Every thread adds 1 to `iters` float4 slots picked by a mixing hash of
// (thread, iteration), all inside buf[0, n16).
__global__ void __launch_bounds__(256) k_reduction_rate(float4* buf, uint32_t n16, int iters) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t pol = tc::policy_evict_last();
  for (int i = 0; i < iters; ++i) {
    uint32_t x = gid * 0x9E3779B1u + (uint32_t)i * 0x85EBCA77u;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    tc::red_add_v4(buf + x % n16, make_float4(1.0f, 1.0f, 1.0f, 1.0f), pol);
  }
}

// Every thread loads 16 independent 8-byte words per iteration from slots
// picked by a mixing hash, all inside buf[0, n8), and folds them into one word
// (stored only under an impossible condition, so that the loads stay).
constexpr int kLoadProbeUnroll = 16;
__global__ void __launch_bounds__(256) k_load_rate(const uint2* __restrict__ buf, uint32_t n8, int iters,
                                                   uint32_t* __restrict__ sink) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    uint2 v[kLoadProbeUnroll];
#pragma unroll
    for (int u = 0; u < kLoadProbeUnroll; ++u) {
      uint32_t x = gid * 0x9E3779B1u + (uint32_t)(i * kLoadProbeUnroll + u) * 0x85EBCA77u;
      x ^= x >> 16;
      x *= 0x7FEB352Du;
      x ^= x >> 15;
      x *= 0x846CA68Bu;
      x ^= x >> 16;
      v[u] = __ldg(buf + x % n8);
    }
#pragma unroll
    for (int u = 0; u < kLoadProbeUnroll; ++u) acc ^= v[u].x + v[u].y;
  }
  if (acc == 0x9E3779B9u && gid == 0xFFFFFFFFu) *sink = acc;
}

}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_probe_load_rate(const void* buf, size_t bytes, int32_t iters, int64_t* ops,
                                                cudaStream_t stream) {
  if (!buf || bytes < 8 || bytes / 8 > 0xFFFFFFFFull || iters <= 0 || !ops ||
      (reinterpret_cast<uintptr_t>(buf) & 7u))
    return set_error(NERFXL_E_INVALID, "bad load probe arguments");
  const int grid = num_sms() * 4;
  // the sink is never written (its condition cannot hold: gid < 2^32 - 1)
  k_load_rate<<<grid, 256, 0, stream>>>(static_cast<const uint2*>(buf), (uint32_t)(bytes / 8), iters,
                                        static_cast<uint32_t*>(const_cast<void*>(buf)));
  *ops = (int64_t)grid * 256 * iters * kLoadProbeUnroll;
  return kernel_launched("k_load_rate");
}

extern "C" nerfxl_status nerfxl_probe_reduction_rate(void* buf, size_t bytes, int32_t iters, int64_t* ops,
                                                     cudaStream_t stream) {
  if (!buf || bytes < 16 || bytes / 16 > 0xFFFFFFFFull || iters <= 0 || !ops ||
      (reinterpret_cast<uintptr_t>(buf) & 15u))
    return set_error(NERFXL_E_INVALID, "bad reduction probe arguments");
  const int grid = num_sms() * 4;
  k_reduction_rate<<<grid, 256, 0, stream>>>(static_cast<float4*>(buf), (uint32_t)(bytes / 16), iters);
  *ops = (int64_t)grid * 256 * iters;
  return kernel_launched("k_reduction_rate");
}

extern "C" nerfxl_status nerfxl_debug_wait_probe(int32_t* status, uint32_t spins, int32_t arrive,
                                                cudaStream_t stream) {
  if (!status || spins == 0 || spins > (1u << 26)) return set_error(NERFXL_E_INVALID, "bad probe arguments");
  k_wait_probe<<<1, 32, 0, stream>>>(status, spins, arrive);
  nerfxl_status st = kernel_launched("k_wait_probe");
  if (st != NERFXL_OK) return st;
  int32_t h = -1;
  if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return launch_check("k_wait_probe result");
  if (h == 0) return set_error(NERFXL_E_TIMEOUT, "bounded wait expired (probe)");
  return NERFXL_OK;
}
