// Bounded-wait probe: exercises the timeout path of the tensor-core kernels'
// mbarrier waits without faulting anything. A single thread initialises an
// mbarrier, arrives on it or not, and waits a bounded number of polls; the
// outcome is written to device memory and reported as NERFXL_OK or
// NERFXL_E_TIMEOUT by the host.

#include <cuda_runtime.h>

#include "nerfxl_host.h"
#include "nerfxl_tc.cuh"

namespace nerfxl {

__global__ void k_wait_probe(int32_t* status, uint32_t spins, int arrive) {
  __shared__ uint64_t mbar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&mbar, 1);
  if (arrive) {
    uint64_t token;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(token) : "r"(tc::smem_u32(&mbar)) : "memory");
    (void)token;
  }
  *status = tc::mbar_wait_bounded(&mbar, 0, spins) ? 1 : 0;
}

}  // namespace nerfxl

using namespace nerfxl;

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
