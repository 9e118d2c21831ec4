// 16-bit operand helpers shared by the tensor-core kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace nerfxl {

template <bool BF16>
struct Half2Of;
template <>
struct Half2Of<true> {
  __device__ static uint32_t pack(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static float load(const void* p, size_t i) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
  }
  __device__ static uint16_t bits(const void* p, size_t i) { return reinterpret_cast<const uint16_t*>(p)[i]; }
  __device__ static float2 unpack(uint32_t v) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
  }
  __device__ static float from_bits(uint16_t v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
};
template <>
struct Half2Of<false> {
  __device__ static uint32_t pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static float load(const void* p, size_t i) { return __half2float(reinterpret_cast<const __half*>(p)[i]); }
  __device__ static uint16_t bits(const void* p, size_t i) { return reinterpret_cast<const uint16_t*>(p)[i]; }
  __device__ static float2 unpack(uint32_t v) { return __half22float2(*reinterpret_cast<const __half2*>(&v)); }
  __device__ static float from_bits(uint16_t v) { return __half2float(__ushort_as_half(v)); }
};


}  // namespace nerfxl
