// Rounding of FP32 values to the tensor-core operand formats (round to
// nearest even), and the test for a non-finite result (an FP16 overflow, or a
// NaN or infinity in either format), which the casting kernels report as
// ST_RANGE.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace gb {

template <typename H>
__device__ __forceinline__ H to16(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to16<__half>(float v) {
  return __float2half_rn(v);
}
template <typename H>
__device__ __forceinline__ bool bad16(H h);
template <>
__device__ __forceinline__ bool bad16<__nv_bfloat16>(__nv_bfloat16 h) {
  return (__bfloat16_as_ushort(h) & 0x7f80u) == 0x7f80u;
}
template <>
__device__ __forceinline__ bool bad16<__half>(__half h) {
  return (__half_as_ushort(h) & 0x7c00u) == 0x7c00u;
}
template <typename H>
__device__ __forceinline__ unsigned short bits16(H h);
template <>
__device__ __forceinline__ unsigned short bits16<__nv_bfloat16>(__nv_bfloat16 h) {
  return __bfloat16_as_ushort(h);
}
template <>
__device__ __forceinline__ unsigned short bits16<__half>(__half h) {
  return __half_as_ushort(h);
}

}  // namespace gb
