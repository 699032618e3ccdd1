// pixel.cuh -- per-dtype pixel conversions and rounding shared by all kernels
// of libds, so that every kernel (fused, general, unfused) produces the same
// bits for the same plan.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace ds {

// Pixel value as float.  uint8 values are exact small integers.
__device__ __forceinline__ float px_to_f(float v) { return v; }
__device__ __forceinline__ float px_to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float px_to_f(uint8_t v) { return (float)v; }

// Rounding applied after each pass.  Float dtypes keep the FP32 sum.  For
// uint8 the sum is an exact integer (|sum| < 2^24, so every FMA of integer
// taps by integer pixels is exact): (acc + 2^13) >> 14 with a floor shift,
// then clamp to [0, 255].  acc * 2^-14 + 1/2 is exact in FP32 for |acc| < 2^23.
template <typename T>
__device__ __forceinline__ float pass_round(float acc) { return acc; }
template <>
__device__ __forceinline__ float pass_round<uint8_t>(float acc) {
  const float v = floorf(fmaf(acc, 1.0f / 16384.0f, 0.5f));
  return fminf(fmaxf(v, 0.0f), 255.0f);
}

// Final conversion of a (pass-rounded) value to the output type.
template <typename T>
__device__ __forceinline__ T f_to_px(float v);
template <>
__device__ __forceinline__ float f_to_px<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half f_to_px<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ uint8_t f_to_px<uint8_t>(float v) { return (uint8_t)(int)v; }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

}  // namespace ds
