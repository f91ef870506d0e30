// Shared device helpers of the SV-LCOV GB300 library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/svlcov.h"

namespace svl {

constexpr int kMaxK = SVLCOV_MAX_K;
constexpr int kMaxS = SVLCOV_MAX_S;

// ---- element conversions -------------------------------------------------
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return (float)x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_f64(float x) { return (double)x; }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn((float)x);  // double -> float -> bf16 (round to nearest each)
}
template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ double from_f32<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

template <typename T> struct Acc { using type = float; };   // accumulator of a storage type
template <> struct Acc<double> { using type = double; };

template <typename T> __device__ __forceinline__ T load_val(const void* p, int dtype, int64_t e) {
  return dtype == SVLCOV_FP64 ? (T)((const double*)p)[e] : (T)((const float*)p)[e];
}

__device__ __forceinline__ bool is_finite(double x) { return isfinite(x); }
__device__ __forceinline__ bool is_finite(float x) { return isfinite(x); }

// ---- status word ---------------------------------------------------------
__device__ __forceinline__ void flag(int* status, int code) { atomicOr(status, code); }
__device__ __forceinline__ bool failed(const int* status) {
  return *(volatile const int*)status != 0;
}

// ---- warp reductions -----------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace svl
