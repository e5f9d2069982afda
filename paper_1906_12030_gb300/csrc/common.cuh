// Device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace mera {

// Linear index -> offset over up to kMaxLeg legs, last leg fastest.
__device__ __forceinline__ int64_t legmap_offset(const LegMap& m, int64_t idx) {
  int64_t off = 0;
#pragma unroll 1
  for (int i = m.n - 1; i >= 0; --i) {
    const int64_t d = m.dim[i];
    const int64_t q = idx / d;
    off += (idx - q * d) * m.stride[i];
    idx = q;
  }
  return off;
}

// Same, for indices below 2^31 (every GEMM row/column index; M, N < 2^31 is
// checked at launch): 32-bit division is several times cheaper.
__device__ __forceinline__ int64_t legmap_offset32(const LegMap& m, uint32_t idx) {
  int64_t off = 0;
#pragma unroll 1
  for (int i = m.n - 1; i >= 0; --i) {
    const uint32_t d = uint32_t(m.dim[i]);
    const uint32_t q = idx / d;
    off += int64_t(idx - q * d) * m.stride[i];
    idx = q;
  }
  return off;
}

// Round a float to TF32 (10 explicit mantissa bits), nearest, ties away.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Store one value into an operand buffer of precision `prec`.
// `plane` is the element distance between the hi and lo planes (BF16X3).
template <int PREC>
struct OperandStore;

template <>
struct OperandStore<PREC_F64> {
  using T = double;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t, double v) {
    static_cast<double*>(base)[off] = v;
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t, float f) {
    static_cast<double*>(base)[off] = double(f);
  }
};
// The reduced-precision stores convert binary64 -> binary32 once and split in
// FP32: GB300's FP64 pipe is ~1/1800 of its BF16 tensor rate, so every extra
// binary64 operation per element shows up directly in the copy time.  FP32
// keeps 24 significant bits, more than any of these operand formats holds.
template <>
struct OperandStore<PREC_TF32> {
  using T = float;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t, double v) {
    store_f(base, off, 0, __double2float_rn(v));
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t, float f) {
    static_cast<float*>(base)[off] = round_tf32(f);
  }
};
template <>
struct OperandStore<PREC_BF16> {
  using T = __nv_bfloat16;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t, double v) {
    store_f(base, off, 0, __double2float_rn(v));
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t, float f) {
    static_cast<__nv_bfloat16*>(base)[off] = __float2bfloat16_rn(f);
  }
};
template <>
struct OperandStore<PREC_BF16X3> {
  using T = __nv_bfloat16;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t plane, double v) {
    store_f(base, off, plane, __double2float_rn(v));
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t plane, float f) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
    static_cast<__nv_bfloat16*>(base)[off] = hi;
    static_cast<__nv_bfloat16*>(base)[off + plane] = lo;
  }
};
template <>
struct OperandStore<PREC_BF16X6> {
  using T = __nv_bfloat16;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t plane, double v) {
    store_f(base, off, plane, __double2float_rn(v));
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t plane, float f) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    __nv_bfloat16* b = static_cast<__nv_bfloat16*>(base);
    b[off] = hi;
    b[off + plane] = mid;
    b[off + 2 * plane] = lo;
  }
};

// Fixed-point split modes: inputs are first stored as an unevaluated pair
// hi + lo of binary32 values (hi = x rounded to binary32, lo = the rest
// rounded; ~48 significant bits) in two planes, then split per block
// (oz_split.cu).
template <>
struct OperandStore<PREC_RAW> {
  using T = float;
  __device__ __forceinline__ static void store(void* base, int64_t off, int64_t plane, double v) {
    const float hi = __double2float_rn(v);
    const float lo = __double2float_rn(v - double(hi));
    static_cast<float*>(base)[off] = hi;
    static_cast<float*>(base)[off + plane] = lo;
  }
  __device__ __forceinline__ static void store_f(void* base, int64_t off, int64_t plane, float f) {
    static_cast<float*>(base)[off] = f;
    static_cast<float*>(base)[off + plane] = 0.0f;
  }
};

}  // namespace mera
