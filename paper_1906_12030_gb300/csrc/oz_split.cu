// Fixed-point split of the operands of the MERA_PREC_OZ3 / OZ4 modes.
//
// Every row of an operand (its contraction index K contiguous) is cut into
// blocks of kOzBlockK elements.  With e the exponent of the block's largest
// entry (2^e <= max |x| < 2^(e+1)), entry x = hi + lo (an unevaluated pair
// of binary32 values) is written as S slices
//   x ~ s_0 + s_1 + ... + s_(S-1),  s_p an integer multiple of 2^(e-7-9p),
// each s_p the remainder after s_0 .. s_(p-1) rounded to its grid, so that
// |s_0| <= 2^(e+1) and |s_p| <= 2^(e-8-9(p-1)) for p >= 1: every slice is
// an integer of at most 256 in magnitude times a power of two, a BF16 value
// exactly.  Slice 0 of every entry of a block is thus an integer multiple of
// 2^(e-7) of magnitude at most 2^(e+1), which is what lets the GEMM sum a
// block's leading products exactly (oz_gemm.cuh).  What the slices leave
// out is at most 2^(e-8-9(S-1)) per entry (OZ3 2^(e-26), OZ4 2^(e-35)).
// This is the splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 59, 2012), with one exponent per row block.
//
// Arithmetic: rounding y to the grid 2^q is (y + c) - c with
// c = 1.5 * 2^(q+23) (exact for |y| < 2^(q+22), the usual binary32 trick);
// the remainder y - s is exact, and it is added to the running lo part with
// Knuth's TwoSum, so the pair (hi, lo) carries the exact remainder through
// every slice.  Everything runs on the FP32 pipe (this GPU's FP64 and 64-bit
// conversion rates are a small fraction of it).  Blocks whose largest entry
// is below 2^-90 (or zero) are written as zeros.
#include "common.cuh"
#include "kernels.h"

namespace mera {
namespace {

// 1.5 * 2^(q + 23) as binary32 bits (q + 150 in [1, 254]).
__device__ __forceinline__ float round_magic(int q) { return __int_as_float(((q + 150) << 23) | (1 << 22)); }

// hi + lo -> (s, hi', lo') with s = hi rounded to the grid of `magic` and
// hi' + lo' = hi + lo - s exactly.
__device__ __forceinline__ float take_slice(float& hi, float& lo, float magic) {
  const float s = __fsub_rn(__fadd_rn(hi, magic), magic);
  const float r = __fsub_rn(hi, s);  // exact
  const float t = __fadd_rn(r, lo);  // TwoSum(r, lo)
  const float bp = __fsub_rn(t, r);
  lo = __fadd_rn(__fsub_rn(r, __fsub_rn(t, bp)), __fsub_rn(lo, bp));
  hi = t;
  return s;
}

template <int S>
__global__ void __launch_bounds__(256) oz_split_kernel(const float* __restrict__ raw, int64_t raw_plane,
                                                       __nv_bfloat16* __restrict__ dst, int64_t dst_plane,
                                                       int64_t rows, int64_t K, int64_t ld) {
  constexpr int kPairs = kOzBlockK / 64;  // element pairs per lane
  const int lane = threadIdx.x & 31;
  const int64_t nblk = (K + kOzBlockK - 1) / kOzBlockK;
  const int64_t items = rows * nblk;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
  for (int64_t it = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; it < items; it += warps) {
    const int64_t r = it / nblk, g = it - r * nblk;
    const int64_t base = r * ld + g * kOzBlockK;  // even: ld is a multiple of 8
    const int n = int(min(int64_t(kOzBlockK), K - g * kOzBlockK));
    float h[2 * kPairs], l[2 * kPairs];
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
      const int k = 2 * lane + 64 * q;
      h[2 * q] = h[2 * q + 1] = l[2 * q] = l[2 * q + 1] = 0.0f;
      if (k + 1 < n) {
        const float2 a = *reinterpret_cast<const float2*>(raw + base + k);
        const float2 b = *reinterpret_cast<const float2*>(raw + raw_plane + base + k);
        h[2 * q] = a.x;
        h[2 * q + 1] = a.y;
        l[2 * q] = b.x;
        l[2 * q + 1] = b.y;
      } else if (k < n) {
        h[2 * q] = raw[base + k];
        l[2 * q] = raw[raw_plane + base + k];
      }
      mx = fmaxf(mx, fmaxf(fabsf(h[2 * q]), fabsf(h[2 * q + 1])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // 2^e <= max |hi| < 2^(e+1); |hi + lo| < 2^(e+1) as well, |lo| being at
    // most half an ulp of hi
    const int e = (__float_as_int(mx) >> 23) - 127;
    const bool zero = !(mx >= 0x1p-90f);  // also catches a NaN maximum
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
      const int k = 2 * lane + 64 * q;
      if (k >= n) continue;
      float hi0 = h[2 * q], lo0 = l[2 * q], hi1 = h[2 * q + 1], lo1 = l[2 * q + 1];
#pragma unroll
      for (int p = 0; p < S; ++p) {
        float s0 = 0.0f, s1 = 0.0f;
        if (!zero) {
          const float c = round_magic(e - 7 - 9 * p);
          s0 = take_slice(hi0, lo0, c);
          s1 = take_slice(hi1, lo1, c);
        }
        __nv_bfloat16* d = dst + p * dst_plane + base + k;
        if (k + 1 < n) {
          *reinterpret_cast<__nv_bfloat162*>(d) = __floats2bfloat162_rn(s0, s1);
        } else {
          d[0] = __float2bfloat16_rn(s0);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_oz_split(const float* raw, int64_t raw_plane, void* dst, int64_t dst_plane, int64_t rows,
                            int64_t K, int64_t ld, int slices, cudaStream_t stream) {
  if (rows <= 0 || K <= 0) return cudaSuccess;
  if (K > ld || (ld & 1) || (raw_plane & 1) || (dst_plane & 1)) return cudaErrorInvalidValue;
  const int64_t items = rows * ((K + kOzBlockK - 1) / kOzBlockK);
  const unsigned grid = unsigned(std::min<int64_t>((items + 7) / 8, int64_t(152) * 16));
  auto* out = static_cast<__nv_bfloat16*>(dst);
  count_launch();
  switch (slices) {
    case 3: oz_split_kernel<3><<<grid, 256, 0, stream>>>(raw, raw_plane, out, dst_plane, rows, K, ld); break;
    case 4: oz_split_kernel<4><<<grid, 256, 0, stream>>>(raw, raw_plane, out, dst_plane, rows, K, ld); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mera
