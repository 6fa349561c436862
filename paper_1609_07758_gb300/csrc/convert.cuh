// FP64 <-> FP32 conversions on the integer pipes.  On GB300 a conversion that involves
// FP64 (F2F) issues to the FP64 pipe, two lanes per SM and cycle, which the FP64 operator
// sweeps saturate: converting the 85M values of its FP32 output there cost 0.13 ms a
// sweep.  These helpers rebuild the IEEE bit patterns with integer and logic operations
// instead (about a dozen instructions, so kernels bound by instruction issue rather than
// by the FP64 pipe keep the conversion instruction).  In the normal range both give exactly the results of the
// conversion instructions (round to nearest even for FP64 -> FP32; FP32 -> FP64 is exact);
// magnitudes below the smallest normal FP32 number flush to zero, and overflow or a NaN
// becomes an infinity of the same sign.
#pragma once
#include <cuda_runtime.h>

namespace hofem {

__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;   // FP32 biased exponent
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
  const unsigned rest = lo & 0x1FFFFFFFu, half = 0x10000000u;
  // exponent and mantissa added so that a rounding carry moves into the exponent
  unsigned bits = ((unsigned)(e > 0 ? e : 0) << 23) + m + ((rest > half || (rest == half && (m & 1u))) ? 1u : 0u);
  bits = e <= 0 ? 0u : (e >= 255 || bits >= 0x7F800000u) ? 0x7F800000u : bits;
  return __uint_as_float(sign | bits);
}

__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned ed = e == 0u ? 0u : e == 255u ? 2047u : e + (1023u - 127u);
  const unsigned mant = e == 0u ? 0u : (b & 0x7FFFFFu);
  const unsigned hi = (b & 0x80000000u) | (ed << 20) | (mant >> 3);
  return __hiloint2double((int)hi, (int)((mant & 0x7u) << 29));
}

}  // namespace hofem
