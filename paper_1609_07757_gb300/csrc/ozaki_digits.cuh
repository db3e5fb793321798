// ozaki_digits.cuh -- the exact bf16 slicing of FP64 values used by the
// tensor-core FP64-accurate products (ozaki.cuh) and by every kernel that cuts
// operands for them (density.cu).  Device functions only.
#pragma once
#include <cuda_bf16.h>

#include "ozaki_types.cuh"

namespace iscsi {

// Slicing in integer arithmetic (GB300's FP64 units are slow): with |v| < 2^e,
// N = round(v 2^(49-e)) is read off the FP64 bit pattern, then cut into
// balanced base-128 digits, least significant first: N = sum_t a_t 2^(7(6-t)),
// |a_t| <= 64 for t >= 1 and |a_0| <= 128, i.e. v 2^-e = 2^-7 sum_t a_t 2^-7t
// up to the rounding of N (<= 2^-50).
__device__ __forceinline__ void oz_digits(double v, int e, int (&a)[OZ_S]) {
  long long bits = __double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7FF);
  long long N = 0;
  if (E != 0) {  // zeros and subnormals give N = 0 (far below the slice resolution)
    long long m = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    int sh = (E - 1075) + 49 - e;  // v = m 2^(E-1075); N = m 2^sh, sh <= -4 when |v| < 2^e
    if (sh >= 0) N = m << (sh > 10 ? 10 : sh);
    else if (sh > -63) N = (m + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) N = -N;
  }
  // the digits in 32-bit halves, N = hi 2^28 + lo with 0 <= lo < 2^28: a digit
  // of x is (x + 64 mod 128) - 64 and leaves floor((x + 64) / 128); the low
  // half's four digits leave a carry of 0 or 1 for the high half
  static_assert(OZ_S == 7, "four digits in the low 28 bits, two and a[0] in the rest");
  int x = (int)(N & 0x0FFFFFFFll);
#pragma unroll
  for (int t = OZ_S - 1; t >= OZ_S - 4; --t) {
    const int s = x + 64;
    a[t] = (s & 127) - 64;
    x = s >> 7;
  }
  x += (int)(N >> 28);
#pragma unroll
  for (int t = OZ_S - 5; t >= 1; --t) {
    const int s = x + 64;
    a[t] = (s & 127) - 64;
    x = s >> 7;
  }
  a[0] = x;
}

__device__ __forceinline__ void oz_store_digits(const int (&a)[OZ_S], __nv_bfloat16* out, long long slice_stride) {
  const float scale[OZ_S] = {1.0f, 0.0078125f, 6.103515625e-05f, 4.76837158203125e-07f, 3.7252902984619141e-09f,
                             2.9103830456733704e-11f, 2.2737367544323206e-13f};  // 2^-7t, exact
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) out[s * slice_stride] = __float2bfloat16_rn(__int2float_rn(a[s]) * scale[s]);
}

// bf16 bit pattern of slice s of a digit: a 2^-7s (exact)
__device__ __forceinline__ uint32_t oz_digit_bits(int a, int s) {
  const float scale[OZ_S] = {1.0f, 0.0078125f, 6.103515625e-05f, 4.76837158203125e-07f, 3.7252902984619141e-09f,
                             2.9103830456733704e-11f, 2.2737367544323206e-13f};  // 2^-7t, exact
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(__int2float_rn(a) * scale[s]));
}

// q 2^e as the nearest double (ties to even), built in integer arithmetic
// (GB300's FP64 units, which the int64 -> double conversion uses, issue about
// two operations per clock per SM); |q| < 2^63; results below the normal
// range give 0
__device__ __forceinline__ double oz_i64_scaled(long long q, int e) {
  if (q == 0) return 0.0;
  unsigned long long u = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  const int lz = __clzll((long long)u);
  u <<= lz;  // leading one at bit 63
  unsigned long long mant = u >> 11;  // 53 bits with the leading one
  const unsigned long long rem = u & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  int ex = 63 - lz + e;  // q 2^e = mant 2^(ex - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const int biased = ex + 1023;
  if (biased <= 0) return 0.0;
  unsigned long long bits = biased >= 2047 ? 0x7FF0000000000000ull
                                           : ((unsigned long long)biased << 52) | (mant & 0xFFFFFFFFFFFFFull);
  if (q < 0) bits |= 1ull << 63;
  return __longlong_as_double((long long)bits);
}

// exponent field of |x|: frexp exponent = field - 1022 for normal x (0 for zero)
__device__ __forceinline__ int oz_exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

}  // namespace iscsi
