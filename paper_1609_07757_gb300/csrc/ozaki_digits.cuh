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
#pragma unroll
  for (int t = OZ_S - 1; t >= 1; --t) {
    int r = (int)(N & 127);
    if (r >= 64) r -= 128;
    a[t] = r;
    N = (N - r) >> 7;
  }
  a[0] = (int)N;
}

__device__ __forceinline__ void oz_store_digits(const int (&a)[OZ_S], __nv_bfloat16* out, long long slice_stride) {
  const float scale[OZ_S] = {1.0f, 0.0078125f, 6.103515625e-05f, 4.76837158203125e-07f, 3.7252902984619141e-09f,
                             2.9103830456733704e-11f, 2.2737367544323206e-13f};  // 2^-7t, exact
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) out[s * slice_stride] = __float2bfloat16_rn(__int2float_rn(a[s]) * scale[s]);
}

// exponent field of |x|: frexp exponent = field - 1022 for normal x (0 for zero)
__device__ __forceinline__ int oz_exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

}  // namespace iscsi
