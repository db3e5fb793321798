// tc32.cuh -- the arithmetic of the FP32 form of the sigma step on the bf16
// tensor cores: operand terms and their slicing (the contraction kernel is
// k_tc32w_gemm in tc32w.cuh).
//
// Every operand element x (FP32 or FP64) is split into three bf16 terms
//   x_0 = bf16(x),  x_1 = bf16(x - x_0),  x_2 = bf16(x - x_0 - x_1)
// (each rounding keeps 8 significant bits, the residuals are exact in the
// input type, so |x - x_0 - x_1 - x_2| <= 2^-27 |x|).  The product keeps the
// six term pairs of order t + u <= 2,
//   T = sum_k sum_{t+u<=2} A_t B_u + O(2^-24 sum_k |A||B|),
// accumulated in FP32 in tensor memory over K chunks of 512 and across
// chunks in FP32 registers with round-to-nearest (the tensor core's own
// FP32 accumulation is not round-to-nearest, so it only ever sums one chunk).
#pragma once
#include <cuda_bf16.h>

#include "ozaki_types.cuh"
#include "tc_ptx.cuh"

namespace iscsi {

constexpr int T3_S = 3;             // bf16 terms per element
constexpr int T3_BM = 128, T3_BK = 16;
constexpr int T3_A_SLICE_BYTES = T3_BM * T3_BK * 2;  // 4096
constexpr int T3_CHUNK_STEPS = 32;  // K = 512 per tensor-memory chunk

// the three bf16 terms of x, slice s at out[s * slice_stride]
template <typename V>
__device__ __forceinline__ void t3_store_terms(V x, __nv_bfloat16* out, long long slice_stride) {
  __nv_bfloat16 h0 = __float2bfloat16_rn((float)x);
  V r = x - (V)__bfloat162float(h0);
  __nv_bfloat16 h1 = __float2bfloat16_rn((float)r);
  r -= (V)__bfloat162float(h1);
  __nv_bfloat16 h2 = __float2bfloat16_rn((float)r);
  out[0] = h0;
  out[slice_stride] = h1;
  out[2 * slice_stride] = h2;
}

// terms of X into out[s][row][k] (row stride ldo, rows_pad rows, zero padded).
// Source column of k: colmap[k] (-1: zero) if colmap, else k (zero beyond cols).
template <typename V>
__global__ void k_t3_slice(const V* __restrict__ X, int rows, int cols, long long ld, int trans,
                           const int* __restrict__ colmap, __nv_bfloat16* __restrict__ out, long long slice_stride,
                           int ldo, int rows_pad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)rows_pad * ldo;
  if (t >= total) return;
  int r = (int)(t / ldo), k = (int)(t % ldo);
  int src = colmap ? colmap[k] : (k < cols ? k : -1);
  V x = (V)0;
  if (r < rows && src >= 0) x = trans ? X[(long long)src * ld + r] : X[(long long)r * ld + src];
  t3_store_terms<V>(x, out + t, slice_stride);
}

}  // namespace iscsi
