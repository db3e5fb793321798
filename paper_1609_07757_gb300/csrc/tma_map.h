// tma_map.h -- host-side TMA descriptors for the bf16 slice arrays read by the
// tensor-core contraction (ozaki.cuh).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace iscsi {

// Descriptor of a K-major slice array [nslice][rows][ld] (bf16, slice_elems
// elements between slices) read in boxes of 16 (K) x box_rows x box_slices
// (default: all slices) with the 32-byte swizzle, the layout smem_desc_sw32
// describes to the MMA.  base must be 16-byte aligned and ld a multiple of 16.
// Returns 0 on success, -1 when the driver entry point is missing or rejects
// the shape.
inline int oz_encode_map(CUtensorMap* map, const void* base, int ld, long long rows, int nslice,
                         long long slice_elems, int box_rows, int box_slices = 0) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)nslice};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)slice_elems * 2};
  cuuint32_t box[3] = {16, (cuuint32_t)box_rows, (cuuint32_t)(box_slices > 0 ? box_slices : nslice)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

}  // namespace iscsi
