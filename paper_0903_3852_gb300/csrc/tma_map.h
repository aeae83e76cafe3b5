// tma_map.h -- host-side construction of TMA tensor maps (cuTensorMapEncodeTiled
// through the runtime's driver entry point), shared by the tensor-core paths.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <string>

#include "common.cuh"

namespace sde {

inline PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D BF16 tensor map over a row-major [rows][cols] array (cols contiguous,
// a multiple of 8 so that rows start 16-byte aligned), loaded in boxes of
// box_rows x 64 elements (one 128-byte swizzle row per tile row).
inline sde_status make_map_bf16(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int box_rows) {
  auto fn = tma_encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SDE_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    return SDE_ERR_CUDA;
  }
  return SDE_OK;
}

// Tensor map over `planes` stacked row-major [rows][cols] arrays of 4-byte
// words (cols contiguous, a multiple of 4), loaded without swizzling in
// boxes of box_rows x box_cols words of one plane (a 2D map when planes == 1).
inline sde_status make_map_w32(CUtensorMap *map, const void *base, int64_t planes, int64_t rows, int64_t cols,
                               int box_rows, int box_cols) {
  auto fn = tma_encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SDE_ERR_CUDA;
  }
  const cuuint32_t rank = planes > 1 ? 3 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 4, (cuuint64_t)(cols * rows) * 4};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    return SDE_ERR_CUDA;
  }
  return SDE_OK;
}

}  // namespace sde
