// Tensor maps (TMA descriptors) over the batch's X for the tcgen05 streaming
// kernels, shared by the mode-P and mode-Q launch sequences.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <stdint.h>

namespace dash {

// cuTensorMapEncodeTiled from the driver, looked up once (no link against
// libcuda); null if the driver does not provide it.
inline PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor map of the rows [0, rows) of a row-major FP32 matrix with J columns
// (16-byte aligned base, J % 4 == 0), boxes of box_x columns × box_y rows,
// zero fill past the edges: 32 × 128 with the 128-byte swizzle for the X·Q_V
// pass, 128 × 32 unswizzled for the F pass.  False if the driver refuses it.
inline bool x_tensor_map(CUtensorMap *map, const float *base, int J, int64_t rows, int box_x, int box_y,
                         bool swizzle) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || rows <= 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || (J % 4) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)J, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)J * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace dash
