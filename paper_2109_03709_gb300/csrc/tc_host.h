// tc_host.h -- host helpers shared by the tensor-core passes (internal).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace ppca {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

// 2-D tiled tensor map: `inner` contiguous elements per row, `outer` rows
// `pitch_bytes` apart, box `box_inner` x `box_outer`, zero fill out of range.
bool encode_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
               uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz);
bool encode_bf16_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch_bytes,
                    uint32_t box_inner, uint32_t box_outer);

// V (d x m column-major FP32) -> S in {1, 2, 3} BF16 pieces, [S][m_pad][ldv], zero padded;
// piece p holds the rounding of what pieces 0..p-1 left over.
cudaError_t launch_split_v(const float* V, int64_t d, int m, int m_pad, int64_t ldv, int S, __nv_bfloat16* Vp,
                           cudaStream_t st);

}  // namespace ppca
