// TMA tensor maps of low-precision (BF16 / FP32-for-TF32) matrices.
#pragma once

#include <cuda.h>

namespace spx {

// Encode a 2-D row-major matrix (rows x cols, leading dimension ld elements,
// dtype SPX_DT_BF16 or SPX_DT_F32) with a box of 128 rows x 128 bytes and the
// 128-byte swizzle that the tcgen05 operand layout expects.  Out-of-range
// boxes read zeros.  Returns SPX_OK, SPX_ERR_INVALID_ARG (alignment: base
// 16 bytes, ld * element size a multiple of 16) or SPX_ERR_CUDA.
int make_tmap(CUtensorMap* out, const void* ptr, int rows, int cols, int ld, int dtype);

}  // namespace spx
