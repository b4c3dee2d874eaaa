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

// Bytes of one split slot of pitch b (eight BF16 digit planes of b x b, then
// b int32 row exponents, rounded up to 256); 0 for b not a multiple of 32 in
// [32, 512].
long long ozaki_slot_bytes(int b);

// Encode a store of nslots split slots at ptr (256-byte aligned) as a 5-D
// BF16 tensor (digit within a 16-digit K chunk, row, K chunk, plane, slot)
// with boxes of 16 digits x box_rows (128, 64 or 32) rows x one chunk x all 8
// planes and the 32-byte swizzle.
int make_tmap_ozaki(CUtensorMap* out, const void* ptr, int nslots, int b, int box_rows);

}  // namespace spx
