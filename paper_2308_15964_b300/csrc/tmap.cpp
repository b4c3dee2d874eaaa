// Tensor-map encoding through the driver entry point (no link-time
// dependency on libcuda).
#include "tmap.h"

#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "spx.h"

namespace spx {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

}  // namespace

int make_tmap(CUtensorMap* out, const void* ptr, int rows, int cols, int ld, int dtype) {
  if (!out || !ptr || rows < 1 || cols < 1 || ld < cols) return SPX_ERR_INVALID_ARG;
  const int elem = dtype == SPX_DT_BF16 ? 2 : (dtype == SPX_DT_F32 ? 4 : 0);
  if (!elem) return SPX_ERR_INVALID_ARG;
  if (((uintptr_t)ptr & 15) || ((size_t)ld * elem) % 16) return SPX_ERR_INVALID_ARG;
  std::call_once(g_encode_once, load_encode);
  if (!g_encode) return SPX_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * elem};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / elem), 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(out, dtype == SPX_DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              2, const_cast<void*>(ptr), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SPX_OK : SPX_ERR_CUDA;
}

long long ozaki_slot_bytes(int b) {
  if (b < 32 || b > 512 || b % 32) return 0;
  const long long raw = 16ll * b * b + 4ll * b;
  return (raw + 255) / 256 * 256;
}

int make_tmap_ozaki(CUtensorMap* out, const void* ptr, int nslots, int b, int box_rows) {
  const long long slot = ozaki_slot_bytes(b);
  if (!out || !ptr || nslots < 1 || !slot || ((uintptr_t)ptr & 255) ||
      (box_rows != 128 && box_rows != 64 && box_rows != 32))
    return SPX_ERR_INVALID_ARG;
  std::call_once(g_encode_once, load_encode);
  if (!g_encode) return SPX_ERR_CUDA;
  // dims: digit within a 16-digit K chunk, row, K chunk, digit plane, slot
  const cuuint64_t dims[5] = {16, (cuuint64_t)b, (cuuint64_t)b / 16, 8, (cuuint64_t)nslots};
  const cuuint64_t strides[4] = {32, (cuuint64_t)b * 32, (cuuint64_t)b * b * 2, (cuuint64_t)slot};
  const cuuint32_t box[5] = {16, (cuuint32_t)box_rows, 1, 8, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(ptr),
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SPX_OK : SPX_ERR_CUDA;
}

}  // namespace spx
