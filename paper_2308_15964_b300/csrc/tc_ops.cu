// Stand-alone form of the low-precision tensor-core tile update (the
// building block of the mixed-precision SYRK / GEMM tasks): a grid of CTAs,
// each running 128 x 128 units of C -= A_lo B_lo^T with tc_gemm_unit.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx.h"
#include "spx_internal.h"
#include "tile_tc.cuh"
#include "tmap.h"

namespace spx {
namespace {

template <bool kBf16>
__global__ void __launch_bounds__(kThreads, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                   double* C, int ldc, int m, int n, int K, int* err) {
  extern __shared__ __align__(16) uint8_t raw[];
  TcBuf& buf = *reinterpret_cast<TcBuf*>(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ TcState st;
  tc_setup(st);
  __syncthreads();
  const int nbc = (n + kTcN - 1) / kTcN;
  const int units = ((m + kTcM - 1) / kTcM) * nbc;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int r0 = (u / nbc) * kTcM, c0 = (u % nbc) * kTcN;
    const bool ok = tc_gemm_unit<kBf16>(st, buf, &amap, 0, r0, &bmap, 0, c0, K,
                                        C + (size_t)r0 * ldc + c0, ldc, min(kTcM, m - r0),
                                        min(kTcN, n - c0), false);
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      break;
    }
  }
  __syncthreads();
  tc_teardown(st);
}

}  // namespace
}  // namespace spx

extern "C" int spx_tc_gemm_nt(double* dev_C, int ldc, int m, int n, const void* dev_A, int lda,
                              const void* dev_B, int ldb, int K, int prec, int* dev_err,
                              void* stream) {
  using namespace spx;
  if (!dev_C || !dev_A || !dev_B || !dev_err || m < 1 || n < 1 || K < 1 || ldc < n || lda < K ||
      ldb < K || (prec != SPX_BF16 && prec != SPX_TF32))
    return SPX_ERR_INVALID_ARG;
  const int dt = prec == SPX_BF16 ? SPX_DT_BF16 : SPX_DT_F32;
  CUtensorMap am, bm;
  int rc = make_tmap(&am, dev_A, m, K, lda, dt);
  if (rc == SPX_OK) rc = make_tmap(&bm, dev_B, n, K, ldb, dt);
  if (rc != SPX_OK) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int units = ((m + kTcM - 1) / kTcM) * ((n + kTcN - 1) / kTcN);
  const int grid = units < 2 * sms ? units : 2 * sms;  // two CTAs per SM
  const size_t smem = sizeof(TcBuf) + 1024;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == SPX_BF16) {
    cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_gemm_kernel<true><<<grid, kThreads, smem, st>>>(am, bm, dev_C, ldc, m, n, K, dev_err);
  } else {
    cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_gemm_kernel<false><<<grid, kThreads, smem, st>>>(am, bm, dev_C, ldc, m, n, K, dev_err);
  }
  return cudaGetLastError() == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}
