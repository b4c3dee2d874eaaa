// Stand-alone form of the low-precision tensor-core tile update (the
// building block of the mixed-precision SYRK / GEMM tasks), C -= A_lo B_lo^T
// in 128 x 128 units: tc_gemm_kernel runs tc_gemm_unit (the persistent
// kernel's unit) per CTA; tc_gemm_pipe_kernel, the form the entry point
// launches, overlaps the epilogue of a unit with the next units' loads and
// MMAs.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx.h"
#include "spx_internal.h"
#include "tile_tc.cuh"
#include "tmap.h"

namespace spx {
namespace {

__device__ __forceinline__ int ld_volatile_i(const int* p) { return *(const volatile int*)p; }

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

// Pipelined form for the stand-alone update (one CTA of 16 warps per SM,
// persistent over its units): warp 0 lane 0 loads operand chunks by TMA into
// kPipeStages stages; warp 1 lane 0 issues the MMAs of unit i into
// accumulator i mod 2 (two 128-column TMEM accumulators); warps 4-7 read a
// finished accumulator 32 columns at a time into shared memory (a warp reads
// its own 32 TMEM lanes) and release it, and warps 2-15 subtract each
// 32-column slice from the FP64 output block (coalesced rows; each thread's
// loads of a slice are issued before it waits for the staged accumulator) and
// pull the next unit's block into L2.  The FP64 read-modify-write of the
// output is the bound (a probe of the same access pattern on this GPU: 2.0
// TB/s without the L2 prefetch, 4.2 with it at 6 warps, 4.8 at 16 warps).
// So the epilogue of unit i, bound by HBM and the FP64 pipe, overlaps the
// loads and MMAs of units i + 1 and i + 2.  Barriers: full / empty per stage
// (TMA landed / MMAs done), acc_full / acc_empty per accumulator.  Every
// wait is bounded; on a timeout the CTA sets *err and every role leaves its
// loop at its next check.
// Five stages (160 KB of operands in flight: the operand stream from L2 is
// bound by bytes in flight over the TMA latency) and a 32-column staging
// slice of the accumulator.
constexpr int kPipeStages = 5;
constexpr int kPipeThreads = 512;  // 16 warps
constexpr int kEpiThreads = kPipeThreads - 64;  // warps 2-15
constexpr int kSlice = 32;        // accumulator columns staged at a time
constexpr int kSliceElems = (kTcM * kSlice + kEpiThreads - 1) / kEpiThreads;  // per thread
struct __align__(1024) PipeBuf {
  uint8_t a[kPipeStages][kTcStageBytes];
  uint8_t b[kPipeStages][kTcStageBytes];
  float e[kTcM][kSlice + 1];  // one 32-column slice of the accumulator
};

__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <bool kBf16>
__global__ void __launch_bounds__(kPipeThreads, 1)
    tc_gemm_pipe_kernel(const __grid_constant__ CUtensorMap amap,
                        const __grid_constant__ CUtensorMap bmap, double* C, int ldc, int m, int n,
                        int K, int* err) {
  extern __shared__ __align__(16) uint8_t raw[];
  PipeBuf& buf = *reinterpret_cast<PipeBuf*>(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[kPipeStages], empty[kPipeStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_err, s_stop;
  constexpr int kElem = kBf16 ? 2 : 4;
  constexpr int kChunk = kTcChunkBytes / kElem;
  constexpr int kMmaK = kBf16 ? 16 : 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(2 * kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kPipeStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // one arrival per reading warp
    }
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int nbc = (n + kTcN - 1) / kTcN;
  const int units = ((m + kTcM - 1) / kTcM) * nbc;
  const int nchunks = (K + kChunk - 1) / kChunk;
  auto fail = [&]() {
    s_err = 1;
    atomicExch(err, 1);
  };
  if (warp == 0 && lane == 0) {  // TMA producer
    uint32_t it = 0;
    for (int u = blockIdx.x; u < units && !ld_volatile_i(&s_err); u += gridDim.x) {
      const int r0 = (u / nbc) * kTcM, c0 = (u % nbc) * kTcN;
      for (int c = 0; c < nchunks; ++c, ++it) {
        const uint32_t st = it % kPipeStages, use = it / kPipeStages;
        if (use >= 1 && !mbar_wait(&empty[st], (use - 1) & 1u)) {
          fail();
          break;
        }
        mbar_arrive_expect_tx(&full[st], 2 * kTcStageBytes);
        tma_load_2d(buf.a[st], &amap, &full[st], c * kChunk, r0);
        tma_load_2d(buf.b[st], &bmap, &full[st], c * kChunk, c0);
      }
    }
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    uint32_t it = 0, ui = 0;
    for (int u = blockIdx.x; u < units && !ld_volatile_i(&s_err); u += gridDim.x, ++ui) {
      const uint32_t b = ui & 1u, use = ui >> 1;
      if (use >= 1 && !mbar_wait(&acc_empty[b], (use - 1) & 1u)) {
        fail();
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + b * kTcTmemCols;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++it) {
        const uint32_t st = it % kPipeStages;
        if (!mbar_wait(&full[st], (it / kPipeStages) & 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(buf.a[st]), b0 = smem_u32(buf.b[st]);
#pragma unroll
        for (int k = 0; k < kChunk / kMmaK; ++k)
          tc_mma<kBf16>(d, smem_desc(a0 + k * kMmaK * kElem), smem_desc(b0 + k * kMmaK * kElem),
                        (c > 0 || k > 0) ? 1u : 0u);
        tc_commit(&empty[st]);
      }
      if (!ok) {
        fail();
        break;
      }
      tc_commit(&acc_full[b]);
    }
  } else if (warp >= 2) {  // epilogue
    // The epilogue warps leave together: thread 64 copies the error flag
    // into s_stop before the first barrier of a slice and every warp reads
    // that copy between the slice's two barriers (the flag itself may change
    // at any time).
    const bool reader = warp >= 4 && warp < 8;  // one warp per TMEM lane quadrant
    const int q = warp & 3, ew = warp - 2;
    uint32_t ui = 0;
    int stop = 0;
    for (int u = blockIdx.x; u < units && !stop; u += gridDim.x, ++ui) {
      const uint32_t b = ui & 1u, use = ui >> 1;
      const int r0 = (u / nbc) * kTcM, c0 = (u % nbc) * kTcN;
      const int mb = min(kTcM, m - r0), nb = min(kTcN, n - c0);
      double* Cb = C + (size_t)r0 * ldc + c0;
      const int un = u + gridDim.x;  // the next unit's output block into L2
      if (un < units) {
        const int nr0 = (un / nbc) * kTcM, nc0 = (un % nbc) * kTcN;
        const int nmb = min(kTcM, m - nr0), lines = (min(kTcN, n - nc0) * 8 + 127) / 128;
        for (int e = tid - 64; e < nmb * lines; e += kEpiThreads)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (size_t)(nr0 + e / lines) * ldc + nc0 +
                                                         (e % lines) * 16));
      }
      int ok = 1;
      if (reader) {
        if (lane == 0) ok = mbar_wait(&acc_full[b], use & 1u) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) fail();
        tc_fence_after();
      }
      for (int cc = 0; cc < kTcN / kSlice; ++cc) {
        // this thread's elements of the slice: e = tid - 64 + kEpiThreads k,
        // row e / 32, column e mod 32 (a warp covers 32 consecutive doubles of
        // a row); their loads go out before the wait for the accumulator
        double cv[kSliceElems];
#pragma unroll
        for (int k = 0; k < kSliceElems; ++k) {
          const int e = tid - 64 + kEpiThreads * k, r = e / kSlice, c = kSlice * cc + e % kSlice;
          cv[k] = (e < kTcM * kSlice && r < mb && c < nb) ? __ldcg(Cb + (size_t)r * ldc + c) : 0.0;
        }
        if (reader && ok) {  // a warp's 32 TMEM lanes (rows), 32 columns
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * kTcTmemCols + (uint32_t)(kSlice * cc),
                    v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) buf.e[32 * q + lane][jj] = v[jj];
          if (cc == kTcN / kSlice - 1) {  // the accumulator is free again
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
          }
        }
        if (tid == 64) s_stop = ld_volatile_i(&s_err);
        named_bar(1, kEpiThreads);
        stop = *(volatile int*)&s_stop;
        if (stop) break;
#pragma unroll
        for (int k = 0; k < kSliceElems; ++k) {
          const int e = tid - 64 + kEpiThreads * k, r = e / kSlice, c = kSlice * cc + e % kSlice;
          if (e < kTcM * kSlice && r < mb && c < nb)
            Cb[(size_t)r * ldc + c] = cv[k] - widen_f32(buf.e[r][e % kSlice]);
        }
        named_bar(1, kEpiThreads);  // the slice buffer (and s_stop) are free
      }
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTcTmemCols));
  }
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
  const int grid = units < sms ? units : sms;  // one pipelined CTA per SM
  const size_t smem = sizeof(PipeBuf) + 1024;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == SPX_BF16) {
    cudaFuncSetAttribute(tc_gemm_pipe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    tc_gemm_pipe_kernel<true><<<grid, kPipeThreads, smem, st>>>(am, bm, dev_C, ldc, m, n, K,
                                                                dev_err);
  } else {
    cudaFuncSetAttribute(tc_gemm_pipe_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    tc_gemm_pipe_kernel<false><<<grid, kPipeThreads, smem, st>>>(am, bm, dev_C, ldc, m, n, K,
                                                                 dev_err);
  }
  return cudaGetLastError() == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}
