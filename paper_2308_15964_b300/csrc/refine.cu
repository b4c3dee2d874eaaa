// FP64 kernels of iterative refinement for the mixed-precision Cholesky:
// the residual R = B - A X with per-column norms and the normwise backward
// error eta_j = ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf)
// (Rigal-Gaches), the infinity norm of A, and the update X += alpha D.  The
// residual reads A once (8 n^2 bytes) and does 2 n^2 nrhs flops; with 8
// right-hand sides that is 2 flop per byte, above the B300's FP64 ridge, so
// it runs on the DFMA pipe: each CTA owns 8 x rows-per-warp rows, stages
// 128-column slices of X in shared memory, and each warp accumulates
// rows-per-warp x nrhs sums in registers.
//
// The compensated form accumulates every row with Dot2 (Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005): each
// product is split exactly into p + q by TwoProduct (q = fma(a, x, -p)), each
// addition into t + e by Knuth's TwoSum, and the errors q + e are summed
// apart; lanes and the right-hand side b are combined by TwoSum as well.  The
// result is as accurate as if computed in twice the working precision and
// then rounded: |r - r_computed| <= u |r| + gamma_n^2 (|A||x| + |b|), so the
// eta it gives bounds the backward error of X to within a relative O(u) (the
// plain FP64 residual can be off by gamma_n (|A||x| + |b|), which is of the
// order of eta itself once refinement has converged).  It costs about ten
// FP64 operations per term instead of one FMA.  The error-free
// transformations use the _rn intrinsics, which the compiler never contracts
// into FMAs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx.h"

namespace {

// rows per warp: 8 x NR accumulators at most, and small CTAs for wide
// right-hand sides, so that the grid has many more CTAs than the GPU holds at
// once (with 64-row CTAs, n = 32768 gave 512 CTAs of about one per SM: the
// last of ~3.5 waves ran half empty)
template <int NR>
constexpr int rows_per_warp() { return NR >= 16 ? 1 : (NR >= 8 ? 2 : (NR >= 4 ? 4 : 8)); }
constexpr int kColSlice = 128;   // columns of X staged per step
constexpr int kMaxRhs = 16;

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)p, (unsigned long long)__double_as_longlong(v));
}

// Error-free transformations (Knuth TwoSum; TwoProduct with an FMA).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double z = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, z)), __dsub_rn(b, z));
}

// (s, c) += a * x with Dot2: the running sum s and the summed errors c.
__device__ __forceinline__ void dot2_step(double& s, double& c, double a, double x) {
  const double p = __dmul_rn(a, x);
  const double q = __fma_rn(a, x, -p);
  double t, e;
  two_sum(s, p, t, e);
  s = t;
  c = __dadd_rn(c, __dadd_rn(q, e));
}

// Combine two Dot2 partial results (s, c) += (s2, c2).
__device__ __forceinline__ void dot2_merge(double& s, double& c, double s2, double c2) {
  double t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __dadd_rn(c, __dadd_rn(c2, e));
}

template <int NR, bool kComp>
__global__ void __launch_bounds__(256) residual_kernel(const double* __restrict__ A, int n, int lda,
                                                       const double* __restrict__ X, int ldx,
                                                       const double* __restrict__ B, int ldb,
                                                       double* __restrict__ R, int ldr,
                                                       int nrhs, double* norms) {
  __shared__ double xs[kColSlice][NR];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int RPW = rows_per_warp<NR>();
  const int row0 = (blockIdx.x * 8 + warp) * RPW;
  double acc[RPW][NR];
  double cmp[kComp ? RPW : 1][kComp ? NR : 1];
#pragma unroll
  for (int i = 0; i < RPW; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      acc[i][j] = 0.0;
      if (kComp) cmp[kComp ? i : 0][kComp ? j : 0] = 0.0;
    }
  for (int c0 = 0; c0 < n; c0 += kColSlice) {
    const int w = min(kColSlice, n - c0);
    for (int e = threadIdx.x; e < kColSlice * NR; e += blockDim.x) {
      const int c = e / NR, j = e % NR;
      xs[c][j] = (c < w && j < nrhs) ? X[(size_t)(c0 + c) * ldx + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const int r = row0 + i;
      if (r >= n) break;
      const double* a = A + (size_t)r * lda + c0;
#pragma unroll
      for (int cc = lane; cc < kColSlice; cc += 32) {
        const double av = cc < w ? __ldcs(a + cc) : 0.0;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (kComp) dot2_step(acc[i][j], cmp[kComp ? i : 0][kComp ? j : 0], av, xs[cc][j]);
          else acc[i][j] = fma(av, xs[cc][j], acc[i][j]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = row0 + i;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      double v = acc[i][j];
      double rv = 0.0;
      if (kComp) {
        double c = cmp[kComp ? i : 0][kComp ? j : 0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
          const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
          dot2_merge(v, c, v2, c2);
        }
        if (lane == 0 && r < n && j < nrhs) {
          // r = b - (v + c): TwoSum(b, -v), then the errors
          double t, e;
          two_sum(B[(size_t)r * ldb + j], -v, t, e);
          rv = __dadd_rn(t, __dsub_rn(e, c));
        }
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && r < n && j < nrhs) rv = B[(size_t)r * ldb + j] - v;
      }
      if (lane == 0 && r < n && j < nrhs) {
        R[(size_t)r * ldr + j] = rv;
        atomic_max_nonneg(norms + j, fabs(rv));
        atomic_max_nonneg(norms + nrhs + j, fabs(X[(size_t)r * ldx + j]));
        atomic_max_nonneg(norms + 2 * nrhs + j, fabs(B[(size_t)r * ldb + j]));
      }
    }
  }
}

// eta_j = max|r_j| / (||A||_inf max|x_j| + max|b_j|) for each right-hand
// side, and their maximum at eta[nrhs].  One warp.
__global__ void eta_kernel(const double* __restrict__ norms, const double* __restrict__ anorm,
                           int nrhs, double* __restrict__ eta) {
  const int lane = threadIdx.x;
  double e = 0.0;
  if (lane < nrhs) {
    const double den = anorm[0] * norms[nrhs + lane] + norms[2 * nrhs + lane];
    e = den > 0.0 ? norms[lane] / den : (norms[lane] > 0.0 ? INFINITY : 0.0);
    eta[lane] = e;
  }
  for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) eta[nrhs] = e;
}

__global__ void norm_inf_kernel(const double* __restrict__ A, int n, int lda, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* a = A + (size_t)warp * lda;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += fabs(__ldcs(a + c));
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomic_max_nonneg(out, s);
}

__global__ void axpy_kernel(double* __restrict__ Y, const double* __restrict__ X, long long count,
                            double alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    Y[i] = fma(alpha, X[i], Y[i]);
}

template <int NR, bool kComp>
cudaError_t launch_residual(const double* A, int n, int lda, const double* X, int ldx,
                            const double* B, int ldb, double* R, int ldr, int nrhs,
                            double* norms, cudaStream_t st) {
  constexpr int rows = 8 * rows_per_warp<NR>();
  residual_kernel<NR, kComp><<<(n + rows - 1) / rows, 256, 0, st>>>(A, n, lda, X, ldx, B, ldb,
                                                                       R, ldr, nrhs, norms);
  return cudaGetLastError();
}

template <bool kComp>
cudaError_t residual_dispatch(const double* A, int n, int lda, const double* X, int ldx,
                              const double* B, int ldb, double* R, int ldr, int nrhs,
                              double* norms, cudaStream_t st) {
  // norms: max|r_j| at [j], max|x_j| at [nrhs + j], max|b_j| at [2 nrhs + j]
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 3 * nrhs, st);
  if (e != cudaSuccess) return e;
  const int nr = nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16;
  switch (nr) {
    case 1: return launch_residual<1, kComp>(A, n, lda, X, ldx, B, ldb, R, ldr, nrhs, norms, st);
    case 2: return launch_residual<2, kComp>(A, n, lda, X, ldx, B, ldb, R, ldr, nrhs, norms, st);
    case 4: return launch_residual<4, kComp>(A, n, lda, X, ldx, B, ldb, R, ldr, nrhs, norms, st);
    case 8: return launch_residual<8, kComp>(A, n, lda, X, ldx, B, ldb, R, ldr, nrhs, norms, st);
    default: return launch_residual<16, kComp>(A, n, lda, X, ldx, B, ldb, R, ldr, nrhs, norms, st);
  }
}

bool residual_args_ok(const double* A, int n, int lda, const double* X, int ldx, const double* B,
                      int ldb, const double* R, int ldr, int nrhs, const double* norms) {
  return A && X && B && R && norms && n >= 1 && lda >= n && nrhs >= 1 && nrhs <= kMaxRhs &&
         ldx >= nrhs && ldb >= nrhs && ldr >= nrhs;
}

}  // namespace

extern "C" int spx_residual_f64(const double* dev_A, int n, int lda, const double* dev_X, int ldx,
                                const double* dev_B, int ldb, double* dev_R, int ldr, int nrhs,
                                double* dev_norms, void* stream) {
  if (!residual_args_ok(dev_A, n, lda, dev_X, ldx, dev_B, ldb, dev_R, ldr, nrhs, dev_norms))
    return SPX_ERR_INVALID_ARG;
  const cudaError_t e = residual_dispatch<false>(dev_A, n, lda, dev_X, ldx, dev_B, ldb, dev_R, ldr,
                                                 nrhs, dev_norms, (cudaStream_t)stream);
  return e == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}

extern "C" int spx_residual_eta_f64(const double* dev_A, int n, int lda, const double* dev_X,
                                    int ldx, const double* dev_B, int ldb, double* dev_R, int ldr,
                                    int nrhs, const double* dev_anorm, double* dev_norms,
                                    double* dev_eta, int compensated, void* stream) {
  if (!residual_args_ok(dev_A, n, lda, dev_X, ldx, dev_B, ldb, dev_R, ldr, nrhs, dev_norms) ||
      !dev_anorm || !dev_eta || (compensated != 0 && compensated != 1))
    return SPX_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = compensated
                      ? residual_dispatch<true>(dev_A, n, lda, dev_X, ldx, dev_B, ldb, dev_R, ldr,
                                                nrhs, dev_norms, st)
                      : residual_dispatch<false>(dev_A, n, lda, dev_X, ldx, dev_B, ldb, dev_R, ldr,
                                                 nrhs, dev_norms, st);
  if (e == cudaSuccess) {
    eta_kernel<<<1, 32, 0, st>>>(dev_norms, dev_anorm, nrhs, dev_eta);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}

extern "C" int spx_norm_inf_f64(const double* dev_A, int n, int lda, double* dev_out, void* stream) {
  if (!dev_A || !dev_out || n < 1 || lda < n) return SPX_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_out, 0, sizeof(double), st) != cudaSuccess) return SPX_ERR_CUDA;
  norm_inf_kernel<<<(n + 7) / 8, 256, 0, st>>>(dev_A, n, lda, dev_out);
  return cudaGetLastError() == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}

extern "C" int spx_axpy_f64(double* dev_Y, const double* dev_X, long long count, double alpha,
                            void* stream) {
  if (!dev_Y || !dev_X || count < 0) return SPX_ERR_INVALID_ARG;
  if (count == 0) return SPX_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (count + 255) / 256;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  axpy_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(dev_Y, dev_X, count, alpha);
  return cudaGetLastError() == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}

extern "C" int spx_copy2d(void* dst, size_t dpitch, const void* src, size_t spitch,
                          size_t width_bytes, size_t rows, void* stream) {
  if (!dst || !src || dpitch < width_bytes || spitch < width_bytes) return SPX_ERR_INVALID_ARG;
  if (!rows || !width_bytes) return SPX_OK;
  const cudaError_t e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width_bytes, rows,
                                          cudaMemcpyDefault, (cudaStream_t)stream);
  return e == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}
