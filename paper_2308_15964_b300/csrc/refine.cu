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

// ---------------------------------------------------------------------------
// GMRES-based iterative refinement (Carson and Higham, "A new analysis of
// iterative refinement and its application to accurate solution of
// ill-conditioned sparse linear systems", SIAM J. Sci. Comput. 2017; and
// "Accelerating the solution of linear systems by iterative refinement in
// three precisions", 2018).  Each refinement step solves the correction
// equation A d = r with GMRES on the left-preconditioned system
// M^{-1} A d = M^{-1} r, M = L L^T the low-precision factor (applied by a
// solve graph the caller built), all in FP64, instead of applying M^{-1}
// once: the step then contracts the error even when kappa(A) u_factor is not
// small.  The nrhs right-hand sides run in lockstep (one Krylov space each,
// vectors stored as n x nrhs row-major blocks); orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2), the Hessenberg least-squares
// problem is kept triangular with Givens rotations, one thread per right-hand
// side.  The host only compares device-computed scalars with tolerances.
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaxGmres = 64;  // Krylov vectors per refinement step

// out[k * nrhs + c] = sum_i V_k[i][c] W[i][c], one CTA per k, fixed-order
// block reduction (deterministic).
__global__ void __launch_bounds__(256) block_dots_kernel(const double* __restrict__ V,
                                                         long long vstride,
                                                         const double* __restrict__ W, int n,
                                                         int nrhs, double* __restrict__ out) {
  __shared__ double red[256];
  const double* v = V + (size_t)blockIdx.x * vstride;
  double acc[kMaxRhs];
#pragma unroll
  for (int c = 0; c < kMaxRhs; ++c) acc[c] = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c)
      if (c < nrhs) acc[c] = fma(v[(size_t)i * nrhs + c], W[(size_t)i * nrhs + c], acc[c]);
  }
  for (int c = 0; c < nrhs; ++c) {
    red[threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)blockIdx.x * nrhs + c] = red[0];
    __syncthreads();
  }
}

// W[i][c] += scale * sum_k coef[k * nrhs + c] V_k[i][c]
__global__ void block_combine_kernel(double* __restrict__ W, const double* __restrict__ V,
                                     int nvec, long long vstride, const double* __restrict__ coef,
                                     double scale, long long len, int nrhs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % nrhs);
    double s = 0.0;
    for (int k = 0; k < nvec; ++k) s = fma(coef[(size_t)k * nrhs + c], V[(size_t)k * vstride + e], s);
    W[e] = fma(scale, s, W[e]);
  }
}

// Y[i][c] = X[i][c] * s[c]
__global__ void block_scale_kernel(double* __restrict__ Y, const double* __restrict__ X,
                                   const double* __restrict__ s, long long len, int nrhs) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    Y[e] = X[e] * s[e % nrhs];
}

// GMRES state of nrhs systems, m Krylov vectors at most, FP64, laid out
// field by field with the right-hand side fastest: H[(m+1) x m], cs[m], sn[m],
// g[m+1], beta, inv (1 / norm of the newest vector), res (relative residual
// estimate |g_{j+1}| / beta); resmax at the end.
struct GmresState {
  double *H, *cs, *sn, *g, *beta, *inv, *res, *resmax;
  __host__ __device__ static size_t doubles(int m, int nrhs) {
    return ((size_t)(m + 1) * m + 2 * (size_t)m + (m + 1) + 4) * nrhs + 1;
  }
  __host__ __device__ GmresState(double* base, int m, int nrhs) {
    H = base;
    cs = H + (size_t)(m + 1) * m * nrhs;
    sn = cs + (size_t)m * nrhs;
    g = sn + (size_t)m * nrhs;
    beta = g + (size_t)(m + 1) * nrhs;
    inv = beta + nrhs;
    res = inv + nrhs;
    resmax = res + nrhs;
  }
};

// Start: beta = ||r0||, g = beta e_1, inv = 1 / beta (0 for r0 = 0).  One warp.
__global__ void gmres_start_kernel(double* base, int m, int nrhs, const double* nrm2) {
  GmresState st(base, m, nrhs);
  const int c = threadIdx.x;
  double r = 0.0;
  if (c < nrhs) {
    const double b = sqrt(nrm2[c]);
    st.beta[c] = b;
    st.inv[c] = b > 0.0 ? 1.0 / b : 0.0;
    for (int k = 0; k <= m; ++k) st.g[(size_t)k * nrhs + c] = k == 0 ? b : 0.0;
    st.res[c] = r = b > 0.0 ? 1.0 : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if (c == 0) *st.resmax = r;
}

// Arnoldi step j: column j of H is h[0..j] (the Gram-Schmidt coefficients)
// and sqrt(hn2) (the norm of the orthogonalised vector); apply the earlier
// rotations, make the new one, update g and the residual estimate, and
// inv = 1 / H[j+1][j] for the next basis vector (0 on breakdown: the Krylov
// space holds the solution).  One warp.
__global__ void gmres_step_kernel(double* base, int m, int nrhs, int j, const double* h,
                                  const double* hn2) {
  GmresState st(base, m, nrhs);
  const int c = threadIdx.x;
  double r = 0.0;
  if (c < nrhs) {
    auto H = [&](int row) -> double& { return st.H[((size_t)row * m + j) * nrhs + c]; };
    for (int k = 0; k <= j; ++k) H(k) = h[(size_t)k * nrhs + c];
    const double hn = sqrt(hn2[c]);
    H(j + 1) = hn;
    for (int i = 0; i < j; ++i) {
      const double a = H(i), b = H(i + 1);
      const double cs = st.cs[(size_t)i * nrhs + c], sn = st.sn[(size_t)i * nrhs + c];
      H(i) = cs * a + sn * b;
      H(i + 1) = -sn * a + cs * b;
    }
    const double a = H(j), b = H(j + 1);
    const double rr = hypot(a, b);
    const double cs = rr > 0.0 ? a / rr : 1.0, sn = rr > 0.0 ? b / rr : 0.0;
    st.cs[(size_t)j * nrhs + c] = cs;
    st.sn[(size_t)j * nrhs + c] = sn;
    H(j) = rr;
    H(j + 1) = 0.0;
    const double gj = st.g[(size_t)j * nrhs + c];
    st.g[(size_t)j * nrhs + c] = cs * gj;
    st.g[(size_t)(j + 1) * nrhs + c] = -sn * gj;
    st.inv[c] = hn > 0.0 ? 1.0 / hn : 0.0;
    const double beta = st.beta[c];
    r = beta > 0.0 ? fabs(st.g[(size_t)(j + 1) * nrhs + c]) / beta : 0.0;
    st.res[c] = r;
  }
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if (c == 0) *st.resmax = r;
}

// y[0..j] = R^{-1} g[0..j], R the rotated (upper triangular) H.  One warp.
__global__ void gmres_backsolve_kernel(const double* base, int m, int nrhs, int j, double* y) {
  GmresState st(const_cast<double*>(base), m, nrhs);
  const int c = threadIdx.x;
  if (c >= nrhs) return;
  for (int k = j; k >= 0; --k) {
    double s = st.g[(size_t)k * nrhs + c];
    for (int l = k + 1; l <= j; ++l)
      s -= st.H[((size_t)k * m + l) * nrhs + c] * y[(size_t)l * nrhs + c];
    const double d = st.H[((size_t)k * m + k) * nrhs + c];
    y[(size_t)k * nrhs + c] = d != 0.0 ? s / d : 0.0;
  }
}

int grid_for(long long len) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long b = (len + 255) / 256;
  return (int)(b < 4LL * sms ? (b > 0 ? b : 1) : 4LL * sms);
}

// Host copy of one device double (the only data the driver reads back).
double read_scalar(const double* p, cudaStream_t st, cudaError_t* e) {
  double v = 0.0;
  *e = cudaMemcpyAsync(&v, p, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (*e == cudaSuccess) *e = cudaStreamSynchronize(st);
  return v;
}

// Apply the preconditioner: the caller's solve graph, in place on R.
int apply_precond(spx_graph_t g, cudaStream_t st) {
  int rc = spx_graph_reset(g);
  if (rc != SPX_OK && rc != SPX_ERR_STATE) return rc;
  rc = spx_graph_execute(g, st);
  if (rc != SPX_OK) return rc;
  int info = 0;
  return spx_graph_wait(g, 0, &info);
}

}  // namespace

extern "C" long long spx_gmres_ir_workspace(int n, int nrhs, int max_inner) {
  if (n < 1 || nrhs < 1 || nrhs > kMaxRhs || max_inner < 1 || max_inner > kMaxGmres) return -1;
  const long long vec = (long long)n * nrhs;
  // basis (max_inner + 1 vectors), zero block, coefficients (2 sets + norms),
  // y, GMRES state, ||A||, norms, eta
  return 8LL * ((max_inner + 1) * vec + vec + 3LL * (max_inner + 1) * nrhs +
                (long long)GmresState::doubles(max_inner, nrhs) + 1 + 3 * nrhs + nrhs + 1 + 64);
}

extern "C" int spx_gmres_ir(const double* dev_A, int n, int lda, const double* dev_B, double* dev_X,
                            int nrhs, spx_graph_t precond, double* dev_R, void* dev_work,
                            long long work_bytes, const spx_gmres_config_t* cfg,
                            spx_gmres_result_t* out, void* stream) {
  if (!dev_A || !dev_B || !dev_X || !precond || !dev_R || !dev_work || !out || n < 1 || lda < n ||
      nrhs < 1 || nrhs > kMaxRhs || dev_R == dev_X || dev_R == dev_B)
    return SPX_ERR_INVALID_ARG;
  spx_gmres_config_t c{};
  if (cfg) c = *cfg;
  const int m = c.max_inner > 0 ? c.max_inner : 30;
  const int maxo = c.max_outer > 0 ? c.max_outer : 20;
  const double itol = c.inner_tol > 0.0 ? c.inner_tol : 1e-10;
  const double tol = c.tol > 0.0 ? c.tol : 1e-14;
  if (m > kMaxGmres || work_bytes < spx_gmres_ir_workspace(n, nrhs, m)) return SPX_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long vec = (long long)n * nrhs;
  double* V = (double*)dev_work;                       // (m + 1) basis blocks
  double* Z = V + (size_t)(m + 1) * vec;               // zero block (B = 0: R = -A v)
  double* h = Z + vec;                                 // CGS coefficients, pass 1
  double* h2 = h + (size_t)(m + 1) * nrhs;             // pass 2
  double* y = h2 + (size_t)(m + 1) * nrhs;             // least-squares solution
  double* S = y + (size_t)(m + 1) * nrhs;              // GMRES state
  double* anorm = S + GmresState::doubles(m, nrhs);
  double* norms = anorm + 1;
  double* eta = norms + 3 * nrhs;
  const GmresState gs(S, m, nrhs);
  const int grid = grid_for(vec);
  cudaError_t e = cudaMemsetAsync(Z, 0, sizeof(double) * vec, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(anorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return SPX_ERR_CUDA;
  norm_inf_kernel<<<(n + 7) / 8, 256, 0, st>>>(dev_A, n, lda, anorm);
  *out = spx_gmres_result_t{};
  bool compensated = false;
  double prev = 0.0;
  int rc = SPX_OK;
  for (int it = 0;; ++it) {
    // residual and its backward error, as in classical refinement: plain
    // residuals until eta reaches tol (or stops falling), then compensated
    e = compensated ? residual_dispatch<true>(dev_A, n, lda, dev_X, nrhs, dev_B, nrhs, dev_R, nrhs,
                                              nrhs, norms, st)
                    : residual_dispatch<false>(dev_A, n, lda, dev_X, nrhs, dev_B, nrhs, dev_R,
                                               nrhs, nrhs, norms, st);
    if (e == cudaSuccess) eta_kernel<<<1, 32, 0, st>>>(norms, anorm, nrhs, eta);
    double et = read_scalar(eta + nrhs, st, &e);
    if (e != cudaSuccess) return SPX_ERR_CUDA;
    if (!compensated && (et <= tol || (it > 0 && et > 0.9 * prev))) {
      compensated = true;
      e = residual_dispatch<true>(dev_A, n, lda, dev_X, nrhs, dev_B, nrhs, dev_R, nrhs, nrhs,
                                  norms, st);
      if (e == cudaSuccess) eta_kernel<<<1, 32, 0, st>>>(norms, anorm, nrhs, eta);
      et = read_scalar(eta + nrhs, st, &e);
      if (e != cudaSuccess) return SPX_ERR_CUDA;
    }
    prev = et;
    out->eta = et;
    out->outer = it;
    if (compensated && et <= tol) {
      out->converged = 1;
      return SPX_OK;
    }
    if (it == maxo) return SPX_OK;
    // GMRES on M^{-1} A d = M^{-1} r, d = 0 to start; x += d at the end
    rc = apply_precond(precond, st);                    // R = M^{-1} r
    if (rc != SPX_OK) return rc;
    block_dots_kernel<<<1, 256, 0, st>>>(dev_R, vec, dev_R, n, nrhs, h);
    gmres_start_kernel<<<1, 32, 0, st>>>(S, m, nrhs, h);
    block_scale_kernel<<<grid, 256, 0, st>>>(V, dev_R, gs.inv, vec, nrhs);
    int j = 0;
    for (; j < m; ++j) {
      double* vj = V + (size_t)j * vec;
      // R = -A v_j (residual with B = 0), then R = A v_j, then M^{-1} A v_j
      e = residual_dispatch<false>(dev_A, n, lda, vj, nrhs, Z, nrhs, dev_R, nrhs, nrhs, norms, st);
      if (e != cudaSuccess) return SPX_ERR_CUDA;
      axpy_kernel<<<grid, 256, 0, st>>>(dev_R, dev_R, vec, -2.0);
      rc = apply_precond(precond, st);
      if (rc != SPX_OK) return rc;
      // CGS2 against v_0 .. v_j
      block_dots_kernel<<<j + 1, 256, 0, st>>>(V, vec, dev_R, n, nrhs, h);
      block_combine_kernel<<<grid, 256, 0, st>>>(dev_R, V, j + 1, vec, h, -1.0, vec, nrhs);
      block_dots_kernel<<<j + 1, 256, 0, st>>>(V, vec, dev_R, n, nrhs, h2);
      block_combine_kernel<<<grid, 256, 0, st>>>(dev_R, V, j + 1, vec, h2, -1.0, vec, nrhs);
      axpy_kernel<<<1, 256, 0, st>>>(h, h2, (long long)(j + 1) * nrhs, 1.0);
      block_dots_kernel<<<1, 256, 0, st>>>(dev_R, vec, dev_R, n, nrhs, h2);
      gmres_step_kernel<<<1, 32, 0, st>>>(S, m, nrhs, j, h, h2);
      if (j + 1 < m)
        block_scale_kernel<<<grid, 256, 0, st>>>(V + (size_t)(j + 1) * vec, dev_R, gs.inv, vec,
                                                 nrhs);
      const double r = read_scalar(gs.resmax, st, &e);
      if (e != cudaSuccess) return SPX_ERR_CUDA;
      ++out->inner;
      if (r <= itol) {
        ++j;
        break;
      }
    }
    if (j > m) j = m;
    // x += V y, y = R^{-1} g over the j vectors built
    gmres_backsolve_kernel<<<1, 32, 0, st>>>(S, m, nrhs, j - 1, y);
    block_combine_kernel<<<grid, 256, 0, st>>>(dev_X, V, j, vec, y, 1.0, vec, nrhs);
    if (cudaGetLastError() != cudaSuccess) return SPX_ERR_CUDA;
  }
}
