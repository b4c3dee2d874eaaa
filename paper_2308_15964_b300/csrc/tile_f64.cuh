// FP64 tile operations, run by all 256 threads of one CTA.
//
// These are the task kernels of the paper's tiled Cholesky (section
// "Numerical applications": POTRF, TRSM, SYRK, GEMM), of its tiled GEMM with
// dependencies on the blocks of C, and of the block triangular solves.  On
// the B300 the FP64 SIMT pipe (DFMA) is faster than FP64 mma.sync, and there is
// no FP64 kind of tcgen05.mma, so every FP64 op is a DFMA loop nest: 64x64
// output blocks, k staged through shared memory in chunks of 16, a 4x4
// register block per thread.  Data written by other tasks is read with
// ld.global.cg (L2), so a CTA never sees stale L1 lines of a tile that another
// SM updated.
#pragma once
#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.h"

namespace spx {
namespace {

constexpr int kKC = 16;        // k chunk staged in shared memory
constexpr int kLds = kBlk + 1; // padded row of a shared 64-wide array (doubles)

struct GemmSmem {
  double a[kKC][kLds];
  double b[kKC][kLds];
};

// Shared memory of the FP64 ops: GEMM staging plus two 64x64 blocks.
struct F64Smem {
  GemmSmem gs;
  double l[kBlk][kLds];   // diagonal block of L
  double x[kBlk][kLds];   // block being solved
  double rinv[kBlk];      // reciprocals of the diagonal of l
  int info;
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// C[0:m, 0:n] += alpha * op(A) op(B), m <= 16 RI, n <= 16 CJ, any K.
//   op(A)(i,k) = A_T ? A[k*lda + i] : A[i*lda + k]
//   op(B)(k,j) = B_KN ? B[k*ldb + j] : B[j*ldb + k]
// lower: only entries with column <= row are written (diagonal SYRK blocks).
// set: C = alpha op(A) op(B) instead of C += ... (products into a fresh tile).
// CJ / RI: output columns / rows per thread (4 / 4: a 64 x 64 block; CJ = 1:
// at most 16 columns, for right-hand-side blocks; RI = 1 or 2: 16- or
// 32-row blocks, for the finer parts of the POTRF and TRSM phases).
template <bool A_T, bool B_KN, int CJ = 4, int RI = 4>
__device__ void gemm_block(double* C, int ldc, const double* A, int lda, const double* B, int ldb,
                           int m, int n, int K, double alpha, bool lower, GemmSmem& s,
                           bool set = false, bool atomic = false) {
  constexpr int BN = 16 * CJ;  // columns of the block
  constexpr int BM = 16 * RI;  // rows of the block
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[RI][CJ];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kKC) {
#pragma unroll
    for (int e = tid; e < BM * kKC; e += kThreads) {
      int i, kk;
      if (A_T) { kk = e / BM; i = e % BM; } else { i = e / kKC; kk = e % kKC; }
      double v = 0.0;
      if (i < m && k0 + kk < K)
        v = ldcg(A_T ? A + (size_t)(k0 + kk) * lda + i : A + (size_t)i * lda + k0 + kk);
      s.a[kk][i] = v;
    }
#pragma unroll
    for (int e = tid; e < BN * kKC; e += kThreads) {
      int j, kk;
      if (B_KN) { kk = e / BN; j = e % BN; } else { j = e / kKC; kk = e % kKC; }
      double v = 0.0;
      if (j < n && k0 + kk < K)
        v = ldcg(B_KN ? B + (size_t)(k0 + kk) * ldb + j : B + (size_t)j * ldb + k0 + kk);
      s.b[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKC; ++kk) {
      double av[RI], bv[CJ];
#pragma unroll
      for (int i = 0; i < RI; ++i) av[i] = s.a[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < CJ; ++j) bv[j] = s.b[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int r = ty + 16 * i;
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int c = tx + 16 * j;
      if (r < m && c < n && (!lower || c <= r)) {
        double* p = C + (size_t)r * ldc + c;
        if (atomic) atomicAdd(p, alpha * acc[i][j]);  // ATOMIC_WRITE on C
        else *p = set ? alpha * acc[i][j] : __ldcg(p) + alpha * acc[i][j];
      }
    }
  }
  __syncthreads();
}

// Narrow right-hand-side blocks: C[0:m, 0:n] += alpha * op(A) B for m <= 16
// rows and n <= 16 columns, any K (B is K x n, row-major).  The 256 threads
// are 16 rows x BN columns x KS = 256 / (16 BN) slices of each 64-deep k
// chunk, so every lane of every FP64 instruction does useful work for
// BN = 2, 4, 8, 16; the slices are summed in a fixed order (deterministic).
// Element type E: double, or float for the FP32 correction solves.
constexpr int kNKC = 64;  // k chunk of a narrow block
template <typename E>
struct NarrowSmemT {
  E a[kNKC][kNarrowRows + 1];
  E b[kNKC][17];
  E red[kThreads];
};
using NarrowSmem = NarrowSmemT<double>;
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

template <bool A_T, int BN, typename E>
__device__ void gemm_narrow_bn(E* C, int ldc, const E* A, int lda, const E* B, int ldb, int m,
                               int n, int K, E alpha, NarrowSmemT<E>& s, bool set) {
  constexpr int KS = kThreads / (kNarrowRows * BN);
  const int tid = threadIdx.x, c = tid % BN, r = (tid / BN) % kNarrowRows,
            ks = tid / (kNarrowRows * BN);
  // The next k chunk is loaded into registers while the current one is
  // multiplied, so its load latency overlaps the barrier and the FMAs (the
  // per-thread summation order is unchanged).
  constexpr int kAE = kNarrowRows * kNKC / kThreads;          // A elements per thread
  constexpr int kBE = (BN * kNKC + kThreads - 1) / kThreads;  // B elements per thread
  static_assert(kAE * kThreads == kNarrowRows * kNKC, "A chunk split");
  E ra[kAE], rb[kBE];
  auto a_pos = [&](int e, int& i, int& kk) {
    if (A_T) { kk = e / kNarrowRows; i = e % kNarrowRows; } else { i = e / kNKC; kk = e % kNKC; }
  };
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < kAE; ++q) {
      int i, kk;
      a_pos(tid + q * kThreads, i, kk);
      ra[q] = (i < m && k0 + kk < K)
                  ? ldcg(A_T ? A + (size_t)(k0 + kk) * lda + i : A + (size_t)i * lda + k0 + kk)
                  : E(0);
    }
#pragma unroll
    for (int q = 0; q < kBE; ++q) {
      const int e = tid + q * kThreads, kk = e / BN, j = e % BN;
      rb[q] = (e < BN * kNKC && j < n && k0 + kk < K) ? ldcg(B + (size_t)(k0 + kk) * ldb + j)
                                                      : E(0);
    }
  };
  E acc0 = 0, acc1 = 0;
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += kNKC) {
#pragma unroll
    for (int q = 0; q < kAE; ++q) {
      int i, kk;
      a_pos(tid + q * kThreads, i, kk);
      s.a[kk][i] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < kBE; ++q) {
      const int e = tid + q * kThreads;
      if (e < BN * kNKC) s.b[e / BN][e % BN] = rb[q];
    }
    __syncthreads();
    if (k0 + kNKC < K) fetch(k0 + kNKC);
#pragma unroll
    for (int kk = ks; kk < kNKC; kk += 2 * KS) {
      acc0 = fma(s.a[kk][r], s.b[kk][c], acc0);
      acc1 = fma(s.a[kk + KS][r], s.b[kk + KS][c], acc1);
    }
    __syncthreads();
  }
  s.red[tid] = acc0 + acc1;
  __syncthreads();
  if (ks == 0) {
    E v = s.red[tid];
#pragma unroll
    for (int q = 1; q < KS; ++q) v += s.red[tid + q * kNarrowRows * BN];
    if (r < m && c < n) {
      E* p = C + (size_t)r * ldc + c;
      *p = set ? alpha * v : __ldcg(p) + alpha * v;
    }
  }
  __syncthreads();
}

template <bool A_T, typename E>
__device__ void gemm_narrow(E* C, int ldc, const E* A, int lda, const E* B, int ldb, int m, int n,
                            int K, E alpha, NarrowSmemT<E>& s, bool set = false) {
  if (n <= 2) gemm_narrow_bn<A_T, 2>(C, ldc, A, lda, B, ldb, m, n, K, alpha, s, set);
  else if (n <= 4) gemm_narrow_bn<A_T, 4>(C, ldc, A, lda, B, ldb, m, n, K, alpha, s, set);
  else if (n <= 8) gemm_narrow_bn<A_T, 8>(C, ldc, A, lda, B, ldb, m, n, K, alpha, s, set);
  else gemm_narrow_bn<A_T, 16>(C, ldc, A, lda, B, ldb, m, n, K, alpha, s, set);
}

// Copy an m x n block (row-major, ld) into a shared 64-wide array and back.
__device__ __forceinline__ void load_block(double (*dst)[kLds], const double* src, int ld, int m,
                                           int n) {
  for (int e = threadIdx.x; e < kBlk * kBlk; e += kThreads) {
    const int r = e / kBlk, c = e % kBlk;
    dst[r][c] = (r < m && c < n) ? __ldcg(src + (size_t)r * ld + c) : 0.0;
  }
}

// The first m rows only (m <= 64), for the 16-row units.
__device__ __forceinline__ void load_rows(double (*dst)[kLds], const double* src, int ld, int m,
                                          int n) {
  for (int e = threadIdx.x; e < m * kBlk; e += kThreads) {
    const int r = e / kBlk, c = e % kBlk;
    dst[r][c] = c < n ? __ldcg(src + (size_t)r * ld + c) : 0.0;
  }
}

__device__ __forceinline__ void store_rows(double* dst, int ld, const double (*src)[kLds], int m,
                                           int n) {
  for (int e = threadIdx.x; e < m * kBlk; e += kThreads) {
    const int r = e / kBlk, c = e % kBlk;
    if (c < n) dst[(size_t)r * ld + c] = src[r][c];
  }
}

__device__ __forceinline__ void store_block(double* dst, int ld, const double (*src)[kLds], int m,
                                            int n, bool lower) {
  for (int e = threadIdx.x; e < kBlk * kBlk; e += kThreads) {
    const int r = e / kBlk, c = e % kBlk;
    if (r < m && c < n && (!lower || c <= r)) dst[(size_t)r * ld + c] = src[r][c];
  }
}

// Unblocked right-looking Cholesky of the w x w block in shared memory
// (lower).  Returns 0 or the 1-based local column of a pivot that is not > 0
// (NaN included).  Every thread returns the same value.  The columns stay
// unscaled while the trailing matrix is updated (S_ic -= S_ij S_cj / S_jj,
// with the correctly rounded reciprocal of each pivot taken once), so the
// chain per column is one reciprocal (about 730 clocks) and two dependent
// FP64 operations instead of a square root and a division (about 2400); at
// the end l_jj = sqrt(S_jj) and l_ij = S_ij (1 / l_jj).
// `rc` and `sc` are w doubles of scratch each.  The FP64 pipe is shared
// by the SM (two FMAs a clock), so the trailing update competes with the
// pivot chain: warps 1..7 form the product -S_ij / S_jj of each row once
// (in sc, behind a barrier of their own) and spend one FMA per entry.
__device__ int potrf_smem(double (*a)[kLds], int w, int* s_info, double* rc, double* sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    const double d = a[0][0];
    *s_info = d > 0.0 ? 0 : 1;
    rc[0] = __drcp_rn(d);
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    if (*s_info) return *s_info;
    const double r = rc[j];
    // Trailing lower triangle (rows and columns j+1..w-1, column <= row).
    // Thread 0 alone updates the next pivot (j+1, j+1) and takes its
    // reciprocal, the chain of the factorization; warps 1..7 update the
    // rest, local row p paired with row t-1-p so that every pair holds t+1
    // entries and no lane idles on the upper half.
    const int t = w - j - 1;
    if (warp == 0) {
      if (lane == 0 && t > 0) {
        const double d = fma(-a[j + 1][j] * r, a[j + 1][j], a[j + 1][j + 1]);
        a[j + 1][j + 1] = d;
        if (d > 0.0) rc[j + 1] = __drcp_rn(d);
        else *s_info = j + 2;
      }
    } else if (t > 1) {  // rows j+2.. (row j+1's one entry is the pivot)
      for (int i = j + 2 + tid - 32; i < w; i += kThreads - 32) sc[i] = -a[i][j] * r;
      asm volatile("bar.sync 1, %0;" ::"n"(kThreads - 32) : "memory");
      for (int p = warp - 1; p < (t + 1) / 2; p += kThreads / 32 - 1) {
        const int ra = p, rb = t - 1 - p;
        const int na = ra + 1, nb = rb != ra ? rb + 1 : 0;
        for (int q = lane + (p == 0 ? 1 : 0); q < na + nb; q += 32) {
          const int rr = q < na ? ra : rb, cc = q < na ? q : q - na;
          const int i = j + 1 + rr, c = j + 1 + cc;
          a[i][c] = fma(sc[i], a[c][j], a[i][c]);
        }
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < w; j += kThreads) {
    const double sd = sqrt(a[j][j]);
    a[j][j] = sd;
    rc[j] = 1.0 / sd;
  }
  __syncthreads();
  for (int e = tid; e < w * w; e += kThreads) {
    const int i = e / w, c = e % w;
    if (i > c) a[i][c] *= rc[c];
  }
  __syncthreads();
  return 0;
}

// In-tile triangular solves.  On this GPU a dependent FP64 FMA takes about
// 128 clocks and a FP64 division about 1100, so the substitutions keep
// divisions and scalings off their dependency chains: prep_lower takes the
// reciprocals of the diagonal once and scales the strict lower part of L by
// them (by column for X L^-T and L^-1 X, by row for L^-T X); the solves then
// carry y_k = x_k l_kk (one FMA per step on the chain) and scale at the end.
// They run warp-synchronously (shuffles, no block barrier per step): X L^-T
// 16 rows at a time (rows are independent), L^-1 X and L^-T X of up to 32
// columns 16 columns at a time (columns are independent).

// l (w x w lower, shared memory): rinv[i] = 1 / l_ii; l_rc *= rinv[c] (by
// column) or rinv[r] (by row) for r > c.  Ends with a barrier.
__device__ void prep_lower(double (*l)[kLds], int w, double* rinv, bool by_row) {
  const int tid = threadIdx.x;
  for (int i = tid; i < w; i += kThreads) rinv[i] = 1.0 / l[i][i];
  __syncthreads();
  for (int e = tid; e < w * w; e += kThreads) {
    const int r = e / w, c = e % w;
    if (c < r) l[r][c] *= rinv[by_row ? r : c];
  }
  __syncthreads();
}

// X <- X L^{-T} for X (m x w) and L (w x w lower, scaled by column) in
// shared memory: y_c = x_c - sum_{k<c} y_k l~_ck, x_c = y_c / l_cc.  Rows
// are independent: 16 at a time, a half-warp per row, lane q holding
// columns q, q+16, q+32, q+48 (about 2x the FMA rate of a barrier per
// step over all rows).
__device__ void trsm_rt_smem(double (*x)[kLds], const double (*l)[kLds], const double* rinv,
                             int m, int w) {
  const int tid = threadIdx.x, q = tid & 15;
  for (int r0 = 0; r0 < m; r0 += 16) {
    const int r = r0 + (tid >> 4);
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = q + 16 * j < w ? x[r][q + 16 * j] : 0.0;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      for (int cl = 0; cl < 16; ++cl) {
        const int c = 16 * jj + cl;
        if (c >= w) break;
        const double yc = __shfl_sync(0xffffffffu, v[jj], cl, 16);
#pragma unroll
        for (int j = jj; j < 4; ++j) {
          const int cc = q + 16 * j;
          if (cc > c && cc < w) v[j] = fma(-yc, l[cc][c], v[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (q + 16 * j < w) x[r][q + 16 * j] = v[j] * rinv[q + 16 * j];
  }
  __syncthreads();
}

// X <- L^{-1} X (forward, L scaled by column) or X <- L^{-T} X (backward, L
// scaled by row) for L (m x m lower, m <= 64) and X (m x w) in shared
// memory.  Up to 32 columns: 16 at a time, a warp per column and the column
// 8 to its right, 2 rows per lane, shuffles instead of barriers (columns are
// independent).  Wider X: one barrier per step over all rows and columns,
// where the warp form would leave most lanes of the late steps idle.
template <bool kTrans>
__device__ void trsm_left_smem(double (*x)[kLds], const double (*l)[kLds], const double* rinv,
                               int m, int w) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (w > 32) {
    for (int s = 0; s + 1 < m; ++s) {
      const int i = kTrans ? m - 1 - s : s, t = m - 1 - s;  // rows still to update
#pragma unroll 4
      for (int e = tid; e < t * w; e += kThreads) {
        const int r = kTrans ? e / w : i + 1 + e / w, c = e % w;
        x[r][c] = fma(-(kTrans ? l[i][r] : l[r][i]), x[i][c], x[r][c]);
      }
      __syncthreads();
    }
    for (int e = tid; e < m * w; e += kThreads) x[e / w][e % w] *= rinv[e / w];
    __syncthreads();
    return;
  }
  for (int cb = 0; cb < w; cb += 16) {
    const int c0 = cb + warp, c1 = cb + warp + 8;
    const bool two = c1 < w;
    if (c0 < w) {
      double a0 = x[lane][c0], a1 = x[lane + 32][c0];
      double b0 = two ? x[lane][c1] : 0.0, b1 = two ? x[lane + 32][c1] : 0.0;
      for (int s = 0; s < m; ++s) {
        const int i = kTrans ? m - 1 - s : s;
        const double ya = __shfl_sync(0xffffffffu, i < 32 ? a0 : a1, i & 31);
        const double l0 = kTrans ? l[i][lane] : l[lane][i];
        const double l1 = kTrans ? l[i][lane + 32] : l[lane + 32][i];
        const bool u0 = kTrans ? lane < i : lane > i, u1 = kTrans ? lane + 32 < i : lane + 32 > i;
        if (u0) a0 = fma(-l0, ya, a0);
        if (u1) a1 = fma(-l1, ya, a1);
        if (two) {
          const double yb = __shfl_sync(0xffffffffu, i < 32 ? b0 : b1, i & 31);
          if (u0) b0 = fma(-l0, yb, b0);
          if (u1) b1 = fma(-l1, yb, b1);
        }
      }
      x[lane][c0] = a0 * rinv[lane];
      x[lane + 32][c0] = a1 * rinv[lane + 32];
      if (two) {
        x[lane][c1] = b0 * rinv[lane];
        x[lane + 32][c1] = b1 * rinv[lane + 32];
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Task ops.  u0..u1 is the range of work units of this part (see
// op_phase_units).
// ---------------------------------------------------------------------------

// Lower block pair (bi >= bj) of unit u in a triangle of blocks.
__device__ __forceinline__ void lower_pair(uint32_t u, int& bi, int& bj) {
  int i = 0;
  while ((uint32_t)((i + 1) * (i + 2) / 2) <= u) ++i;
  bi = i;
  bj = (int)(u - (uint32_t)(i * (i + 1) / 2));
}

// POTRF phase `phase`, units u0..u1 (see op_phase_units): right-looking
// over 64-column block steps j.  Returns 0 or the 1-based column (within the
// tile) of a pivot that is not > 0.
__device__ int op_potrf_units(const TileDesc& A, uint32_t phase, uint32_t u0, uint32_t u1,
                              F64Smem& s, bool fine) {
  double* a = (double*)A.ptr;
  const int n = A.rows, lda = A.ld;
  const int j = (int)(phase / 3), jb = j * kBlk, w = min(kBlk, n - jb);
  double* ajj = a + (size_t)jb * lda + jb;
  switch (phase % 3) {
    case 0: {  // factor the diagonal block
      load_block(s.l, ajj, lda, w, w);
      __syncthreads();
      const int info = potrf_smem(s.l, w, &s.info, s.rinv, &s.x[0][0]);
      if (info) return jb + info;
      store_block(ajj, lda, s.l, w, w, true);
      __syncthreads();
      return 0;
    }
    case 1: {  // row blocks below the diagonal block: X <- X L_jj^{-T}
      const int rb = fine ? 16 : kBlk;
      load_block(s.l, ajj, lda, w, w);
      __syncthreads();
      prep_lower(s.l, w, s.rinv, false);
      for (uint32_t u = u0; u < u1; ++u) {
        const int ib = jb + w + rb * (int)u, mb = min(rb, n - ib);
        load_rows(s.x, a + (size_t)ib * lda + jb, lda, mb, w);
        __syncthreads();
        trsm_rt_smem(s.x, s.l, s.rinv, mb, w);
        store_rows(a + (size_t)ib * lda + jb, lda, s.x, mb, w);
        __syncthreads();
      }
      return 0;
    }
    default: {  // trailing lower blocks (i, l), l <= i: A_il -= L_ij L_lj^T
      for (uint32_t u = u0; u < u1; ++u) {
        int bi, bl;
        lower_pair(u, bi, bl);
        if (fine) {
          const int ib = jb + w + 32 * bi, lb = jb + w + 32 * bl;
          gemm_block<false, false, 2, 2>(a + (size_t)ib * lda + lb, lda,
                                         a + (size_t)ib * lda + jb, lda,
                                         a + (size_t)lb * lda + jb, lda, min(32, n - ib),
                                         min(32, n - lb), w, -1.0, bi == bl, s.gs);
        } else {
          const int ib = jb + w + kBlk * bi, lb = jb + w + kBlk * bl;
          gemm_block<false, false>(a + (size_t)ib * lda + lb, lda, a + (size_t)ib * lda + jb,
                                   lda, a + (size_t)lb * lda + jb, lda, min(kBlk, n - ib),
                                   min(kBlk, n - lb), w, -1.0, bi == bl, s.gs);
        }
      }
      return 0;
    }
  }
}

// POTRF of P with the solve Q <- Q L^{-T} folded into its steps (one task on
// the critical path instead of two): in step j, after P's diagonal block is
// factored, Q's rows are solved with it beside P's rows below it, and Q's
// columns right of block j are updated beside P's trailing blocks.  Units of
// a phase: POTRF's own first, then Q's (row blocks, or row blocks x 64-column
// blocks); each Q unit is the TRSM op's unit of the same step, so the result
// is that of POTRF then TRSM.  Returns POTRF's info.
__device__ int op_potrf_panel_units(const TileDesc& P, const TileDesc& Q, uint32_t phase,
                                    uint32_t u0, uint32_t u1, F64Smem& s, bool fine) {
  const double* l = (const double*)P.ptr;
  double* a = (double*)Q.ptr;
  const int n = P.rows, m = Q.rows, lda = Q.ld, ldl = P.ld;
  // phases: POTRF's 3 nb - 2, then one more (j = nb - 1, phase % 3 == 1)
  // solving Q's last column block
  const int j = (int)(phase / 3), jb = j * kBlk, w = min(kBlk, n - jb);
  const int below = max(0, n - jb - w), rb = fine ? 16 : kBlk;
  if (phase % 3 == 0) return op_potrf_units(P, phase, u0, u1, s, fine);
  if (phase % 3 == 1) {
    const uint32_t np = fine ? cdiv16(below) : cdiv64(below);
    if (u0 < np) op_potrf_units(P, phase, u0, min(u1, np), s, fine);
    if (u1 <= np) return 0;
    load_block(s.l, l + (size_t)jb * ldl + jb, ldl, w, w);
    __syncthreads();
    prep_lower(s.l, w, s.rinv, false);
    for (uint32_t u = max(u0, np); u < u1; ++u) {
      const int ib = rb * (int)(u - np), mb = min(rb, m - ib);
      double* x = a + (size_t)ib * lda + jb;
      load_rows(s.x, x, lda, mb, w);
      __syncthreads();
      trsm_rt_smem(s.x, s.l, s.rinv, mb, w);
      store_rows(x, lda, s.x, mb, w);
      __syncthreads();
    }
    return 0;
  }
  const uint32_t q = fine ? cdiv32(below) : cdiv64(below), np = q * (q + 1) / 2;
  if (u0 < np) op_potrf_units(P, phase, u0, min(u1, np), s, fine);
  const uint32_t right = cdiv64(n) - 1 - (uint32_t)j;
  for (uint32_t u = max(u0, np); u < u1; ++u) {
    const uint32_t v = u - np;
    const int ib = rb * (int)(v / right), lb = (j + 1 + (int)(v % right)) * kBlk;
    double* c = a + (size_t)ib * lda + lb;
    const double* ap = a + (size_t)ib * lda + jb;
    const double* bp = l + (size_t)lb * ldl + jb;
    if (fine)
      gemm_block<false, false, 4, 1>(c, lda, ap, lda, bp, ldl, min(16, m - ib), min(kBlk, n - lb),
                                     w, -1.0, false, s.gs);
    else
      gemm_block<false, false>(c, lda, ap, lda, bp, ldl, min(kBlk, m - ib), min(kBlk, n - lb), w,
                               -1.0, false, s.gs);
  }
  return 0;
}

// TRSM phase `phase`, units u0..u1: A (m x n) <- A L^{-T}, right-looking over
// 64-column blocks j of A: solve block column j, then update the columns to
// its right.
__device__ void op_trsm_units(const TileDesc& Lt, const TileDesc& At, uint32_t phase, uint32_t u0,
                              uint32_t u1, F64Smem& s, bool fine) {
  const double* l = (const double*)Lt.ptr;
  double* a = (double*)At.ptr;
  const int m = At.rows, n = At.cols, lda = At.ld, ldl = Lt.ld;
  const int j = (int)(phase / 2), jb = j * kBlk, w = min(kBlk, n - jb);
  const int rb = fine ? 16 : kBlk;
  if (phase % 2 == 0) {  // row-block units
    load_block(s.l, l + (size_t)jb * ldl + jb, ldl, w, w);
    __syncthreads();
    prep_lower(s.l, w, s.rinv, false);
    for (uint32_t u = u0; u < u1; ++u) {
      const int ib = rb * (int)u, mb = min(rb, m - ib);
      double* x = a + (size_t)ib * lda + jb;
      load_rows(s.x, x, lda, mb, w);
      __syncthreads();
      trsm_rt_smem(s.x, s.l, s.rinv, mb, w);
      store_rows(x, lda, s.x, mb, w);
      __syncthreads();
    }
  } else {  // row-block x 64-column units
    const uint32_t right = cdiv64(n) - 1 - (uint32_t)j;
    for (uint32_t u = u0; u < u1; ++u) {
      const int ib = rb * (int)(u / right), lb = (j + 1 + (int)(u % right)) * kBlk;
      double* c = a + (size_t)ib * lda + lb;
      const double* ap = a + (size_t)ib * lda + jb;
      const double* bp = l + (size_t)lb * ldl + jb;
      if (fine)
        gemm_block<false, false, 4, 1>(c, lda, ap, lda, bp, ldl, min(16, m - ib),
                                       min(kBlk, n - lb), w, -1.0, false, s.gs);
      else
        gemm_block<false, false>(c, lda, ap, lda, bp, ldl, min(kBlk, m - ib), min(kBlk, n - lb),
                                 w, -1.0, false, s.gs);
    }
  }
}

// X <- X L^{-T} for m <= 16 rows of a shared array (row pitch ldx, the
// w-column block at column c0), L scaled by column: the arithmetic of
// trsm_rt_smem (a half-warp per row).  Warps whose two rows are both past m
// return at once; no barrier inside.
__device__ void trsm_rt_rows(double* xs, int ldx, int c0, const double (*l)[kLds],
                             const double* rinv, int m, int w) {
  const int tid = threadIdx.x, q = tid & 15, r = tid >> 4;
  if ((r & ~1) >= m) return;
  double* x = xs + (size_t)r * ldx + c0;
  double v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = q + 16 * j < w ? x[q + 16 * j] : 0.0;
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    for (int cl = 0; cl < 16; ++cl) {
      const int c = 16 * jj + cl;
      if (c >= w) break;
      const double yc = __shfl_sync(0xffffffffu, v[jj], cl, 16);
#pragma unroll
      for (int j = jj; j < 4; ++j) {
        const int cc = q + 16 * j;
        if (cc > c && cc < w) v[j] = fma(-yc, l[cc][c], v[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (q + 16 * j < w) x[q + 16 * j] = v[j] * rinv[q + 16 * j];
}

// TRSM in row form (critical-path tasks, n <= kTrsmRowMaxN): A (m x n) <- A
// L^{-T} in one phase; unit u = rows [kTrsmRows u, kTrsmRows (u + 1)), held
// in shared memory while every column block j of them is solved (the column
// form's in-block substitution) and subtracted, times L's blocks below the
// diagonal, from the blocks to its right (the column form's update: one FMA
// chain over k per entry, then one subtraction).  The same operations on
// the same values as op_trsm_units, so the result is bit-identical; each
// next L block is fetched into registers during the FMAs of the current one.
__device__ __noinline__ void op_trsm_rows(const TileDesc& Lt, const TileDesc& At, uint32_t u0,
                                          uint32_t u1, F64Smem& s) {
  static_assert(sizeof(GemmSmem) >= sizeof(double) * kTrsmRows * kTrsmRowMaxN, "row buffer");
  static_assert(kTrsmRows * kBlk == kThreads, "one update entry per thread");
  constexpr int kPre = kBlk * kBlk / kThreads;  // L entries fetched per thread
  const double* l = (const double*)Lt.ptr;
  double* a = (double*)At.ptr;
  const int m = At.rows, n = At.cols, lda = At.ld, ldl = Lt.ld;
  const int nb = (n + kBlk - 1) / kBlk;
  double* xs = reinterpret_cast<double*>(&s.gs);  // kTrsmRows x n, pitch n
  const int tid = threadIdx.x, ur = tid / kBlk, uc = tid % kBlk;
  double pre[kPre];
  auto fetch = [&](int jb, int w, int ib) {  // L block (ib, j) into pre
    const int lb = ib * kBlk, wc = min(kBlk, n - lb);
#pragma unroll
    for (int i = 0; i < kPre; ++i) {
      const int e = tid + kThreads * i, rr = e / kBlk, cc = e % kBlk;
      pre[i] = (rr < wc && cc < w) ? __ldcg(l + (size_t)(lb + rr) * ldl + jb + cc) : 0.0;
    }
  };
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = kTrsmRows * (int)u, mr = min(kTrsmRows, m - r0);
    for (int e = tid; e < kTrsmRows * n; e += kThreads) {
      const int r = e / n, c = e % n;
      xs[e] = r < mr ? __ldcg(a + (size_t)(r0 + r) * lda + c) : 0.0;
    }
    for (int j = 0; j < nb; ++j) {
      const int jb = j * kBlk, w = min(kBlk, n - jb);
      load_block(s.l, l + (size_t)jb * ldl + jb, ldl, w, w);
      if (j + 1 < nb) fetch(jb, w, j + 1);
      __syncthreads();
      prep_lower(s.l, w, s.rinv, false);
      trsm_rt_rows(xs, n, jb, s.l, s.rinv, mr, w);
      for (int ib = j + 1; ib < nb; ++ib) {
        __syncthreads();  // the solved block is in xs; s.x is free
#pragma unroll
        for (int i = 0; i < kPre; ++i) {
          const int e = tid + kThreads * i;
          s.x[e / kBlk][e % kBlk] = pre[i];
        }
        __syncthreads();
        if (ib + 1 < nb) fetch(jb, w, ib + 1);
        const int lb = ib * kBlk, wc = min(kBlk, n - lb);
        if (ur < mr && uc < wc) {
          const double* xr = xs + (size_t)ur * n + jb;
          double acc = 0.0;
          for (int k = 0; k < w; ++k) acc = fma(xr[k], s.x[uc][k], acc);
          double* p = xs + (size_t)ur * n + lb + uc;
          *p = *p - acc;
        }
      }
      __syncthreads();  // xs complete through block j; s.l is reloaded next
    }
    for (int e = tid; e < mr * n; e += kThreads)
      a[(size_t)(r0 + e / n) * lda + e % n] = xs[e];
    __syncthreads();
  }
}

// SYRK: C (n x n, lower) -= L L^T, L (n x k); units = lower 64-block pairs.
__device__ void op_syrk(const TileDesc& Lt, const TileDesc& Ct, uint32_t u0, uint32_t u1,
                        F64Smem& s, bool fine) {
  const double* l = (const double*)Lt.ptr;
  double* c = (double*)Ct.ptr;
  const int n = Ct.rows, k = Lt.cols;
  for (uint32_t u = u0; u < u1; ++u) {
    int bi, bj;
    lower_pair(u, bi, bj);
    if (fine) {  // 32 x 32 block pairs
      const int r0 = bi * 32, c0 = bj * 32;
      gemm_block<false, false, 2, 2>(c + (size_t)r0 * Ct.ld + c0, Ct.ld, l + (size_t)r0 * Lt.ld,
                                     Lt.ld, l + (size_t)c0 * Lt.ld, Lt.ld, min(32, n - r0),
                                     min(32, n - c0), k, -1.0, bi == bj, s.gs);
    } else {
      const int r0 = bi * kBlk, c0 = bj * kBlk;
      gemm_block<false, false>(c + (size_t)r0 * Ct.ld + c0, Ct.ld, l + (size_t)r0 * Lt.ld, Lt.ld,
                               l + (size_t)c0 * Lt.ld, Lt.ld, min(kBlk, n - r0),
                               min(kBlk, n - c0), k, -1.0, bi == bj, s.gs);
    }
  }
}

// Output-block GEMMs; units = 64x64 blocks of C, row-major (16 x 64 blocks
// for fine tasks).
template <bool A_T, bool B_KN>
__device__ void op_gemm(const TileDesc& At, const TileDesc& Bt, const TileDesc& Ct, int K,
                        double alpha, uint32_t u0, uint32_t u1, F64Smem& s, bool fine,
                        bool atomic = false) {
  const double* a = (const double*)At.ptr;
  const double* b = (const double*)Bt.ptr;
  double* c = (double*)Ct.ptr;
  const uint32_t nbc = (Ct.cols + kBlk - 1) / kBlk;
  const int rb = fine ? 16 : kBlk;
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / nbc) * rb, c0 = (int)(u % nbc) * kBlk;
    const double* ap = A_T ? a + r0 : a + (size_t)r0 * At.ld;
    const double* bp = B_KN ? b + c0 : b + (size_t)c0 * Bt.ld;
    double* cp = c + (size_t)r0 * Ct.ld + c0;
    const int mb = min(rb, Ct.rows - r0), nb = min(kBlk, Ct.cols - c0);
    if (fine)
      gemm_block<A_T, B_KN, 4, 1>(cp, Ct.ld, ap, At.ld, bp, Bt.ld, mb, nb, K, alpha, false, s.gs,
                                  false, atomic);
    else if (nb <= 16)
      gemm_block<A_T, B_KN, 1>(cp, Ct.ld, ap, At.ld, bp, Bt.ld, mb, nb, K, alpha, false, s.gs,
                               false, atomic);
    else
      gemm_block<A_T, B_KN>(cp, Ct.ld, ap, At.ld, bp, Bt.ld, mb, nb, K, alpha, false, s.gs, false,
                            atomic);
  }
}

// The narrow-block staging overlays the two 64x64 blocks (unused by GEMM
// parts).
static_assert(sizeof(NarrowSmem) <= 2 * sizeof(double) * kBlk * kLds, "narrow staging");
template <typename E = double>
__device__ __forceinline__ NarrowSmemT<E>& narrow_smem(F64Smem& s) {
  return *reinterpret_cast<NarrowSmemT<E>*>(&s.l[0][0]);
}

// C (rows x r) -= op(A) B for the block solves (units: see op_phase_units):
// 16-row units of all columns when r <= 16, else 64 x 64 output blocks.
// op(A) = A (A_T false) or A^T (A_T true); r0_c / r0_a: first row of C and
// of op(A) covered by unit 0.  E = float: FP32 operands, narrow shapes only
// (the operand checks keep FP32 solves to at most 16 columns).
template <bool A_T, typename E = double>
__device__ void rhs_update(const E* a, int lda, const E* b, int ldb, E* c, int ldc, int rows,
                           int cols, int K, uint32_t u0, uint32_t u1, F64Smem& s) {
  const int rb = (int)rhs_unit_rows(cols);
  const uint32_t ncb = rhs_col_blocks(cols);
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / ncb) * rb, c0 = (int)(u % ncb) * kBlk;
    const int m = min(rb, rows - r0), w = rhs_narrow(cols) ? cols : min(kBlk, cols - c0);
    const E* ap = A_T ? a + r0 : a + (size_t)r0 * lda;
    E* cp = c + (size_t)r0 * ldc + c0;
    if (rhs_narrow(cols))
      gemm_narrow<A_T>(cp, ldc, ap, lda, b + c0, ldb, m, w, K, E(-1), narrow_smem<E>(s));
    else if constexpr (std::is_same<E, double>::value) {
      if (w <= 16)
        gemm_block<A_T, true, 1>(cp, ldc, ap, lda, b + c0, ldb, m, w, K, -1.0, false, s.gs);
      else
        gemm_block<A_T, true>(cp, ldc, ap, lda, b + c0, ldb, m, w, K, -1.0, false, s.gs);
    }
  }
}

// Diagonal step of a block solve: X[ib:ib+mb, column block u] <- L_jj^{-1}
// (or L_jj^{-T}) times itself, L_jj = L[ib:ib+mb, ib:ib+mb].
template <bool kTrans>
__device__ void rhs_diag(const double* l, int ldl, double* x, int ldx, int ib, int mb, int cols,
                         uint32_t u0, uint32_t u1, F64Smem& s) {
  for (uint32_t u = u0; u < u1; ++u) {
    const int c0 = rhs_narrow(cols) ? 0 : (int)u * kBlk;
    const int w = rhs_narrow(cols) ? cols : min(kBlk, cols - c0);
    load_block(s.l, l + (size_t)ib * ldl + ib, ldl, mb, mb);
    load_block(s.x, x + (size_t)ib * ldx + c0, ldx, mb, w);
    __syncthreads();
    prep_lower(s.l, mb, s.rinv, kTrans);
    trsm_left_smem<kTrans>(s.x, s.l, s.rinv, mb, w);
    store_block(x + (size_t)ib * ldx + c0, ldx, s.x, mb, w, false);
    __syncthreads();
  }
}

// X <- L^{-1} X (forward substitution, L n x n lower, X n x r), right-looking
// over 64-row blocks j: phase 2j solves block j, phase 2j+1 updates the rows
// below it (X_below -= L[below, j] X_j).
__device__ void op_trsm_fwd(const TileDesc& Lt, const TileDesc& Xt, uint32_t phase, uint32_t u0,
                            uint32_t u1, F64Smem& s) {
  const double* l = (const double*)Lt.ptr;
  double* x = (double*)Xt.ptr;
  const int n = Lt.rows, ldl = Lt.ld, ldx = Xt.ld, cols = Xt.cols;
  const int ib = (int)(phase / 2) * kBlk, mb = min(kBlk, n - ib);
  if (phase % 2 == 0) {
    rhs_diag<false>(l, ldl, x, ldx, ib, mb, cols, u0, u1, s);
    return;
  }
  const int r0 = ib + mb;
  rhs_update<false>(l + (size_t)r0 * ldl + ib, ldl, x + (size_t)ib * ldx, ldx,
                    x + (size_t)r0 * ldx, ldx, n - r0, cols, mb, u0, u1, s);
}

// X <- L^{-T} X (back substitution), over 64-row blocks from the last:
// phase 2q solves block j = nb-1-q with L_jj^T, phase 2q+1 updates the rows
// above it (X_above -= L[j, above]^T X_j).
__device__ void op_trsm_bwd(const TileDesc& Lt, const TileDesc& Xt, uint32_t phase, uint32_t u0,
                            uint32_t u1, F64Smem& s) {
  const double* l = (const double*)Lt.ptr;
  double* x = (double*)Xt.ptr;
  const int n = Lt.rows, ldl = Lt.ld, ldx = Xt.ld, cols = Xt.cols;
  const int nb = (n + kBlk - 1) / kBlk;
  const int ib = (nb - 1 - (int)(phase / 2)) * kBlk, mb = min(kBlk, n - ib);
  if (phase % 2 == 0) {
    rhs_diag<true>(l, ldl, x, ldx, ib, mb, cols, u0, u1, s);
    return;
  }
  rhs_update<true>(l + (size_t)ib * ldl, ldl, x + (size_t)ib * ldx, ldx, x, ldx, ib, cols, mb, u0,
                   u1, s);
}

// Y <- T X (trans false) or T^T X (trans true) for T (n x n, zero above its
// diagonal) and X, Y (n x r, distinct tiles); the units of GEMM_FWD.  Each
// unit covers rows r0..r0+m-1 of Y and multiplies over the part of T that
// can be nonzero for them: columns [0, r0 + m) of T, or rows [r0, n) of T
// for the transpose.  E = float: FP32 tiles, narrow shapes only.
template <typename E = double>
__device__ void op_trmm(const TileDesc& Tt, const TileDesc& Xt, const TileDesc& Yt, bool trans,
                        uint32_t u0, uint32_t u1, F64Smem& s) {
  const E* tp = (const E*)Tt.ptr;
  const E* x = (const E*)Xt.ptr;
  E* y = (E*)Yt.ptr;
  const int n = Tt.rows, cols = Yt.cols, ldt = Tt.ld, ldx = Xt.ld, ldy = Yt.ld;
  const int rb = (int)rhs_unit_rows(cols);
  const uint32_t ncb = rhs_col_blocks(cols);
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / ncb) * rb, c0 = (int)(u % ncb) * kBlk;
    const int m = min(rb, n - r0), w = rhs_narrow(cols) ? cols : min(kBlk, cols - c0);
    E* yp = y + (size_t)r0 * ldy + c0;
    if (!trans) {  // rows r0.. of T, columns [0, r0 + m)
      const E* ap = tp + (size_t)r0 * ldt;
      const int K = r0 + m;
      if (rhs_narrow(cols))
        gemm_narrow<false>(yp, ldy, ap, ldt, x + c0, ldx, m, w, K, E(1), narrow_smem<E>(s), true);
      else if constexpr (std::is_same<E, double>::value) {
        if (w <= 16)
          gemm_block<false, true, 1>(yp, ldy, ap, ldt, x + c0, ldx, m, w, K, 1.0, false, s.gs,
                                     true);
        else
          gemm_block<false, true>(yp, ldy, ap, ldt, x + c0, ldx, m, w, K, 1.0, false, s.gs, true);
      }
    } else {  // columns r0.. of T, rows [r0, n)
      const E* ap = tp + (size_t)r0 * ldt + r0;
      const E* bp = x + (size_t)r0 * ldx + c0;
      const int K = n - r0;
      if (rhs_narrow(cols))
        gemm_narrow<true>(yp, ldy, ap, ldt, bp, ldx, m, w, K, E(1), narrow_smem<E>(s), true);
      else if constexpr (std::is_same<E, double>::value) {
        if (w <= 16)
          gemm_block<true, true, 1>(yp, ldy, ap, ldt, bp, ldx, m, w, K, 1.0, false, s.gs, true);
        else
          gemm_block<true, true>(yp, ldy, ap, ldt, bp, ldx, m, w, K, 1.0, false, s.gs, true);
      }
    }
  }
}

// TRTRI by blocks, phase `phase`, units u0..u1: V (n x n) <- L^{-1} for the
// lower triangle of L (see trtri_phases).  Phase 0, unit j: the inverse of
// the diagonal block L_jj, as the transpose of X = I L_jj^{-T} (the in-tile
// row solve), and zeros to its right.  Level phases: for each pair of
// diagonal s-blocks T = [p, p+s), B = [p+s, p+s+sB):
//   a) W^T = V_TT^T L_BT^T (s x sB) into V[p:p+s, p+s:p+s+sB], which is above
//      the diagonal (zero in the result, so free scratch); V_TT lower, so
//      output row j of W^T sums over k >= j only;
//   b) V_BT = -V_BB W, V_BB lower, so output row i sums over k <= i only.
// The k ranges start and end on 16-row bands inside the diagonal 64-blocks,
// so no product reads the scratch of an earlier level.  Last phase: the part
// of V above the diagonal 64-blocks back to zero.
__device__ void op_trtri_units(const TileDesc& Lt, const TileDesc& Vt, uint32_t phase, uint32_t u0,
                               uint32_t u1, F64Smem& s) {
  const double* l = (const double*)Lt.ptr;
  double* v = (double*)Vt.ptr;
  const int n = Lt.rows, ldl = Lt.ld, ldv = Vt.ld;
  if (phase == 0) {
    for (uint32_t u = u0; u < u1; ++u) {
      const int jb = (int)u * kBlk, w = min(kBlk, n - jb);
      load_block(s.l, l + (size_t)jb * ldl + jb, ldl, w, w);
      for (int e = threadIdx.x; e < kBlk * kBlk; e += kThreads)
        s.x[e / kBlk][e % kBlk] = (e / kBlk == e % kBlk) ? 1.0 : 0.0;
      __syncthreads();
      prep_lower(s.l, w, s.rinv, false);
      trsm_rt_smem(s.x, s.l, s.rinv, w, w);  // X = L_jj^{-T}
      for (int e = threadIdx.x; e < w * (n - jb); e += kThreads) {
        const int r = e / (n - jb), c = e % (n - jb);
        v[(size_t)(jb + r) * ldv + jb + c] = c < w ? s.x[c][r] : 0.0;
      }
      __syncthreads();
    }
    return;
  }
  if (phase + 1 == trtri_phases(n)) {  // zero above the diagonal 64-blocks
    for (uint32_t u = u0; u < u1; ++u) {
      const int jb = (int)u * kBlk, w = min(kBlk, n - jb), c0 = jb + w;
      for (int e = threadIdx.x; e < w * (n - c0); e += kThreads)
        v[(size_t)(jb + e / (n - c0)) * ldv + c0 + e % (n - c0)] = 0.0;
    }
    return;
  }
  for (uint32_t u = u0; u < u1; ++u) {
    int pr[4];
    trtri_level_units(n, phase, u, pr);
    const int p = pr[0], sz = pr[1], sb = pr[2], lu = pr[3];
    double* wt = v + (size_t)p * ldv + p + sz;  // W^T scratch, s x sB
    if (phase % 2 == 1) {
      // unit: 16 rows [j0, j0+16) of W^T x 64 columns [c0, c0+64)
      const uint32_t ncb = cdiv64(sb);
      const int j0 = 16 * (int)(lu / ncb), c0 = kBlk * (int)(lu % ncb);
      const double* vtt = v + (size_t)p * ldv + p;              // V_TT, A^T operand
      const double* lbt = l + (size_t)(p + sz) * ldl + p;       // L_BT, B stored n x k
      gemm_block<true, false, 4, 1>(wt + (size_t)j0 * ldv + c0, ldv, vtt + (size_t)j0 * ldv + j0,
                                    ldv, lbt + (size_t)c0 * ldl + j0, ldl, min(16, sz - j0),
                                    min(kBlk, sb - c0), sz - j0, 1.0, false, s.gs, true);
    } else {
      // unit: 16 rows [i0, i0+16) of V_BT x 64 columns [c0, c0+64)
      const uint32_t ncb = (uint32_t)(sz / kBlk);
      const int i0 = 16 * (int)(lu / ncb), c0 = kBlk * (int)(lu % ncb);
      const double* vbb = v + (size_t)(p + sz) * ldv + p + sz;  // V_BB
      double* vbt = v + (size_t)(p + sz) * ldv + p;
      // W[k][c] = W^T[c][k]: B stored n x k
      gemm_block<false, false, 4, 1>(vbt + (size_t)i0 * ldv + c0, ldv, vbb + (size_t)i0 * ldv, ldv,
                                     wt + (size_t)c0 * ldv, ldv, min(16, sb - i0), kBlk,
                                     min(i0 + 16, sb), -1.0, false, s.gs, true);
    }
  }
}

// V <- I on 64-row units (phase 0 of TRTRI).
__device__ void op_identity(const TileDesc& Vt, uint32_t u0, uint32_t u1) {
  double* v = (double*)Vt.ptr;
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)u * kBlk, mb = min(kBlk, Vt.rows - r0);
    for (int e = threadIdx.x; e < mb * Vt.cols; e += kThreads) {
      const int r = r0 + e / Vt.cols, c = e % Vt.cols;
      v[(size_t)r * Vt.ld + c] = r == c ? 1.0 : 0.0;
    }
  }
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Y <- X (axpy = false) or Y <- Y + alpha X (axpy = true) on 64-row blocks
// u0..u1, for X and Y each FP64 or FP32 (EX, EY); FP32 -> FP64 is exact,
// FP64 -> FP32 rounds to nearest.  In Y's type: fl(fl(alpha x) + y), the
// product skipped when alpha = 1 (no contraction into an FMA: the paper's
// FP32 AXPY has one rounding per operation).
// Contiguous tiles of one element type (ld == cols, 16-byte aligned): a unit
// is one flat range, read and written with 16-byte vector accesses, four per
// thread in flight (the HBM-bound AXPY test case).
template <typename E>
__device__ void copy_axpy_flat(const E* __restrict__ x, E* __restrict__ y, size_t n, bool axpy,
                               E a, bool one) {
  constexpr int kV = 16 / sizeof(E);  // elements per vector
  using V = typename std::conditional<sizeof(E) == 4, float4, double2>::type;
  const size_t nv = n / kV;
  const V* xv = reinterpret_cast<const V*>(x);
  V* yv = reinterpret_cast<V*>(y);
  size_t i = threadIdx.x;
  for (; i + 3 * kThreads < nv; i += 4 * kThreads) {
    V xs[4], ys[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xs[k] = __ldcs(xv + i + k * kThreads);
      if (axpy) ys[k] = __ldcs(yv + i + k * kThreads);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      E* xe = reinterpret_cast<E*>(&xs[k]);
      E* ye = reinterpret_cast<E*>(&ys[k]);
#pragma unroll
      for (int c = 0; c < kV; ++c) ye[c] = axpy ? add_rn(ye[c], one ? xe[c] : mul_rn(a, xe[c])) : xe[c];
      __stcs(yv + i + k * kThreads, ys[k]);
    }
  }
  for (; i < nv; i += kThreads) {
    V xs = __ldcs(xv + i), ys = axpy ? __ldcs(yv + i) : xs;
    E* xe = reinterpret_cast<E*>(&xs);
    E* ye = reinterpret_cast<E*>(&ys);
#pragma unroll
    for (int c = 0; c < kV; ++c) ye[c] = axpy ? add_rn(ye[c], one ? xe[c] : mul_rn(a, xe[c])) : xe[c];
    __stcs(yv + i, ys);
  }
  for (size_t e = nv * kV + threadIdx.x; e < n; e += kThreads)
    y[e] = axpy ? add_rn(y[e], one ? x[e] : mul_rn(a, x[e])) : x[e];
}

template <typename EX, typename EY>
__device__ void copy_axpy_t(const TileDesc& Xt, const TileDesc& Yt, uint32_t u0, uint32_t u1,
                            bool axpy, bool atomic, double alpha) {
  const EX* x = (const EX*)Xt.ptr;
  EY* y = (EY*)Yt.ptr;
  const EY a = (EY)alpha;
  const bool one = alpha == 1.0;
  if constexpr (sizeof(EX) == sizeof(EY)) {
    if (!atomic && Xt.ld == Xt.cols && Yt.ld == Yt.cols && ((uintptr_t)x & 15) == 0 &&
        ((uintptr_t)y & 15) == 0) {
      const size_t r0 = (size_t)u0 * kBlk;
      const size_t r1 = min((size_t)u1 * kBlk, (size_t)Yt.rows);
      copy_axpy_flat<EY>(reinterpret_cast<const EY*>(x) + r0 * Yt.cols, y + r0 * Yt.cols,
                         (r1 - r0) * Yt.cols, axpy, a, one);
      return;
    }
  }
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)u * kBlk, mb = min(kBlk, Yt.rows - r0);
    for (int e = threadIdx.x; e < mb * Yt.cols; e += kThreads) {
      const int r = r0 + e / Yt.cols, c = e % Yt.cols;
      const EY v = (EY)__ldcg(x + (size_t)r * Xt.ld + c);
      EY* py = y + (size_t)r * Yt.ld + c;
      const EY av = one ? v : mul_rn(a, v);
      if (axpy && atomic) atomicAdd(py, av);  // ATOMIC_WRITE on Y
      else *py = axpy ? add_rn(__ldcg(py), av) : v;
    }
  }
}

__device__ void op_copy_axpy(const TileDesc& Xt, const TileDesc& Yt, uint32_t u0, uint32_t u1,
                             bool axpy, bool atomic = false, double alpha = 1.0) {
  const bool xf = Xt.dtype == SPX_DT_F32, yf = Yt.dtype == SPX_DT_F32;
  if (!xf && !yf) copy_axpy_t<double, double>(Xt, Yt, u0, u1, axpy, atomic, alpha);
  else if (!xf) copy_axpy_t<double, float>(Xt, Yt, u0, u1, axpy, atomic, alpha);
  else if (!yf) copy_axpy_t<float, double>(Xt, Yt, u0, u1, axpy, atomic, alpha);
  else copy_axpy_t<float, float>(Xt, Yt, u0, u1, axpy, atomic, alpha);
}

// Coulomb interactions (the paper's particle test case): targets
// [t0, t0 + mt) of group T (n x 8 FP64 rows: x, y, z, q, phi, E) against all
// ns sources of group S; self: S is T, and a target skips itself.  Each
// interaction adds q_j / r to phi_i and q_j (x_i - x_j) / r^3 to E_i, r = 0
// skipped; 1 / r is 1 / sqrt(r^2) with IEEE square root and division.  The
// 256 threads are 64 targets x 4 source slices (slice q: sources j = q mod
// 4, in order), sources staged 256 at a time in shared memory; the four
// partial sums of a target are added in slice order (deterministic).
__device__ void nbody_block(double* T, int ldt, int t0, int mt, const double* S, int lds, int ns,
                            bool self, F64Smem& s) {
  const int tid = threadIdx.x, ti = tid & 63, q = tid >> 6;
  const int i = t0 + ti;
  const bool live = ti < mt;
  const double xi = live ? T[(size_t)i * ldt + 0] : 0.0;
  const double yi = live ? T[(size_t)i * ldt + 1] : 0.0;
  const double zi = live ? T[(size_t)i * ldt + 2] : 0.0;
  double phi = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
  double* src = &s.l[0][0];  // [256][4]: x, y, z, q
  static_assert(sizeof(s.l) >= 256 * 4 * sizeof(double), "source staging");
  static_assert(sizeof(s.x) >= 4 * 64 * 4 * sizeof(double), "partial sums");
  for (int j0 = 0; j0 < ns; j0 += 256) {
    const int nj = min(256, ns - j0);
    __syncthreads();
    for (int e = tid; e < nj * 4; e += kThreads) src[e] = __ldcg(S + (size_t)(j0 + e / 4) * lds + e % 4);
    __syncthreads();
    if (live) {
      for (int jj = q; jj < nj; jj += 4) {
        if (self && j0 + jj == i) continue;
        const double dx = xi - src[4 * jj + 0];
        const double dy = yi - src[4 * jj + 1];
        const double dz = zi - src[4 * jj + 2];
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (r2 > 0.0) {
          const double rinv = 1.0 / sqrt(r2);
          const double qr = src[4 * jj + 3] * rinv;
          const double s3 = qr * rinv * rinv;
          phi += qr;
          ex = fma(s3, dx, ex);
          ey = fma(s3, dy, ey);
          ez = fma(s3, dz, ez);
        }
      }
    }
  }
  double* red = &s.x[0][0];  // [4 slices][64 targets][4]
  __syncthreads();
  red[(q * 64 + ti) * 4 + 0] = phi;
  red[(q * 64 + ti) * 4 + 1] = ex;
  red[(q * 64 + ti) * 4 + 2] = ey;
  red[(q * 64 + ti) * 4 + 3] = ez;
  __syncthreads();
  if (tid < 64 && live) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int qq = 0; qq < 4; ++qq)
      for (int c = 0; c < 4; ++c) a[c] += red[(qq * 64 + ti) * 4 + c];
    for (int c = 0; c < 4; ++c) T[(size_t)i * ldt + 4 + c] += a[c];
  }
  __syncthreads();
}

// NBODY_SELF / NBODY_PAIR units: 64-target blocks of P (against P itself,
// or against Q), then, for a pair, of Q against P.
__device__ void op_nbody(const TileDesc& Pt, const TileDesc* Qt, uint32_t u0, uint32_t u1,
                         F64Smem& s) {
  const uint32_t np = cdiv64(Pt.rows);
  for (uint32_t u = u0; u < u1; ++u) {
    const bool onp = u < np;
    const TileDesc& Tg = onp ? Pt : *Qt;
    const TileDesc& Sg = Qt ? (onp ? *Qt : Pt) : Pt;
    const int t0 = (int)(onp ? u : u - np) * kBlk;
    nbody_block((double*)Tg.ptr, Tg.ld, t0, min(kBlk, Tg.rows - t0), (const double*)Sg.ptr, Sg.ld,
                Sg.rows, Qt == nullptr, s);
  }
}

}  // namespace
}  // namespace spx
