// FP64 trailing updates emulated on the BF16 tensor cores by splitting (the
// Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), for the paper's tiled
// Cholesky, whose flops are almost all in SYRK and GEMM (section "Numerical
// applications").  This GPU's FP64 SIMT pipe peaks near 1.2 TFLOP/s, its
// BF16 tensor cores near 2 PFLOP/s.
//
// Split (a final phase of the TRSM that produced the tile), per row r:
//   e_r  = Ef - 1022, Ef the biased exponent field of max_k |a_rk|: the
//          smallest e with every |a_rk| < 2^e; -1022 when Ef = 0 (a row of
//          zeros and subnormals);
//   X_rk = a_rk 2^(55 - e_r) rounded to the nearest integer, ties to even
//          (|X_rk| <= 2^55; exact when ulp(a_rk) >= 2^(e_r - 55));
//   X_rk = sum_{s=0..7} sigma_s 128^(7-s), balanced digits taken from the
//          bottom: sigma_s = ((X + 64) mod 128) - 64 in [-64, 63], X <- (X -
//          sigma_s) / 128; the top digit sigma_0 in [-64, 64].
// The slot of the tile holds the eight digit planes as BF16 (integers of
// magnitude <= 64 are exact in BF16), each cut into 16-digit K chunks stored
// one after another (plane s, chunk j, row r, digit i at element
// ((s (b/16) + j) b + r) 16 + i), so that the operand of one K step is a
// contiguous run of rows; then the exponents e_r.
//
// Product, C -= A B^T with A, B split (rows r of A, rows c of B), K <= 512:
//   P_d = sum_{s+t=d} sum_k sigma_s[r,k] tau_t[c,k],  d = 0..7,
// the pairs with s + t > 7 dropped.  |sigma tau| <= 2^12 and at most 8
// pairs per d, so |P_d| <= 8 * 512 * 2^12 = 2^24: every partial sum is an
// integer that FP32 holds exactly, whatever the order of accumulation.
//   F = sum_d P_d 128^(7-d) = Fh 2^28 + Fl,
//       Fh = sum_{d<4} P_d 128^(3-d), Fl = sum_{d>=4} P_d 128^(7-d) (int64);
//   v = RN(F 2^(e_r + f_c - 61)) = RN(Fh 2^(28+x) + Fl 2^x), x = e_r + f_c - 61
//       (both terms exact FP64, one rounded addition); C_rc <- RN(C_rc - v).
//
// Tensor-core unit: 128 output rows x 32 output columns.  Eight FP32
// accumulators of 32 TMEM columns, accumulator d at column 32 d.  For each
// 16-wide K step, digit plane s of A (128 x 16) multiplies the planes
// t = 0..7-s of B stacked along N (32 (8 - s) rows) in one MMA whose output
// starts at accumulator s: output block t lands in accumulator s + t.  The K
// step's operands (8 planes x 128 rows of A, 8 planes x 32 rows of B, 40 KB)
// arrive by one 5-D TMA box each (32-byte swizzle), two stages.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.h"
#include "tile_tc.cuh"

namespace spx {
namespace {

constexpr int kOzPlanes = 8;
constexpr int kOzN = 32;                              // output columns per unit
constexpr int kOzStageA = kOzPlanes * kTcM * 32;      // 32 KB: 8 planes x 128 rows x 16 digits
constexpr int kOzStageB = kOzPlanes * kOzN * 32;      // 8 KB
constexpr int kOzStage = kOzStageA + kOzStageB;
constexpr int kOzStages = 2;
static_assert(kOzStages * kOzStage <= (int)sizeof(TcBuf), "split operand stages fit the buffer");
static_assert(kOzPlanes * kOzN <= (int)kTcCtaCols, "eight accumulators fit the CTA's TMEM");
static_assert(kOzStage % 1024 == 0, "stages stay aligned");

// K-major operand, 32-byte swizzle (rows of 32 bytes, 8-row groups 256 bytes
// apart), descriptor version 1.
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t oz_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 5-D box (digit, row, K chunk, plane, slot) of the split store.
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int row, int kchunk, int slot) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(0), "r"(row), "r"(kchunk), "r"(0), "r"(slot)
      : "memory");
}

// 8 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// N * 2^y as FP64 when that is exact and normal: |N| < 2^53 and the result's
// exponent in the normal range.  Built from the bits (integer pipe only).
__device__ __forceinline__ bool oz_i2d(long long N, int y, double& out) {
  if (N == 0) {
    out = 0.0;
    return true;
  }
  const unsigned long long sgn = N < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = N < 0 ? (unsigned long long)(-N) : (unsigned long long)N;
  const int L = 64 - __clzll((long long)a);  // bit length, 1..53
  const int ef = L - 1 + 1023 + y;
  if (ef < 1 || ef > 2046) return false;
  const unsigned long long mant = (a << (53 - L)) & 0xFFFFFFFFFFFFFull;
  out = __longlong_as_double((long long)(sgn | ((unsigned long long)ef << 52) | mant));
  return true;
}

// X = a 2^(55 - e) rounded to the nearest integer, ties to even (|a| < 2^e).
__device__ __forceinline__ long long oz_fixed(unsigned long long bits, int e) {
  const int ef = (int)((bits >> 52) & 0x7FFu);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  int E;
  if (ef == 0) {
    E = -1074;
  } else {
    m |= 1ull << 52;
    E = ef - 1075;
  }
  if (m == 0) return 0;
  const int sh = E + 55 - e;  // <= 3, since m 2^sh < 2^55
  unsigned long long X;
  if (sh >= 0) {
    X = m << sh;
  } else if (-sh >= 54) {
    X = 0;  // m < 2^53: below half a unit
  } else {
    const int k = -sh;
    const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
    X = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  return (bits >> 63) ? -(long long)X : (long long)X;
}

// Split rows [64 u, 64 u + 64) of the FP64 tile Lt into its slot (lowp =
// slot address, lowp_ld = pitch b <= 512).  Columns cols..b-1 of each digit
// plane are written as zeros (the K padding the tensor cores read).  One
// warp per row, 16 columns per lane.
__device__ __noinline__ void op_oz_split(const TileDesc& Lt, uint32_t u0, uint32_t u1) {
  const int b = Lt.lowp_ld;
  __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(Lt.lowp);
  int* Ex = reinterpret_cast<int*>(reinterpret_cast<char*>(Lt.lowp) + (size_t)16 * b * b);
  const double* A = reinterpret_cast<const double*>(Lt.ptr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nj = b / 32;
  for (uint32_t u = u0; u < u1; ++u) {
    const int rend = min((int)(u + 1) * 64, Lt.rows);
    for (int r = (int)u * 64 + warp; r < rend; r += kThreads / 32) {
      unsigned long long bits[16];
      unsigned long long mx = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = lane + 32 * j;
        bits[j] = (j < nj && c < Lt.cols)
                      ? (unsigned long long)__double_as_longlong(__ldcg(A + (size_t)r * Lt.ld + c))
                      : 0ull;
        const unsigned long long mag = bits[j] & 0x7FFFFFFFFFFFFFFFull;
        mx = mag > mx ? mag : mx;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = y > mx ? y : mx;
      }
      const int ef = (int)(mx >> 52);
      const int e = ef ? ef - 1022 : -1022;
      if (lane == 0) Ex[r] = e;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j >= nj) break;
        const int c = lane + 32 * j;
        long long X = oz_fixed(bits[j], e);
        int sg[kOzPlanes];
#pragma unroll
        for (int s = kOzPlanes - 1; s >= 1; --s) {
          const int d = (int)((X + 64) & 127) - 64;
          sg[s] = d;
          X = (X - d) >> 7;
        }
        sg[0] = (int)X;
#pragma unroll
        // K-chunked layout: plane s, 16-digit chunk c / 16, row r, digit c % 16
        for (int s = 0; s < kOzPlanes; ++s)
          S[(((size_t)s * (b / 16) + c / 16) * b + r) * 16 + (c & 15)] =
              __float2bfloat16_rn((float)sg[s]);
      }
    }
  }
}

// One 128 x 32 output unit: C[0:m, 0:n] -= (A B^T) by the split product.
// A rows come from slot a_slot rows a_r0.. (TMA map amap, 128-row boxes),
// B rows from slot b_slot rows b_r0.. (bmap, 32-row boxes); K digits.
// a_exp / b_exp: the exponents of those rows.  Entries with column >
// row + diag are left alone (SYRK's diagonal blocks).  All threads; false on
// a barrier timeout.  store: C = A B^T instead (v rounded once, no
// subtraction).
__device__ bool oz_unit(TcState& s, TcBuf& buf, const CUtensorMap* amap, int a_slot, int a_r0,
                        const CUtensorMap* bmap, int b_slot, int b_r0, int K, const int* a_exp,
                        const int* b_exp, double* C, int ldc, int m, int n, int diag,
                        bool store = false) {
  const int nsteps = (K + 15) / 16;
  const int tid = threadIdx.x;
  const uint32_t tmem = s.tmem_base;
  uint8_t* const sb = reinterpret_cast<uint8_t*>(&buf);
  // the stages may hold generic-proxy writes of an earlier op: order them
  // before the TMA writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid >= 32 && !store) {
    // pull the FP64 output block into L2 while the MMAs run (32 columns =
    // two 128-byte lines per row)
    for (int e = tid - 32; e < 2 * m; e += kThreads - 32) {
      const int r = e >> 1, l = e & 1;
      if (l * 16 < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (size_t)r * ldc + l * 16));
    }
  }
  if (tid == 0) {
    tc_fence_after();
    bool ok = true;
    uint32_t fph = s.full_phase, eph = s.empty_phase;
    auto issue = [&](int st, int step) {
      uint8_t* dst = sb + st * kOzStage;
      mbar_arrive_expect_tx(&s.full[st], kOzStage);
      tma_load_5d(dst, amap, &s.full[st], a_r0, step, a_slot);
      tma_load_5d(dst + kOzStageA, bmap, &s.full[st], b_r0, step, b_slot);
    };
    const int pre = nsteps < kOzStages ? nsteps : kOzStages;
    for (int c = 0; c < pre; ++c) issue(c, c);
    int waited = 0;
    for (int c = 0; c < nsteps && ok; ++c) {
      const int st = c % kOzStages;
      ok = mbar_wait(&s.full[st], (fph >> st) & 1u);
      fph ^= 1u << st;
      if (!ok) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sb + st * kOzStage), b0 = a0 + kOzStageA;
#pragma unroll
      for (int p = 0; p < kOzPlanes; ++p)
        oz_mma(tmem + (uint32_t)(kOzN * p), oz_desc(a0 + (uint32_t)(p * kTcM * 32)), oz_desc(b0),
               oz_idesc((uint32_t)(kOzN * (kOzPlanes - p))), (c > 0 || p > 0) ? 1u : 0u);
      tc_commit(&s.empty[st]);
      const int pc = c - 1;
      if (pc >= 0 && pc + kOzStages < nsteps) {
        const int ps = pc % kOzStages;
        ok = mbar_wait(&s.empty[ps], (eph >> ps) & 1u);
        eph ^= 1u << ps;
        waited = pc + 1;
        if (!ok) break;
        issue(ps, pc + kOzStages);
      }
    }
    tc_commit(&s.done);
    if (ok) ok = mbar_wait(&s.done, s.done_phase & 1u);
    s.done_phase ^= 1u;
    for (int c = waited; c < nsteps && ok; ++c) {
      const int st = c % kOzStages;
      ok = mbar_wait(&s.empty[st], (eph >> st) & 1u);
      eph ^= 1u << st;
    }
    s.full_phase = fph;
    s.empty_phase = eph;
    if (!ok) s.error = 1;
  }
  __syncthreads();
  if (s.error) return false;
  tc_fence_after();
  // Epilogue, 1: warp w reads TMEM lanes 32 (w % 4).. (rows) and columns
  // 16 (w / 4).. of every accumulator, 8 at a time, forms v in integers plus
  // one FP64 addition and stages it in shared memory (the operand stages are
  // free: every MMA has completed).
  constexpr int kLdv = kOzN + 1;
  static_assert(sizeof(double) * kTcM * kLdv <= sizeof(TcBuf), "staging fits the stages");
  double* V = reinterpret_cast<double*>(sb);
  const int warp = tid >> 5, lane = tid & 31;
  const int r = 32 * (warp & 3) + lane;
  const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const int er = r < m ? a_exp[r] : 0;
#pragma unroll 1
  for (int sub = 0; sub < 2; ++sub) {
    const int cb = 16 * (warp >> 2) + 8 * sub;
    long long fh[8], fl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) fh[j] = fl[j] = 0;
#pragma unroll
    for (int d = 0; d < kOzPlanes; ++d) {
      uint32_t v[8];
      tmem_ld8(lanes + (uint32_t)(kOzN * d + cb), v);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long p = __float2int_rn(__uint_as_float(v[j]));
        if (d < 4) fh[j] = fh[j] * 128 + p;
        else fl[j] = fl[j] * 128 + p;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = cb + j;
      double v = 0.0;
      if (r < m && c < n) {
        const int x = er + b_exp[c] - 61;
        double vh, vl;
        if (oz_i2d(fh[j], 28 + x, vh) && oz_i2d(fl[j], x, vl))
          v = __dadd_rn(vh, vl);
        else
          v = scalbn(__fma_rn(__ll2double_rn(fh[j]), 268435456.0, __ll2double_rn(fl[j])), x);
      }
      V[r * kLdv + c] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  // Epilogue, 2: coalesced read-modify-write of the output block (a warp
  // covers a row's 32 columns); each thread's loads are issued before any of
  // its stores.
  constexpr int kPer = kTcM * kOzN / kThreads;
  double cv[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int rr = warp + (kThreads / 32) * i, c = lane;
    cv[i] = (!store && rr < m && c < n && c <= rr + diag) ? C[(size_t)rr * ldc + c] : 0.0;
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int rr = warp + (kThreads / 32) * i, c = lane;
    if (rr < m && c < n && c <= rr + diag)
      C[(size_t)rr * ldc + c] = store ? V[rr * kLdv + c] : __dsub_rn(cv[i], V[rr * kLdv + c]);
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ const int* oz_exps(const TileDesc& t) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(t.lowp) +
                                      (size_t)16 * t.lowp_ld * t.lowp_ld);
}

// GEMM_NT_SUB: C (FP64) -= A B^T from the slots of A and B; units are the
// 128 x 32 blocks of C, row block by row block.
__device__ __noinline__ bool op_oz_gemm(const DevGraph& g, const TileDesc& At, const TileDesc& Bt,
                                        const TileDesc& Ct, uint32_t u0, uint32_t u1,
                                        TcState* st, TcBuf* buf) {
  double* c = (double*)Ct.ptr;
  const uint32_t nbc = cdiv32(Ct.cols);
  const int* ae = oz_exps(At);
  const int* be = oz_exps(Bt);
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / nbc) * kTcM, c0 = (int)(u % nbc) * kOzN;
    if (!oz_unit(*st, *buf, g.maps + At.lmap, At.lr0, r0, g.maps + Bt.lmap + 1, Bt.lr0, c0,
                 At.cols, ae + r0, be + c0, c + (size_t)r0 * Ct.ld + c0, Ct.ld,
                 min(kTcM, Ct.rows - r0), min(kOzN, Ct.cols - c0), 1 << 30))
      return false;
  }
  return true;
}

// SYRK: C (FP64, lower) -= L L^T from the slot of L; units are the 128 x 32
// blocks of C that reach the lower triangle.
__device__ __noinline__ bool op_oz_syrk(const DevGraph& g, const TileDesc& Lt, const TileDesc& Ct,
                                        uint32_t u0, uint32_t u1, TcState* st, TcBuf* buf) {
  double* c = (double*)Ct.ptr;
  const int* le = oz_exps(Lt);
  for (uint32_t u = u0; u < u1; ++u) {
    uint32_t ij[2] = {0, 0};
    oz_syrk_units(Ct.rows, u, ij);
    const int r0 = (int)ij[0] * kTcM, c0 = (int)ij[1] * kOzN;
    if (!oz_unit(*st, *buf, g.maps + Lt.lmap, Lt.lr0, r0, g.maps + Lt.lmap + 1, Lt.lr0, c0,
                 Lt.cols, le + r0, le + c0, c + (size_t)r0 * Ct.ld + c0, Ct.ld,
                 min(kTcM, Ct.rows - r0), min(kOzN, Ct.cols - c0), r0 - c0))
      return false;
  }
  return true;
}

// TRSM by the inverse: A (FP64) <- A V^T, V = L_kk^{-1}, from the slots of
// A (split in the task's previous phase) and of V; units are the 128 x 32
// blocks of A.  The product only reads the slots, so it may overwrite A.
__device__ __noinline__ bool op_oz_trsm_inv(const DevGraph& g, const TileDesc& Vt,
                                            const TileDesc& At, uint32_t u0, uint32_t u1,
                                            TcState* st, TcBuf* buf) {
  double* a = (double*)At.ptr;
  const uint32_t nbc = cdiv32(At.cols);
  const int* ae = oz_exps(At);
  const int* ve = oz_exps(Vt);
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / nbc) * kTcM, c0 = (int)(u % nbc) * kOzN;
    if (!oz_unit(*st, *buf, g.maps + At.lmap, At.lr0, r0, g.maps + Vt.lmap + 1, Vt.lr0, c0,
                 At.cols, ae + r0, ve + c0, a + (size_t)r0 * At.ld + c0, At.ld,
                 min(kTcM, At.rows - r0), min(kOzN, At.cols - c0), 1 << 30, true))
      return false;
  }
  return true;
}

}  // namespace
}  // namespace spx
