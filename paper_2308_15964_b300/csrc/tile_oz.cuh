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
// Tensor-core units (run by the one-CTA-per-SM instance of the persistent
// kernel, which owns all 512 TMEM columns): 128 output rows x 64 output
// columns, eight FP32 accumulators of 64 columns, accumulator d at column
// 64 d.  For each 16-wide K step, digit plane s of A (128 x 16) multiplies
// the planes t = 0..7-s of B stacked along N (64 (8 - s) rows, at most 256
// per MMA) with output block t landing in accumulator s + t.  The K step's
// operands (8 planes x 128 rows of A, 8 planes x 64 rows of B, 48 KB) arrive
// by one 5-D TMA box each (32-byte swizzle), three stages.  Up to eight
// column blocks of one row block form a pipelined group: the drain of a
// block's accumulators and its read-modify-write overlap the next block's
// loads and MMAs.  Measured in isolation (a harness running the same code):
// the operand traffic is the bound, the L2-to-SM rate near 7.3 TB/s on this
// GPU; 128 x 64 blocks read 40 % fewer operand bytes per flop than 128 x 32.
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

// 8 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes; the
// registers are valid after tmem_wait4 (several loads share one wait).
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}

// Wait for the warp's TMEM loads; the four 8-register groups pass through an
// empty statement after the wait so that no use of them moves above it.
__device__ __forceinline__ void tmem_wait4(uint32_t (*v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int d = 0; d < 4; ++d)
    asm volatile(""
                 : "+r"(v[d][0]), "+r"(v[d][1]), "+r"(v[d][2]), "+r"(v[d][3]), "+r"(v[d][4]),
                   "+r"(v[d][5]), "+r"(v[d][6]), "+r"(v[d][7]));
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

// The eight balanced base-128 digits sigma_0..7 of X (|X| <= 2^55) as the
// FP32 bit patterns of their values: the bottom four from the low 28 bits
// of X, the top four from X >> 28 plus the carry left by the bottom ones,
// in 32-bit integers.  The same digits as peeling X from the bottom in 64
// bits: a digit only depends on its remainder mod 128, and X = (X >> 28)
// 2^28 + (X mod 2^28) with 2^28 a multiple of 128^4.  The upper half of
// each pattern is the digit's BF16 encoding (|sigma| <= 64: exact).
__device__ __forceinline__ void oz_digits(long long X, uint32_t* fb) {
  int lo = (int)((unsigned long long)X & 0x0FFFFFFFull);
  int hi = (int)(X >> 28);
#pragma unroll
  for (int s = kOzPlanes - 1; s >= 4; --s) {
    const int d = ((lo + 64) & 127) - 64;
    fb[s] = __float_as_uint((float)d);
    lo = (lo - d) >> 7;
  }
  hi += lo;  // 0 or 1
#pragma unroll
  for (int s = 3; s >= 1; --s) {
    const int d = ((hi + 64) & 127) - 64;
    fb[s] = __float_as_uint((float)d);
    hi = (hi - d) >> 7;
  }
  fb[0] = __float_as_uint((float)hi);
}

// Split rows [64 u, 64 u + 64) of the FP64 tile Lt into its slot (lowp =
// slot address, lowp_ld = pitch b <= 512).  Columns cols..b-1 of each digit
// plane are written as zeros (the K padding the tensor cores read).  A warp
// per row: the row is read coalesced (column lane + 32 j) and its exponent
// reduced over the warp, the row is staged in shared memory (one double of
// skew per 16 columns, so that a lane's 16 consecutive columns fall in
// distinct banks), and lane i then splits the 16-digit K chunk i: its digits
// of one plane are the 32 contiguous bytes of the slot's (plane, chunk, row)
// run, written as two 16-byte stores.  scratch: kOzSplitStage doubles of
// shared memory per warp.
constexpr int kOzSplitStage = 544;  // 512 columns + 32 skew
__device__ __noinline__ void op_oz_split(const TileDesc& Lt, uint32_t u0, uint32_t u1,
                                         double* scratch) {
  // the descriptor's fields in registers (the stores below may alias it)
  const int b = Lt.lowp_ld, nch = b / 16, rows = Lt.rows, cols = Lt.cols, ld = Lt.ld;
  uint4* S = reinterpret_cast<uint4*>(Lt.lowp);
  int* Ex = reinterpret_cast<int*>(reinterpret_cast<char*>(Lt.lowp) + (size_t)16 * b * b);
  const double* A = reinterpret_cast<const double*>(Lt.ptr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* row = scratch + warp * kOzSplitStage;
  // this warp's rows of units u0..u1, the next row's loads in flight while
  // the current one is split
  auto load_row = [&](int r, unsigned long long* v) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = lane + 32 * j;
      v[j] = (c < cols)
                 ? (unsigned long long)__double_as_longlong(__ldcg(A + (size_t)r * ld + c))
                 : 0ull;
    }
  };
  auto next_row = [&](uint32_t& u, int r) {  // the row after r, or -1
    r += kThreads / 32;
    while (u < u1 && r >= min((int)(u + 1) * 64, rows)) {
      ++u;
      r = (int)u * 64 + warp;
    }
    return u < u1 ? r : -1;
  };
  uint32_t u = u0;
  int r = next_row(u, (int)u0 * 64 + warp - kThreads / 32);
  unsigned long long v[16];
  if (r >= 0) load_row(r, v);
  while (r >= 0) {
    unsigned long long mx = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = lane + 32 * j;
      if (c < b) {
        const unsigned long long mag = v[j] & 0x7FFFFFFFFFFFFFFFull;
        mx = mag > mx ? mag : mx;
        row[c + (c >> 4)] = __longlong_as_double((long long)v[j]);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
      mx = y > mx ? y : mx;
    }
    const int ef = (int)(mx >> 52);
    const int e = ef ? ef - 1022 : -1022;
    if (lane == 0) Ex[r] = e;
    const int rn = next_row(u, r);
    if (rn >= 0) load_row(rn, v);
    __syncwarp();
    if (lane < nch) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // 8 columns: one 16-byte store per plane
        uint32_t pk[kOzPlanes][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {  // two columns: one 32-bit word per plane
          const double* x = row + lane * 17 + 8 * h + i;
          uint32_t f0[kOzPlanes], f1[kOzPlanes];
          oz_digits(oz_fixed((unsigned long long)__double_as_longlong(x[0]), e), f0);
          oz_digits(oz_fixed((unsigned long long)__double_as_longlong(x[1]), e), f1);
#pragma unroll
          for (int s = 0; s < kOzPlanes; ++s) pk[s][i >> 1] = __byte_perm(f0[s], f1[s], 0x7632);
        }
#pragma unroll
        for (int s = 0; s < kOzPlanes; ++s)
          S[(((size_t)s * nch + lane) * b + r) * 2 + h] =
              make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
      }
    }
    __syncwarp();  // the staging row is reused
    r = rn;
  }
}

// Split the transpose of the FP64 tile Xt into its slot: slot row c is column
// c of Xt (exponent e_c = the column's), the K index is Xt's row, so that a
// product reading this slot as its B operand forms A Xt (the NN form of the
// tiled GEMM).  Unit u = columns [64 u, 64 u + 64); K indices rows..b-1 are
// written as zeros.  Warp w takes the 32 columns 64 u + 32 (w & 1) + lane and
// the 16-row K chunks j = w / 2, w / 2 + 4, ...: loads of one row are 256
// coalesced bytes, and one lane's 16 digits of a chunk and plane are the 32
// contiguous bytes of its slot row, so a warp's stores are 1 KB runs.  The
// column maximum is reduced over the four chunk warps through red (2 KB of
// shared memory, 4 x 64 words).
__device__ __noinline__ void op_oz_split_t(const TileDesc& Xt, uint32_t u0, uint32_t u1,
                                           unsigned long long* red) {
  // the descriptor's fields in registers (the stores below may alias it)
  const int b = Xt.lowp_ld, nch = b / 16, rows = Xt.rows, cols = Xt.cols, ld = Xt.ld;
  uint4* S = reinterpret_cast<uint4*>(Xt.lowp);  // 32 bytes = 2 x uint4 per (plane, chunk, row)
  int* Ex = reinterpret_cast<int*>(reinterpret_cast<char*>(Xt.lowp) + (size_t)16 * b * b);
  const double* A = reinterpret_cast<const double*>(Xt.ptr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = warp & 1, q = warp >> 1;
  for (uint32_t u = u0; u < u1; ++u) {
    const int c = (int)u * 64 + 32 * half + lane;
    const bool live = c < cols;
    unsigned long long mx = 0;
    for (int j = q; j < nch; j += 4) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int r = 16 * j + i;
        if (live && r < rows) {
          const unsigned long long mag =
              (unsigned long long)__double_as_longlong(__ldcg(A + (size_t)r * ld + c)) &
              0x7FFFFFFFFFFFFFFFull;
          mx = mag > mx ? mag : mx;
        }
      }
    }
    red[q * 64 + 32 * half + lane] = mx;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned long long y = red[k * 64 + 32 * half + lane];
      mx = y > mx ? y : mx;
    }
    __syncthreads();  // red is reused by the next unit
    const int ef = (int)(mx >> 52);
    const int e = ef ? ef - 1022 : -1022;
    if (!live) continue;  // slot rows past the tile's columns are never read
    if (q == 0) Ex[c] = e;
    for (int j = q; j < nch; j += 4) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // 8 rows: one 16-byte store per plane
        uint32_t pk[kOzPlanes][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {  // two rows: one 32-bit word per plane
          const int r = 16 * j + 8 * h + i;
          const unsigned long long b0 =
              r < rows
                  ? (unsigned long long)__double_as_longlong(__ldcg(A + (size_t)r * ld + c))
                  : 0ull;
          const unsigned long long b1 =
              r + 1 < rows ? (unsigned long long)__double_as_longlong(
                                    __ldcg(A + (size_t)(r + 1) * ld + c))
                              : 0ull;
          uint32_t f0[kOzPlanes], f1[kOzPlanes];
          oz_digits(oz_fixed(b0, e), f0);
          oz_digits(oz_fixed(b1, e), f1);
#pragma unroll
          for (int s = 0; s < kOzPlanes; ++s) pk[s][i >> 1] = __byte_perm(f0[s], f1[s], 0x7632);
        }
#pragma unroll
        for (int s = 0; s < kOzPlanes; ++s)
          S[(((size_t)s * nch + j) * b + c) * 2 + h] =
              make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
      }
    }
  }
}

// Shared-memory bytes of one K step of the split operands: 8 planes x (128
// rows of A + kN rows of B) x 16 digits.
__host__ __device__ constexpr int oz_stage_bytes(int kN) { return kOzPlanes * (kTcM + kN) * 32; }

// Bounded wait that also gives up once the CTA's error flag is set.
__device__ __forceinline__ bool mbar_wait_or_error(uint64_t* bar, uint32_t parity,
                                                   const volatile int* err) {
  for (uint32_t i = 0; i < kTcSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 1023u) == 1023u && *err) return false;
  }
  return false;
}

// Split-product unit of the one-CTA-per-SM kernel: nblk <= kOzGroup
// consecutive 128 x 64 output blocks of one row block, C[0:m, 0:n] -= A B^T
// (C at the first block; n counts columns from there).  Eight accumulators
// of 64 TMEM columns (all 512).  Per block:
//   thread 0   issues the block's TMA loads and MMAs (kS stages of 48 KB at
//              sb; the loads run kS - 1 steps ahead, across block
//              boundaries) and commits the block to s.done;
//   all warps  wait for it and drain the accumulators (warp w: TMEM lane
//              quarter w % 4, columns 32 (w / 4)..) into V (128 x 65
//              doubles): v formed in integers plus one FP64 addition;
//   warps 1-7  update the block from V (coalesced rows, a batch's loads
//              before its stores) while thread 0 issues the next block.
// V is free again when every warp has reached the next block's drain.
// Every wait is bounded; a timeout sets s.error and the loop finishes its
// blocks without work.
template <int kS>
__device__ bool oz_row_pipe(TcState& s, uint8_t* sb, double* V, const CUtensorMap* amap,
                            int a_slot, int a_r0, const CUtensorMap* bmap, int b_slot, int b_c0,
                            int nblk, int K, const int* a_exp, const int* b_exp, double* C,
                            int ldc, int m, int n, int diag, int wmode) {
  constexpr int kN = 64, kStage = oz_stage_bytes(kN), kStageA = kOzPlanes * kTcM * 32;
  static_assert(kStage % 1024 == 0 && kS <= kTcBars, "stages");
  constexpr int kLdv = kN + 1;
  const int nsteps = (K + 15) / 16, total = nblk * nsteps;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tmem = s.tmem_base;
  const uint32_t done0 = s.done_phase;
  const volatile int* err = &s.error;
  // thread 0's pipeline state
  uint32_t fph = s.full_phase, eph = s.empty_phase;
  int waited = 0;
  bool ok = true;
  auto issue = [&](int st, int g) {
    const int blk = g / nsteps, ks = g % nsteps;
    uint8_t* dst = sb + st * kStage;
    mbar_arrive_expect_tx(&s.full[st], kStage);
    tma_load_5d(dst, amap, &s.full[st], a_r0, ks, a_slot);
    tma_load_5d(dst + kStageA, bmap, &s.full[st], b_c0 + kN * blk, ks, b_slot);
  };
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const int pre = total < kS ? total : kS;
    for (int g = 0; g < pre; ++g) issue(g, g);
  }
  const int r = 32 * (warp & 3) + lane;  // drain: TMEM lane = output row
  const int cq = 32 * (warp >> 2);       // drain: this warp's 32 columns
  const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const int er = r < m ? a_exp[r] : 0;
  for (int blk = 0; blk < nblk; ++blk) {
    if (tid == 0 && ok) {
      for (int ks = 0; ks < nsteps && ok; ++ks) {
        const int g = blk * nsteps + ks, st = g % kS;
        ok = mbar_wait(&s.full[st], (fph >> st) & 1u);
        fph ^= 1u << st;
        if (!ok) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(sb + st * kStage), b0 = a0 + kStageA;
        // plane p of A times planes t = 0..7-p of B stacked along N, output
        // block t into accumulator p + t; at most 256 columns per MMA
#pragma unroll
        for (int p = 0; p < kOzPlanes; ++p) {
#pragma unroll
          for (int t0 = 0; t0 < kOzPlanes - p; t0 += 256 / kN) {
            const int nt = (kOzPlanes - p - t0) < 256 / kN ? (kOzPlanes - p - t0) : 256 / kN;
            oz_mma(tmem + (uint32_t)(kN * (p + t0)), oz_desc(a0 + (uint32_t)(p * kTcM * 32)),
                   oz_desc(b0 + (uint32_t)(t0 * kN * 32)), oz_idesc((uint32_t)(kN * nt)),
                   (ks > 0 || p > 0) ? 1u : 0u);
          }
        }
        tc_commit(&s.empty[st]);
        if (ks == nsteps - 1) tc_commit(&s.done);  // the block's accumulators complete
        const int pc = g - 1;
        if (pc >= 0 && pc + kS < total) {
          const int ps = pc % kS;
          ok = mbar_wait(&s.empty[ps], (eph >> ps) & 1u);
          eph ^= 1u << ps;
          waited = pc + 1;
          if (!ok) break;
          issue(ps, pc + kS);
        }
      }
      if (!ok) s.error = 1;
    }
    __syncthreads();  // V free: the previous block's update is done
    {
      const bool got = mbar_wait_or_error(&s.done, (done0 + blk) & 1u, err);
      tc_fence_after();
      if (__all_sync(0xFFFFFFFFu, got && !*err)) {
#pragma unroll 1
        for (int cb = cq; cb < cq + 32; cb += 8) {
          // accumulators 0-3 (Fh), then 4-7 (Fl): four loads per wait
          long long fh[8], fl[8];
#pragma unroll
          for (int hl = 0; hl < 2; ++hl) {
            uint32_t v[4][8];
#pragma unroll
            for (int d = 0; d < 4; ++d)
              tmem_ld8_async(lanes + (uint32_t)(kN * (4 * hl + d) + cb), v[d]);
            tmem_wait4(v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              long long f = 0;
#pragma unroll
              for (int d = 0; d < 4; ++d) f = f * 128 + __float2int_rn(__uint_as_float(v[d][j]));
              if (hl == 0) fh[j] = f;
              else fl[j] = f;
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = kN * blk + cb + j;
            double v = 0.0;
            if (r < m && c < n) {
              const int x = er + b_exp[c] - 61;
              double vh, vl;
              if (oz_i2d(fh[j], 28 + x, vh) && oz_i2d(fl[j], x, vl))
                v = __dadd_rn(vh, vl);
              else
                v = scalbn(__fma_rn(__ll2double_rn(fh[j]), 268435456.0, __ll2double_rn(fl[j])), x);
            }
            V[r * kLdv + cb + j] = v;
          }
        }
      } else if (lane == 0) {
        s.error = 1;
      }
      tc_fence_before();
    }
    __syncthreads();  // V ready; the accumulators are free for the next block
    if (warp >= 1 && !*err) {
      constexpr int kBatch = 8;
      for (int e0 = tid - 32; e0 < kTcM * kN; e0 += 224 * kBatch) {
        double cv[kBatch];
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          const int e = e0 + 224 * i, rr = e / kN, c = e % kN, cg = kN * blk + c;
          cv[i] = (wmode != 1 && e < kTcM * kN && rr < m && cg < n && cg <= rr + diag)
                      ? C[(size_t)rr * ldc + cg]
                      : 0.0;
        }
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
          const int e = e0 + 224 * i, rr = e / kN, c = e % kN, cg = kN * blk + c;
          if (e < kTcM * kN && rr < m && cg < n && cg <= rr + diag)
            C[(size_t)rr * ldc + cg] = wmode == 1   ? V[rr * kLdv + c]  // store
                                       : wmode == 2 ? __dadd_rn(cv[i], V[rr * kLdv + c])
                                                    : __dsub_rn(cv[i], V[rr * kLdv + c]);
        }
      }
    }
  }
  if (tid == 0) {
    for (int g = waited; g < total && ok; ++g) {  // consume the stage-free phases
      const int st = g % kS;
      ok = mbar_wait(&s.empty[st], (eph >> st) & 1u);
      eph ^= 1u << st;
    }
    s.full_phase = fph;
    s.empty_phase = eph;
    s.done_phase = done0 ^ ((uint32_t)nblk & 1u);
    if (!ok) s.error = 1;
  }
  __syncthreads();
  return !s.error;
}

// Write modes of a split product into its FP64 output.
constexpr int kOzSub = 0, kOzStore = 1, kOzAdd = 2;

// Shared-memory layout of the split ops in the one-CTA-per-SM kernel:
// three operand stages, then the staging of one finished block.
constexpr int kOzPipeStages = 3;
struct __align__(1024) OzBuf {
  uint8_t stages[kOzPipeStages][oz_stage_bytes(64)];
  double v[kTcM][65];  // also the split's row staging (kOzSplitStage per warp)
};
static_assert(sizeof(OzBuf::v) >= sizeof(double) * kOzSplitStage * (kThreads / 32), "staging");

__device__ __forceinline__ const int* oz_exps(const TileDesc& t) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(t.lowp) +
                                      (size_t)16 * t.lowp_ld * t.lowp_ld);
}

// C (FP64, rows x cols) -= / = / += A B^T (wmode kOzSub / kOzStore / kOzAdd)
// from the slots of A and B, units u0..u1
// of oz_units (lower: SYRK's blocks; C's (0,0) is the output's).
__device__ __noinline__ bool oz_product_units(const DevGraph& g, const TileDesc& At,
                                              const TileDesc& Bt, double* C, int ldc, int rows,
                                              int cols, bool lower, bool fine, int wmode,
                                              uint32_t u0, uint32_t u1, TcState* st, OzBuf* buf) {
  const int* ae = oz_exps(At);
  const int* be = oz_exps(Bt);
  for (uint32_t u = u0; u < u1; ++u) {
    uint32_t blk[3] = {0, 0, 0};
    oz_units(rows, cols, lower, fine, u, blk);
    const int r0 = (int)blk[0] * kTcM, c0 = (int)blk[1] * 64;
    if (!oz_row_pipe<kOzPipeStages>(*st, &buf->stages[0][0], &buf->v[0][0], g.maps + At.lmap,
                                    At.lr0, r0, g.maps + Bt.lmap + 1, Bt.lr0, c0, (int)blk[2],
                                    At.cols, ae + r0, be + c0, C + (size_t)r0 * ldc + c0, ldc,
                                    min(kTcM, rows - r0), cols - c0, lower ? r0 - c0 : 1 << 30,
                                    wmode))
      return false;
  }
  return true;
}

}  // namespace
}  // namespace spx
