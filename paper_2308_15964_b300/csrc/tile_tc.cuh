// Low-precision trailing updates on the 5th-generation tensor cores.
//
// One work unit = one 128 x 128 block of an FP64 tile C:
//     C[r0:r0+128, c0:c0+128] -= A_lo[ar0:ar0+128, 0:K] * B_lo[br0:br0+128, 0:K]^T
// where A_lo and B_lo are BF16 or TF32 copies of factor tiles (both K-major,
// i.e. row-major with K contiguous).  The operands arrive in shared memory by
// TMA (cp.async.bulk.tensor, 128-byte swizzle, one 128-row x 128-byte box per
// operand and K chunk, three stages), one thread issues tcgen05.mma
// (M = 128, N = 128, FP32 accumulation in TMEM, K = 16 for BF16 / 8 for
// TF32 per instruction), tcgen05.commit signals completion on mbarriers, and
// all eight warps read the accumulator back with tcgen05.ld and subtract it
// from the FP64 block (the paper's mixed-precision workload keeps the
// trailing matrix in FP64 and runs only the update products in low precision).
//
// Every wait on an mbarrier is bounded; on expiry the unit returns false and
// the caller reports an error (the TMEM allocation is released by the caller
// at kernel exit).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.h"

namespace spx {
namespace {

constexpr int kTcM = 128, kTcN = 128;
constexpr int kTcStages = 3;
constexpr int kTcChunkBytes = 128;                 // K bytes per stage (one swizzle row)
constexpr int kTcStageBytes = kTcM * kTcChunkBytes; // 16 KB per operand per stage
constexpr uint32_t kTcTmemCols = 128;              // FP32 accumulator columns
// TMEM columns a CTA of the persistent kernel allocates: the 128 x 128
// accumulator of a low-precision unit, or the eight 32-column accumulators of
// a split-FP64 unit (tile_oz.cuh).  Two CTAs per SM use all 512.
constexpr uint32_t kTcCtaCols = 256;
constexpr uint32_t kTcSpinLimit = 1u << 26;

// Operand stages (1024-byte aligned for the 128-byte swizzle atoms).  In the
// persistent kernel they share shared memory with the FP64 ops.
struct __align__(1024) TcBuf {
  uint8_t a[kTcStages][kTcStageBytes];
  uint8_t b[kTcStages][kTcStageBytes];
};

// Barriers and accumulator address; live for the whole kernel.
constexpr int kTcBars = 4;  // stage barrier pairs (the split unit of the one-CTA-per-SM kernel uses 4)

struct TcState {
  uint64_t full[kTcBars];   // TMA landed
  uint64_t empty[kTcBars];  // MMAs that read the stage finished
  uint64_t done;              // all MMAs of the unit finished
  uint32_t tmem_base, tmem_cols;
  uint32_t full_phase, empty_phase, done_phase;  // parity bit s = stage s
  int error;
};

// Exact FP32 -> FP64 widening from the IEEE-754 formats, on the integer
// pipe only, so that the epilogue's FP64 pipe (2 operations per clock per SM
// on this GPU) does nothing but the subtraction:
//   normal (1 <= e <= 254): sign, exponent e - 127 + 1023, mantissa << 29;
//   zero: the sign alone;
//   subnormal (e = 0, m != 0): m 2^-149 with m of bit length L = 32 - clz(m):
//     shift m left by s = 24 - L so its leading one sits at bit 23, then
//     exponent L - 150 + 1023 = 897 - s and the 23 bits below the leading one
//     as the mantissa;
//   infinity / NaN (e = 255): exponent 2047, mantissa << 29 (payload kept).
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  uint32_t e64, mm;
  if (e == 0u) {
    if (m == 0u) return __longlong_as_double((long long)sign);
    const uint32_t sh = (uint32_t)__clz(m) - 8u;
    e64 = 897u - sh;
    mm = (m << sh) & 0x7FFFFFu;
  } else {
    e64 = e == 0xFFu ? 2047u : e + 896u;
    mm = m;
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)e64 << 52) | ((unsigned long long)mm << 29)));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kTcSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core groups 1024 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, A and B of type `fmt` (1 = BF16
// for kind::f16, 2 = TF32 for kind::tf32), both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) |
         ((uint32_t)(kTcM >> 4) << 24);
}

template <bool kBf16>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  if (kBf16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(tc_idesc(1)), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(tc_idesc(2)), "r"(accumulate));
  }
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Allocate the CTA's accumulator columns (warp 0, all lanes) and initialise
// the barriers (thread 0).  Call once per kernel, before __syncthreads.
__device__ __forceinline__ void tc_setup(TcState& s, uint32_t cols = kTcCtaCols) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s.tmem_base)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    s.tmem_cols = cols;
    for (int i = 0; i < kTcBars; ++i) {
      mbar_init(&s.full[i], 1);
      mbar_init(&s.empty[i], 1);
    }
    mbar_init(&s.done, 1);
    s.full_phase = s.empty_phase = s.done_phase = 0;
    s.error = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
}

// Release the accumulator columns (warp 0).  Call once at kernel exit, after
// a __syncthreads that follows the last tcgen05 use.
__device__ __forceinline__ void tc_teardown(TcState& s) {
  tc_fence_after();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem_base),
                 "r"(s.tmem_cols));
  }
}

// One 128 x 128 unit (see the file comment).  m, n: valid rows / columns of
// the output block (<= 128); K: reduction length (elements); the A rows
// start at (ay, ax0) and the B rows at (by, bx0) in their tensor maps (x is
// the K coordinate).  lower: write only entries with column <= row.  All
// threads call it; returns false on a barrier timeout.
template <bool kBf16>
__device__ bool tc_gemm_unit(TcState& s, TcBuf& buf, const CUtensorMap* amap, int ax0, int ay,
                             const CUtensorMap* bmap, int bx0, int by, int K, double* C, int ldc,
                             int m, int n, bool lower) {
  constexpr int kElem = kBf16 ? 2 : 4;
  constexpr int kChunk = kTcChunkBytes / kElem;   // K elements per stage
  constexpr int kMmaK = kBf16 ? 16 : 8;           // K per instruction
  const int nchunks = (K + kChunk - 1) / kChunk;
  const int tid = threadIdx.x;
  const uint32_t tmem = s.tmem_base;
  // the stages may hold generic-proxy writes (the previous epilogue, or an
  // FP64 op's buffers that share this memory): order them before TMA writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid >= 32) {
    // while thread 0 drives TMA and the MMAs, pull the FP64 output block
    // into L2 for the epilogue (one prefetch per 128-byte line)
    const int lines_per_row = (n * 8 + 127) / 128;
    for (int e = tid - 32; e < m * lines_per_row; e += kThreads - 32) {
      const int r = e / lines_per_row, l = e % lines_per_row;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (size_t)r * ldc + l * 16));
    }
  }
  if (tid == 0) {
    tc_fence_after();
    bool ok = true;
    uint32_t fph = s.full_phase, eph = s.empty_phase;
    const int pre = nchunks < kTcStages ? nchunks : kTcStages;
    for (int c = 0; c < pre; ++c) {
      mbar_arrive_expect_tx(&s.full[c], 2 * kTcStageBytes);
      tma_load_2d(buf.a[c], amap, &s.full[c], ax0 + c * kChunk, ay);
      tma_load_2d(buf.b[c], bmap, &s.full[c], bx0 + c * kChunk, by);
    }
    int waited = 0;  // chunks whose stage-free (empty) phase has been consumed
    for (int c = 0; c < nchunks && ok; ++c) {
      const int st = c % kTcStages;
      ok = mbar_wait(&s.full[st], (fph >> st) & 1u);
      fph ^= 1u << st;
      if (!ok) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(buf.a[st]), b0 = smem_u32(buf.b[st]);
#pragma unroll
      for (int k = 0; k < kChunk / kMmaK; ++k) {
        tc_mma<kBf16>(tmem, smem_desc(a0 + k * kMmaK * kElem), smem_desc(b0 + k * kMmaK * kElem),
                      (c > 0 || k > 0) ? 1u : 0u);
      }
      tc_commit(&s.empty[st]);
      // refill the stage of the previous chunk (its MMAs were issued one
      // step earlier) while this chunk's MMAs run
      const int pc = c - 1;
      if (pc >= 0 && pc + kTcStages < nchunks) {
        const int ps = pc % kTcStages;
        ok = mbar_wait(&s.empty[ps], (eph >> ps) & 1u);
        eph ^= 1u << ps;
        waited = pc + 1;
        if (!ok) break;
        mbar_arrive_expect_tx(&s.full[ps], 2 * kTcStageBytes);
        tma_load_2d(buf.a[ps], amap, &s.full[ps], ax0 + (pc + kTcStages) * kChunk, ay);
        tma_load_2d(buf.b[ps], bmap, &s.full[ps], bx0 + (pc + kTcStages) * kChunk, by);
      }
    }
    tc_commit(&s.done);
    if (ok) ok = mbar_wait(&s.done, s.done_phase & 1u);
    s.done_phase ^= 1u;
    // consume the stage-free phases not waited on above, in chunk order
    for (int c = waited; c < nchunks && ok; ++c) {
      const int st = c % kTcStages;
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
  // epilogue, 1: accumulator -> shared memory (the operand stages are free
  // now).  Warp w reads TMEM lanes 32*(w%4).. (rows), columns 64*(w/4)..+64.
  constexpr int kLde = kTcN + 1;
  static_assert(sizeof(float) * kTcM * kLde <= sizeof(TcBuf), "epilogue staging fits the stages");
  float* E = reinterpret_cast<float*>(&buf);
  const int warp = tid >> 5, lane = tid & 31;
  {
    const int row = 32 * (warp & 3) + lane;
    const int col0 = 64 * (warp >> 2);
    float v[32];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int cb = col0 + 32 * h;
      tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) E[row * kLde + cb + j] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  // epilogue, 2: coalesced FP64 read-modify-write of the output block; each
  // warp loads 4 rows (4 columns per lane each) before writing any of them
  constexpr int kWarps = kThreads / 32;
  for (int r0 = warp; r0 < m; r0 += 4 * kWarps) {
    double cv[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + kWarps * k;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        cv[k][q] = (r < m && c < n && (!lower || c <= r)) ? __ldcg(C + (size_t)r * ldc + c) : 0.0;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + kWarps * k;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        if (r < m && c < n && (!lower || c <= r))
          C[(size_t)r * ldc + c] = cv[k][q] - widen_f32(E[r * kLde + c]);
      }
    }
  }
  __syncthreads();
  return true;
}

// FP64 -> two TF32 parts held in FP32 bit patterns: hi = x rounded to the 11
// significant bits of TF32 (to nearest, ties away from zero, as
// cvt.rna.tf32.f32), lo = (x rounded to FP32) - hi, rounded the same way;
// |x - hi - lo| <= 1.25 * 2^-22 |x|.  For x in the FP32 normal range both
// roundings are done on the integer pipe from the FP64 bit pattern (FP64
// operations run at 2 per clock per SM on this GPU) and the FP32 difference
// is exact (hi and x rounded to FP32 lie within a factor of two of each
// other); zeros, subnormals and values outside that range take the hardware
// conversions.
__device__ __forceinline__ void split_tf32(double x, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FFu) - 1023 + 127;
  float f;
  if (e >= 2 && e <= 252) {
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const uint32_t top = ((uint32_t)(b >> 63) << 31) | ((uint32_t)e << 23);
    hi = (top | ((uint32_t)(m >> 42) << 13)) + (((uint32_t)(m >> 41) & 1u) << 13);
    f = __uint_as_float((top | (uint32_t)(m >> 29)) + ((uint32_t)(m >> 28) & 1u));
  } else {
    f = __double2float_rn(x);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(f));
  }
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(f - __uint_as_float(hi)));
}

// TRSM by the inverse on the tensor cores, one block of m <= 128 rows of A:
//     A[0:m, 0:n] <- A[0:m, 0:n] V^T,   V = L^{-1} (n x n FP64, lower, zero
// above the diagonal; n a multiple of 32).  Every FP64 operand entry is split
// into TF32 hi + lo (split_tf32) and the accumulator collects hi*hi + hi*lo +
// lo*hi per K step (kind::tf32, M = N = 128, K = 8).  The 128-column output
// blocks run right to left: output column c needs input columns <= c only
// (V^T is upper triangular), so block c0 reads columns < c0 + 128, none of
// which a later block writes, and the update is in place.  Per 32-column K
// chunk all threads load the chunk (16 rows of A and of V per warp, one
// element per lane, all loads in flight together) and convert it into the
// four 128-byte-swizzled operand buffers; thread 0 issues the twelve MMAs and
// waits for them (bounded) before the buffers are rewritten.
// The epilogue writes the accumulator widened exactly to FP64 into A and its
// rounding (BF16 when kBf16, else TF32 in FP32 storage) into the
// low-precision copy (lowp, ld lowp_ld).  All threads; false on a timeout.
template <bool kBf16>
__device__ bool tc_trsm_inv_rows(TcState& s, TcBuf& buf, const double* V, int ldv, double* A,
                                 int lda, int m, int n, void* lowp, int lowp_ld) {
  constexpr int kChunk = 32;                          // K per chunk: 128 bytes of TF32
  constexpr int kRowsPerWarp = kTcM / (kThreads / 32);
  static_assert(kRowsPerWarp * (kThreads / 32) == kTcM, "rows per warp");
  uint8_t* const a_hi = buf.a[0];
  uint8_t* const a_lo = buf.a[1];
  uint8_t* const v_hi = buf.b[0];
  uint8_t* const v_lo = buf.b[1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tmem = s.tmem_base;
  constexpr int kLde = kTcN + 1;
  float* E = reinterpret_cast<float*>(&buf);
  for (int c0 = (n - 1) / kTcN * kTcN; c0 >= 0; c0 -= kTcN) {
    const int nc = min(kTcN, n - c0);
    const int nchunks = (c0 + nc) / kChunk;
    for (int c = 0; c < nchunks; ++c) {
      __syncthreads();  // the previous chunk's MMAs are done (thread 0 waited)
      if (s.error) return false;
      // rows warp, warp + 8, ... of the A block and of the V block (V rows
      // are the output columns c0 ..), element k0 + lane of each, stored
      // K-major with the 128-byte swizzle: the 16-byte group j of row r sits
      // at group j ^ (r mod 8) of the row (the layout TMA writes)
      const int k0 = c * kChunk;
#pragma unroll 4
      for (int i = 0; i < kRowsPerWarp; ++i) {
        const int r = warp + 8 * i;
        const double xa = r < m ? __ldcg(A + (size_t)r * lda + k0 + lane) : 0.0;
        const double xv = r < nc ? __ldcg(V + (size_t)(c0 + r) * ldv + k0 + lane) : 0.0;
        const uint32_t off =
            (uint32_t)r * 128u + ((((uint32_t)lane >> 2) ^ ((uint32_t)r & 7u)) << 4) +
            (((uint32_t)lane & 3u) << 2);
        uint32_t h, l;
        split_tf32(xa, h, l);
        *reinterpret_cast<uint32_t*>(a_hi + off) = h;
        *reinterpret_cast<uint32_t*>(a_lo + off) = l;
        split_tf32(xv, h, l);
        *reinterpret_cast<uint32_t*>(v_hi + off) = h;
        *reinterpret_cast<uint32_t*>(v_lo + off) = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
        const uint32_t vh = smem_u32(v_hi), vl = smem_u32(v_lo);
#pragma unroll
        for (int k = 0; k < kChunk / 8; ++k) {
          const uint32_t o = (uint32_t)k * 32u;  // 8 TF32 elements per K step
          tc_mma<false>(tmem, smem_desc(ah + o), smem_desc(vh + o), (c > 0 || k > 0) ? 1u : 0u);
          tc_mma<false>(tmem, smem_desc(ah + o), smem_desc(vl + o), 1u);
          tc_mma<false>(tmem, smem_desc(al + o), smem_desc(vh + o), 1u);
        }
        tc_commit(&s.done);
      }
      if (tid == 0) {
        if (!mbar_wait(&s.done, s.done_phase & 1u)) s.error = 1;
        s.done_phase ^= 1u;
      }
    }
    __syncthreads();
    if (s.error) return false;
    tc_fence_after();
    {  // accumulator -> shared memory, as in tc_gemm_unit
      const int row = 32 * (warp & 3) + lane;
      const int col0 = 64 * (warp >> 2);
      float v[32];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = col0 + 32 * h;
        tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) E[row * kLde + cb + j] = v[j];
      }
    }
    tc_fence_before();
    __syncthreads();
    for (int e = tid; e < m * nc; e += kThreads) {
      const int r = e / nc, c = e % nc;
      const float v = E[r * kLde + c];
      A[(size_t)r * lda + c0 + c] = widen_f32(v);
      if (kBf16) {
        reinterpret_cast<__nv_bfloat16*>(lowp)[(size_t)r * lowp_ld + c0 + c] = __float2bfloat16_rn(v);
      } else {
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
        reinterpret_cast<uint32_t*>(lowp)[(size_t)r * lowp_ld + c0 + c] = t;
      }
    }
    __syncthreads();
  }
  return true;
}

}  // namespace
}  // namespace spx

namespace spx {
namespace {

// Shared-memory context of the tensor-core ops inside the persistent kernel.
struct OzBuf;

struct TcCtx {
  TcState* st;
  TcBuf* buf;
  OzBuf* oz;  // the same memory, laid out for the split ops (one-CTA-per-SM instance)
};

// SYRK on the tensor cores: C (n x n, FP64, lower) -= L_lo L_lo^T; units are
// the lower 128-block pairs of C.
template <bool kBf16>
__device__ bool op_tc_syrk(const DevGraph& g, const TileDesc& Lt, const TileDesc& Ct, uint32_t u0,
                           uint32_t u1, TcCtx& tc) {
  double* c = (double*)Ct.ptr;
  const CUtensorMap* map = g.maps + Lt.lmap;
  for (uint32_t u = u0; u < u1; ++u) {
    int i = 0;
    while ((uint32_t)((i + 1) * (i + 2) / 2) <= u) ++i;
    const int bi = i, bj = (int)(u - (uint32_t)(i * (i + 1) / 2));
    const int r0 = bi * kTcM, c0 = bj * kTcN;
    if (!tc_gemm_unit<kBf16>(*tc.st, *tc.buf, map, Lt.lc0, Lt.lr0 + r0, map, Lt.lc0, Lt.lr0 + c0,
                             Lt.cols, c + (size_t)r0 * Ct.ld + c0, Ct.ld, min(kTcM, Ct.rows - r0),
                             min(kTcN, Ct.cols - c0), bi == bj))
      return false;
  }
  return true;
}

// GEMM on the tensor cores: C (m x n, FP64) -= A_lo B_lo^T; units are the
// 128 x 128 blocks of C, row-major.
template <bool kBf16>
__device__ bool op_tc_gemm(const DevGraph& g, const TileDesc& At, const TileDesc& Bt,
                           const TileDesc& Ct, uint32_t u0, uint32_t u1, TcCtx& tc) {
  double* c = (double*)Ct.ptr;
  const uint32_t nbc = cdiv128(Ct.cols);
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)(u / nbc) * kTcM, c0 = (int)(u % nbc) * kTcN;
    if (!tc_gemm_unit<kBf16>(*tc.st, *tc.buf, g.maps + At.lmap, At.lc0, At.lr0 + r0,
                             g.maps + Bt.lmap, Bt.lc0, Bt.lr0 + c0, At.cols,
                             c + (size_t)r0 * Ct.ld + c0, Ct.ld, min(kTcM, Ct.rows - r0),
                             min(kTcN, Ct.cols - c0), false))
      return false;
  }
  return true;
}

// TRSM_INV on the tensor cores: A_ik <- A_ik V^T, units are the 128-row
// blocks of A_ik (see tc_trsm_inv_rows).  Not inlined: it keeps its
// registers out of the persistent kernel's main loop.
template <bool kBf16>
__device__ __noinline__ bool op_tc_trsm_inv(const TileDesc& Vt, const TileDesc& At, uint32_t u0,
                                            uint32_t u1, TcCtx& tc) {
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)u * kTcM;
    char* lowp = (char*)At.lowp + (size_t)r0 * At.lowp_ld * (kBf16 ? 2 : 4);
    if (!tc_trsm_inv_rows<kBf16>(*tc.st, *tc.buf, (const double*)Vt.ptr, Vt.ld,
                                 (double*)At.ptr + (size_t)r0 * At.ld, At.ld,
                                 min(kTcM, At.rows - r0), At.cols, lowp, At.lowp_ld))
      return false;
  }
  return true;
}

// Low-precision copy of 64-row blocks u0..u1 of a FP64 tile: BF16 by
// round-to-nearest-even, or TF32 (FP64 -> FP32 nearest, then cvt.rna.tf32)
// kept in FP32 storage.
template <bool kBf16>
__device__ void op_lowp_copy(const TileDesc& At, uint32_t u0, uint32_t u1) {
  const double* a = (const double*)At.ptr;
  for (uint32_t u = u0; u < u1; ++u) {
    const int r0 = (int)u * kBlk, mb = min(kBlk, At.rows - r0);
    for (int e = threadIdx.x; e < mb * At.cols; e += kThreads) {
      const int r = r0 + e / At.cols, c = e % At.cols;
      const double v = __ldcg(a + (size_t)r * At.ld + c);
      if (kBf16) {
        ((__nv_bfloat16*)At.lowp)[(size_t)r * At.lowp_ld + c] = __double2bfloat16(v);
      } else {
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(__double2float_rn(v)));
        ((uint32_t*)At.lowp)[(size_t)r * At.lowp_ld + c] = t;
      }
    }
  }
}

}  // namespace
}  // namespace spx
