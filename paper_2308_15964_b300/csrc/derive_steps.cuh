// Device steps of the dependency derivation, shared by the derivation
// kernels.  One CTA (kDeriveThreads threads unless given) runs every step; block
// barriers separate the steps.  See derive.cu for the model and the steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.h"

namespace spx {
namespace {

constexpr int kDeriveThreads = 1024;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// In-place exclusive scan of a[0..n) by the whole CTA of NT threads
// (sh: NT/32 + 1 words); returns the total.  Every thread must call it.
template <int NT = kDeriveThreads>
__device__ uint32_t block_excl_scan(uint32_t* a, uint32_t n, uint32_t* sh) {
  constexpr int kItems = 4;
  constexpr int kWarps = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < n; base += NT * kItems) {
    uint32_t v[kItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t idx = base + tid * kItems + i;
      v[i] = idx < n ? a[idx] : 0u;
      sum += v[i];
    }
    const uint32_t incl = warp_incl_scan(sum);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = lane < kWarps ? sh[lane] : 0u;
      const uint32_t wi = warp_incl_scan(w);
      if (lane < kWarps) sh[lane] = wi - w;
      if (lane == kWarps - 1) sh[kWarps] = wi;
    }
    __syncthreads();
    uint32_t run = carry + sh[warp] + incl - sum;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t idx = base + tid * kItems + i;
      if (idx < n) a[idx] = run;
      run += v[i];
    }
    carry += sh[kWarps];
    __syncthreads();
  }
  return carry;
}

// A list entry opens a new group unless it continues a run of READs, of
// COMMUTATIVE_WRITEs or of ATOMIC_WRITEs; a WRITE or MAYBE_WRITE is a group of
// its own.
__device__ __forceinline__ bool group_start(const DevGraph& g, uint32_t p) {
  const uint8_t m = g.s_mode[p];
  return g.s_first[p] || m == SPX_WRITE || m == SPX_MAYBE_WRITE || m != g.s_mode[p - 1];
}

// Unique successors of task u: merge of the next-group ranges of its
// accesses.  With col == nullptr only counts; else writes col[0..] and bumps
// the successors' in-degrees.
__device__ uint32_t merge_successors(const DevGraph& g, uint32_t u, uint32_t ngroups,
                                     uint32_t* col) {
  uint32_t a[kMaxHandles], b[kMaxHandles];
  const uint32_t r0 = g.task_rec[u], r1 = g.task_rec[u + 1];
  const int k = (int)(r1 - r0);
  for (int i = 0; i < k; ++i) {
    const uint32_t p = g.rec_pos[r0 + i];
    const uint32_t gi = g.gid[p];
    a[i] = b[i] = 0;
    if (gi + 1 < ngroups) {
      const uint32_t q = g.gpos[gi + 1];
      if (!g.s_first[q]) {  // next group on the same handle
        a[i] = q;
        b[i] = g.gpos[gi + 2];
      }
    }
  }
  uint32_t count = 0;
  for (;;) {
    uint32_t mn = 0xFFFFFFFFu;
    for (int i = 0; i < k; ++i)
      if (a[i] < b[i]) mn = min(mn, g.s_task[a[i]]);
    if (mn == 0xFFFFFFFFu) break;
    if (col) {
      col[count] = mn;
      atomicAdd(&g.indeg[mn], 1u);
    }
    ++count;
    for (int i = 0; i < k; ++i)
      if (a[i] < b[i] && g.s_task[a[i]] == mn) ++a[i];
  }
  return count;
}

// Steps 1-4: per-handle lists, groups, unique successors (row_ptr, col,
// indeg).  Reads rec_*, task_rec; uses hptr, s_task, s_mode, s_first,
// rec_pos, gid, gpos as scratch.  The edge total E is summed in 64 bits
// before any scan: E can exceed 2^32 for valid inputs (65536 READs followed by
// 65536 COMMUTATIVE_WRITEs on one handle give 2^32 edges).  Returns false,
// with row_ptr[ntasks] = E (0xFFFFFFFF when E does not fit 32 bits) and col /
// indeg not written, when E > ecap.  Every thread must call it.
// Steps 1-4 run by a CTA of NT threads (sh: NT/32 + 1 words).
template <int NT = kDeriveThreads>
__device__ bool derive_dag(const DevGraph& g, uint32_t* sh) {
  __shared__ unsigned long long e_total;
  const uint32_t N = g.ntasks, H = g.ntiles, M = g.nrec;
  const int tid = threadIdx.x;

  // 1. accesses per handle -> list offsets
  for (uint32_t i = tid; i <= H; i += NT) g.hptr[i] = 0;
  if (tid == 0) e_total = 0;
  __syncthreads();
  for (uint32_t r = tid; r < M; r += NT) atomicAdd(&g.hptr[g.rec_handle[r]], 1u);
  __syncthreads();
  block_excl_scan<NT>(g.hptr, H + 1, sh);
  __syncthreads();

  // 2. per-handle lists in insertion order
  for (uint32_t u = tid; u < N; u += NT) {
    for (uint32_t r = g.task_rec[u]; r < g.task_rec[u + 1]; ++r) {
      const uint32_t seq = g.rec_seq[r];
      const uint32_t p = g.hptr[g.rec_handle[r]] + seq;
      g.s_task[p] = u;
      g.s_mode[p] = g.rec_mode[r];
      g.s_first[p] = seq == 0 ? 1 : 0;
      g.rec_pos[r] = p;
    }
  }
  __syncthreads();

  // 3. groups
  for (uint32_t p = tid; p < M; p += NT) g.gid[p] = group_start(g, p) ? 1u : 0u;
  __syncthreads();
  const uint32_t G = block_excl_scan<NT>(g.gid, M, sh);
  __syncthreads();
  for (uint32_t p = tid; p < M; p += NT) {
    const bool f = group_start(g, p);
    const uint32_t gi = g.gid[p] + (f ? 1u : 0u) - 1u;
    g.gid[p] = gi;
    if (f) g.gpos[gi] = p;
  }
  if (tid == 0) g.gpos[G] = M;
  __syncthreads();

  // 4. unique successors: count (64-bit total), scan, write
  unsigned long long mine = 0;
  for (uint32_t u = tid; u < N; u += NT) {
    const uint32_t c = merge_successors(g, u, G, nullptr);
    g.row_ptr[u] = c;
    mine += c;
  }
  if (tid == 0) g.row_ptr[N] = 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((tid & 31) == 0 && mine) atomicAdd(&e_total, mine);
  __syncthreads();
  const unsigned long long E = e_total;
  if (E <= 0xFFFFFFFFull) {
    block_excl_scan<NT>(g.row_ptr, N + 1, sh);
  } else if (tid == 0) {
    g.row_ptr[N] = 0xFFFFFFFFu;
  }
  __syncthreads();
  if (E > (unsigned long long)g.ecap) return false;
  for (uint32_t i = tid; i < N; i += NT) g.indeg[i] = 0;
  __syncthreads();
  for (uint32_t u = tid; u < N; u += NT) merge_successors(g, u, G, g.col + g.row_ptr[u]);
  __syncthreads();
  return true;
}

}  // namespace
}  // namespace spx
