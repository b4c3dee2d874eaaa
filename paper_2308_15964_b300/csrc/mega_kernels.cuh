// Persistent device-scheduled executor and the one-launch-per-task baseline
// (device code; each kernel instantiation is compiled in its own file,
// mega_k_*.cu, and launched from mega.cu).
//
// Scheduling model (Specx paper, section "Scheduling"): ready tasks are pushed
// into a scheduler and idle workers pop them.  Here the workers are
// persistent CTAs (two per SM) and the scheduler is three FIFO queues in HBM,
// popped in order: critical path, high and normal priority (section "Task
// insertion": priorities are a hint the scheduler may use).  A task runs in
// phases, each split into parts (independent sub-tile pieces); a queue entry
// is one phase of one task.
//
//   pop    thread 0: take part p of an entry near the queue head (a
//          pseudo-random one of the first 16, so that idle CTAs do not all
//          race for one slot) with an atomicAdd on the slot's claim counter
//          (bounded wait for an entry that is reserved but not yet written);
//          the head moves only over slots whose parts are all claimed.
//   run    all 256 threads execute the part's tile op.
//   finish a part decrements the task's remaining-part counter; the CTA that
//          finishes the last part of a phase publishes the next phase and
//          runs its part 0 itself; after the last phase, warp 0 decrements the
//          successors' in-degree counters (one lane per successor), ballots
//          the ones that reached zero and reserves their queue entries with
//          one atomicAdd per queue for the whole warp.
//
// Memory order: the writes of a part are published by __syncthreads +
// __threadfence before the counter decrement; the releasing CTA fences again
// before writing queue entries; a popping CTA fences after reading an entry.
// Tile data are read with ld.global.cg.
//
// Every wait is bounded: a watchdog on the time since the last finished part
// sets SPX_ERR_TIMEOUT and the abort flag, and every CTA drains and exits.
// COMMUTATIVE_WRITE tasks run as one part and take per-tile locks in
// ascending handle order before running (the paper locks data handles sorted
// by address, section "Internal implementation"); a lock is held only by a
// running task, so the ordered wait cannot deadlock.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "derive_steps.cuh"
#include "spx_internal.h"
#include "tile_f64.cuh"
#include "tile_tc.cuh"
#include "tile_oz.cuh"

namespace spx {
namespace {

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %smid;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *(const volatile uint32_t*)p;
}

// Task descriptors and access records are read from L2 (ld.global.cg): in
// stream mode they are uploaded while the kernel runs, and a line cached in
// an SM's L1 from an earlier batch may hold older bytes of them.
__device__ __forceinline__ TaskDesc load_task(const TaskDesc* p) {
  static_assert(sizeof(TaskDesc) == 32, "two 16-byte loads");
  const uint4 a = __ldcg(reinterpret_cast<const uint4*>(p));
  const uint4 b = __ldcg(reinterpret_cast<const uint4*>(p) + 1);
  TaskDesc t;
  uint4* d = reinterpret_cast<uint4*>(&t);
  d[0] = a;
  d[1] = b;
  return t;
}

__device__ __forceinline__ void set_error(RunState* rs, uint32_t code, int info) {
  if (atomicCAS(&rs->status, 0u, code) == 0u) rs->info = info;
  atomicExch(&rs->abort, 1u);
}

// Expired when the last finished part is older than the watchdog.  The stamp
// may come from another SM whose %globaltimer reading is slightly ahead of
// ours, so the difference is signed (a negative age is not a stall).
__device__ __forceinline__ bool watchdog_expired(const DevGraph& g) {
  const uint32_t last = ld_volatile(&g.rs->progress.v);
  const uint32_t now = (uint32_t)(globaltimer() >> 10);  // ~1 us units
  return (int32_t)(now - last) > (int32_t)(g.watchdog_ns >> 10);
}

__device__ __forceinline__ void touch_progress(const DevGraph& g) {
  *(volatile uint32_t*)&g.rs->progress.v = (uint32_t)(globaltimer() >> 10);
}

// Claims are spread over the first entries of a queue: when tasks have one
// part, every idle CTA reading the head slot would race for the same entry,
// and one claim per L2 atomic round trip (about 0.7 us) would be handed out.
constexpr uint32_t kPopSpread = 16;  // a pop starts at one of the first 16 entries
constexpr uint32_t kPopScan = 64;    // entries looked at per queue and attempt

// Wait (bounded) for the entry of slot h, reserved by a pusher that may still
// be writing it.  False on abort or timeout.
__device__ bool entry_at(const DevGraph& g, int q, uint32_t h, uint32_t& v) {
  uint32_t spins = 0;
  while ((v = ld_volatile(&g.queue[q][h])) == kEmpty) {
    if ((++spins & 1023u) == 0) {
      if (ld_volatile(&g.rs->abort)) return false;
      if (watchdog_expired(g)) {
        set_error(g.rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
        return false;
      }
    }
  }
  return true;
}

// Move the head of queue q over the slots whose parts are all claimed; it
// never passes a slot with parts left.
__device__ void advance_head(const DevGraph& g, int q, uint32_t t) {
  uint32_t h = ld_volatile(&g.rs->head[q].v);
  while (h < t) {
    const uint32_t v = ld_volatile(&g.queue[q][h]);
    if (v == kEmpty || ld_volatile(&g.qclaim[q][h]) < (v & (kMaxParts - 1u)) + 1u) break;
    atomicMax(&g.rs->head[q].v, h + 1u);
    ++h;
  }
}

// Pop one queue entry (task << 8 | part), or kExit.  Called by one thread;
// rnd is the CTA's pseudo-random state for the start of the scan.
constexpr uint32_t kAdmit = 0xFFFFFFFCu;  // pop result: tasks claimed for admission (stream)
constexpr uint32_t kAdmitBatch = 64;     // tasks per admission claim

__device__ uint32_t pop(const DevGraph& g, uint32_t& empties, uint32_t& rnd, uint32_t* adm) {
  RunState* rs = g.rs;
  uint32_t backoff = 32;
  uint32_t iter = 0;
  for (;;) {
    if (ld_volatile(&rs->abort)) return kExit;
    if (g.sctl) {  // stream: admit newly published tasks first
      const uint32_t pub = ld_volatile(&g.sctl->published);
      uint32_t c = ld_volatile(&rs->admit_claim.v);
      while (c < pub) {
        const uint32_t e = min(pub, c + kAdmitBatch);
        const uint32_t prev = atomicCAS(&rs->admit_claim.v, c, e);
        if (prev == c) {
          adm[0] = c;
          adm[1] = e;
          return kAdmit;
        }
        c = prev;
      }
    }
    for (int q = 0; q < kQueues; ++q) {
      const uint32_t h0 = ld_volatile(&rs->head[q].v);
      const uint32_t t = min(ld_volatile(&rs->tail[q].v), g.qcap);
      if (h0 >= t) continue;
      // Slots h0.. hold one phase of a task each; its parts are claimed with
      // atomicAdd on the slot's counter.
      const uint32_t n = min(t - h0, kPopScan);
      rnd = rnd * 1664525u + 1013904223u;
      const uint32_t start = (rnd >> 16) % min(n, kPopSpread);
      for (uint32_t i = 0; i < n; ++i) {
        const uint32_t h = h0 + (start + i) % n;
        uint32_t v;
        if (!entry_at(g, q, h, v)) return kExit;
        const uint32_t np = (v & (kMaxParts - 1u)) + 1u;
        if (ld_volatile(&g.qclaim[q][h]) >= np) continue;  // exhausted: no atomic
        const uint32_t p = atomicAdd(&g.qclaim[q][h], 1u);
        if (p < np) {
          if (p + 1u == np) advance_head(g, q, t);
          __threadfence();
          return (v & ~(kMaxParts - 1u)) | p;
        }
      }
      advance_head(g, q, t);  // every entry looked at was taken
    }
    if (g.sctl) {
      // stream: leave once the host has ended it and every published task
      // was admitted and has finished
      if (ld_volatile(&g.sctl->end)) {
        const uint32_t pub = ld_volatile(&g.sctl->published);
        if (ld_volatile(&rs->admitted.v) >= pub && ld_volatile(&rs->done.v) >= pub) return kExit;
      }
    } else if (ld_volatile(&rs->done.v) >= g.ntasks) {
      return kExit;
    }
    ++empties;
    __nanosleep(backoff);
    if (backoff < 1024) backoff <<= 1;
    if ((++iter & 63u) == 0 && watchdog_expired(g)) {
      set_error(rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
      return kExit;
    }
  }
}

// Warp 0: push one queue entry (phase 0 of task s, np parts) for each lane
// with ready set, one atomicAdd per queue for the whole warp.
__device__ void push_ready_warp(const DevGraph& g, bool ready, uint32_t s, uint32_t np,
                                uint32_t pq) {
  const int lane = threadIdx.x & 31;
  __threadfence();  // order the predecessors' data before the queue entries
  for (uint32_t q = 0; q < (uint32_t)kQueues; ++q) {
    const bool mine = ready && pq == q;
    const uint32_t cnt = mine ? 1u : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    uint32_t slot = 0;
    if (lane == 0) {
      slot = atomicAdd(&g.rs->tail[q].v, total);
      atomicMax(&g.rs->hiwater, slot + total);
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot + total > g.qcap) {
      if (lane == 0) set_error(g.rs, (uint32_t)SPX_ERR_QUEUE_FULL, 0);
      continue;
    }
    if (mine) *(volatile uint32_t*)&g.queue[q][slot + incl - 1] = (s << kPartBits) | (np - 1);
  }
}

// Release the successors of a finished task (warp 0, all 32 lanes).
__device__ void release(const DevGraph& g, uint32_t task) {
  const int lane = threadIdx.x & 31;
  const uint32_t r0 = g.row_ptr[task], r1 = g.row_ptr[task + 1];
  for (uint32_t base = r0; base < r1; base += 32) {
    const uint32_t idx = base + lane;
    bool ready = false;
    uint32_t s = 0, np = 0, pq = 0;
    if (idx < r1) {
      s = g.col[idx];
      ready = atomicSub(&g.indeg_w[s], 1u) == 1u;
      if (ready) {
        const TaskDesc ts = load_task(&g.tasks[s]);
        np = ts.nparts;
        pq = graph_queue(ts.prio);
      }
    }
    push_ready_warp(g, ready, s, np, pq);
  }
}

// Stream mode, warp 0: admit tasks a0..a1-1.  Per task (one lane): a guard
// count of 1 on its remaining predecessors, then for each predecessor p a
// count of 1 and a slot on p's successor list; when p has finished already
// (its slot count is closed) the count is taken back.  Dropping the guard
// last makes the task ready exactly once: here when every predecessor had
// finished, else in the release of its last predecessor.
__device__ void admit_tasks(const DevGraph& g, uint32_t a0, uint32_t a1) {
  const int lane = threadIdx.x & 31;
  for (uint32_t base = a0; base < a1; base += 32) {
    const uint32_t v = base + lane;
    bool ready = false;
    uint32_t np = 0, pq = 0;
    if (v < a1) {
      const TaskDesc t = load_task(&g.tasks[v]);
      g.remaining[v] = t.nparts;
      g.phase[v] = 0;
      g.indeg_w[v] = 1u;
      __threadfence();
      const uint32_t i1 = __ldcg(&g.pred_ptr[v + 1]);
      for (uint32_t i = __ldcg(&g.pred_ptr[v]); i < i1; ++i) {
        const uint32_t p = __ldcg(&g.pred[i]);
        atomicAdd(&g.indeg_w[v], 1u);
        const uint32_t old = atomicAdd(&g.succ_cnt[p], 1u);
        if ((old & kSuccClosed) || old >= kStreamSucc) {
          atomicSub(&g.indeg_w[v], 1u);
          if (!(old & kSuccClosed)) set_error(g.rs, (uint32_t)SPX_ERR_QUEUE_FULL, 0);
        } else {
          *(volatile uint32_t*)&g.succ[(size_t)p * kStreamSucc + old] = v;
        }
      }
      __threadfence();
      ready = atomicSub(&g.indeg_w[v], 1u) == 1u;
      if (ready) {
        np = t.nparts;
        pq = graph_queue(t.prio);
      }
    }
    push_ready_warp(g, ready, v, np, pq);
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      atomicAdd(&g.rs->admitted.v, min(32u, a1 - base));
    }
  }
  if (lane == 0) touch_progress(g);
}

// Stream mode, warp 0: close the successor list of a finished task and
// release the successors attached so far (an attachment reserved before the
// close but not yet written is waited for, bounded).
__device__ void release_stream(const DevGraph& g, uint32_t u) {
  const int lane = threadIdx.x & 31;
  uint32_t c = 0;
  if (lane == 0) c = atomicOr(&g.succ_cnt[u], kSuccClosed) & ~kSuccClosed;
  c = __shfl_sync(0xffffffffu, c, 0);
  if (c > kStreamSucc) c = kStreamSucc;
  for (uint32_t base = 0; base < c; base += 32) {
    const uint32_t idx = base + lane;
    bool ready = false;
    uint32_t s = 0, np = 0, pq = 0;
    if (idx < c) {
      const uint32_t* slot = &g.succ[(size_t)u * kStreamSucc + idx];
      uint32_t spins = 0;
      while ((s = ld_volatile(slot)) == kEmpty) {
        if ((++spins & 1023u) == 0 && (ld_volatile(&g.rs->abort) || watchdog_expired(g))) break;
      }
      if (s != kEmpty) {
        ready = atomicSub(&g.indeg_w[s], 1u) == 1u;
        if (ready) {
          const TaskDesc ts = load_task(&g.tasks[s]);
          np = ts.nparts;
          pq = graph_queue(ts.prio);
        }
      } else {
        set_error(g.rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
      }
    }
    push_ready_warp(g, ready, s, np, pq);
  }
}

// Bounded spin until t ns have passed (SPX_OP_SPIN); false on abort/timeout.
__device__ bool spin_for(const DevGraph& g, long long ns) {
  const unsigned long long t0 = globaltimer();
  for (;;) {
    const unsigned long long dt = globaltimer() - t0;
    if ((long long)dt >= ns) return true;
    if (ld_volatile(&g.rs->abort)) return false;
    if (dt > g.watchdog_ns) {
      set_error(g.rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
      return false;
    }
    __nanosleep(1000);
  }
}

// Run units u0..u1 of one phase of a task with the whole CTA.  Returns 0,
// a POTRF info (1-based column in the tile), -1 for an op this kernel cannot
// run, or -2 when a tensor-core wait timed out.  Low-precision tasks need
// the tensor-core instances (kMode 1: two CTAs per SM; kMode 2: one CTA per
// SM, which alone runs the split-FP64 products).
template <int kMode>
__device__ int run_units(const DevGraph& g, const TaskDesc& t, uint32_t phase, uint32_t u0,
                         uint32_t u1, F64Smem& s, TcCtx& tc) {
  const TileDesc* T = g.tiles;
  const bool lowp = t.prec != SPX_F64;
  constexpr bool kTc = kMode >= 1;
  if (lowp && !kTc) return -1;
  if (t.prec == SPX_F64_OZAKI && kMode != 2) return -1;
  switch (t.op) {
    case SPX_OP_POTRF:
      return op_potrf_units(T[t.h[0]], phase, u0, u1, s, t.flags & kFlagFine);
    case SPX_OP_POTRF_PANEL:
      if (t.prec == SPX_F64_OZAKI && phase + 1 == op_phases(t.op, t.prec, T, t.h)) {
        if constexpr (kMode == 2) {
          op_oz_split(T[t.h[1]], u0, u1, &tc.oz->v[0][0]);
          return 0;
        }
        return -1;
      }
      return op_potrf_panel_units(T[t.h[0]], T[t.h[1]], phase, u0, u1, s, t.flags & kFlagFine);
    case SPX_OP_TRSM:
      if constexpr (kTc) {
        if (lowp && phase + 1 == op_phases(t.op, t.prec, T, t.h, t.flags & kFlagFine)) {
          if (t.prec == SPX_F64_OZAKI) op_oz_split(T[t.h[1]], u0, u1, &tc.oz->v[0][0]);
          else if (t.prec == SPX_BF16) op_lowp_copy<true>(T[t.h[1]], u0, u1);
          else op_lowp_copy<false>(T[t.h[1]], u0, u1);
          return 0;
        }
      }
      if (trsm_row_form(T[t.h[1]].cols, t.flags & kFlagFine))
        op_trsm_rows(T[t.h[0]], T[t.h[1]], u0, u1, s);
      else
        op_trsm_units(T[t.h[0]], T[t.h[1]], phase, u0, u1, s, t.flags & kFlagFine);
      return 0;
    case SPX_OP_SYRK:
      if constexpr (kTc) {
        if constexpr (kMode == 2) {
          if (t.prec == SPX_F64_OZAKI) {
            const TileDesc &Lt = T[t.h[0]], &Ct = T[t.h[1]];
            if (Lt.lmap < 0) return -1;
            return oz_product_units(g, Lt, Lt, (double*)Ct.ptr, Ct.ld, Ct.rows, Ct.cols, true,
                                    t.flags & kFlagFine, kOzSub, u0, u1, tc.st, tc.oz)
                       ? 0
                       : -2;
          }
        }
        if (lowp) {
          if (T[t.h[0]].lmap < 0) return -1;
          const bool ok = t.prec == SPX_BF16 ? op_tc_syrk<true>(g, T[t.h[0]], T[t.h[1]], u0, u1, tc)
                                             : op_tc_syrk<false>(g, T[t.h[0]], T[t.h[1]], u0, u1, tc);
          return ok ? 0 : -2;
        }
      }
      op_syrk(T[t.h[0]], T[t.h[1]], u0, u1, s, t.flags & kFlagFine);
      return 0;
    case SPX_OP_GEMM_NT_SUB:
      if constexpr (kTc) {
        if constexpr (kMode == 2) {
          if (t.prec == SPX_F64_OZAKI) {
            const TileDesc &At = T[t.h[0]], &Bt = T[t.h[1]], &Ct = T[t.h[2]];
            if (At.lmap < 0 || Bt.lmap < 0) return -1;
            return oz_product_units(g, At, Bt, (double*)Ct.ptr, Ct.ld, Ct.rows, Ct.cols, false,
                                    t.flags & kFlagFine, kOzSub, u0, u1, tc.st, tc.oz)
                       ? 0
                       : -2;
          }
        }
        if (lowp) {
          if (T[t.h[0]].lmap < 0 || T[t.h[1]].lmap < 0) return -1;
          const bool ok =
              t.prec == SPX_BF16
                  ? op_tc_gemm<true>(g, T[t.h[0]], T[t.h[1]], T[t.h[2]], u0, u1, tc)
                  : op_tc_gemm<false>(g, T[t.h[0]], T[t.h[1]], T[t.h[2]], u0, u1, tc);
          return ok ? 0 : -2;
        }
      }
      op_gemm<false, false>(T[t.h[0]], T[t.h[1]], T[t.h[2]], T[t.h[0]].cols, -1.0, u0, u1, s,
                            t.flags & kFlagFine);
      return 0;
    case SPX_OP_GEMM_NN_ADD:
      if constexpr (kMode == 2) {
        if (t.prec == SPX_F64_OZAKI) {  // C += A B from A's row split and B's column split
          const TileDesc &At = T[t.h[0]], &Bt = T[t.h[1]], &Ct = T[t.h[2]];
          if (At.lmap < 0 || Bt.lmap < 0) return -1;
          return oz_product_units(g, At, Bt, (double*)Ct.ptr, Ct.ld, Ct.rows, Ct.cols, false,
                                  t.flags & kFlagFine, kOzAdd, u0, u1, tc.st, tc.oz)
                     ? 0
                     : -2;
        }
      }
      op_gemm<false, true>(T[t.h[0]], T[t.h[1]], T[t.h[2]], T[t.h[0]].cols, 1.0, u0, u1, s,
                           t.flags & kFlagFine, t.flags & kFlagAtomic);
      return 0;
    case SPX_OP_TRSM_L_FWD:
      op_trsm_fwd(T[t.h[0]], T[t.h[1]], phase, u0, u1, s);
      return 0;
    case SPX_OP_GEMM_FWD:
    case SPX_OP_GEMM_BWD: {
      const TileDesc &L = T[t.h[0]], &Xk = T[t.h[1]], &Xi = T[t.h[2]];
      if (L.dtype == SPX_DT_F32) {  // FP32 correction solve (all operands FP32)
        if (t.op == SPX_OP_GEMM_FWD)
          rhs_update<false, float>((const float*)L.ptr, L.ld, (const float*)Xk.ptr, Xk.ld,
                                   (float*)Xi.ptr, Xi.ld, Xi.rows, Xi.cols, L.cols, u0, u1, s);
        else
          rhs_update<true, float>((const float*)L.ptr, L.ld, (const float*)Xk.ptr, Xk.ld,
                                  (float*)Xi.ptr, Xi.ld, Xi.rows, Xi.cols, L.rows, u0, u1, s);
        return 0;
      }
      if (t.op == SPX_OP_GEMM_FWD)
        rhs_update<false>((const double*)L.ptr, L.ld, (const double*)Xk.ptr, Xk.ld,
                          (double*)Xi.ptr, Xi.ld, Xi.rows, Xi.cols, L.cols, u0, u1, s);
      else
        rhs_update<true>((const double*)L.ptr, L.ld, (const double*)Xk.ptr, Xk.ld,
                         (double*)Xi.ptr, Xi.ld, Xi.rows, Xi.cols, L.rows, u0, u1, s);
      return 0;
    }
    case SPX_OP_TRSM_LT_BWD:
      op_trsm_bwd(T[t.h[0]], T[t.h[1]], phase, u0, u1, s);
      return 0;
    case SPX_OP_COPY:
    case SPX_OP_AXPY:
      op_copy_axpy(T[t.h[0]], T[t.h[1]], u0, u1, t.op == SPX_OP_AXPY, t.flags & kFlagAtomic,
                   (t.op == SPX_OP_AXPY && t.arg) ? __longlong_as_double(t.arg) : 1.0);
      return 0;
    case SPX_OP_TRMM:
      if (T[t.h[0]].dtype == SPX_DT_F32)
        op_trmm<float>(T[t.h[0]], T[t.h[1]], T[t.h[2]], t.arg != 0, u0, u1, s);
      else
        op_trmm<double>(T[t.h[0]], T[t.h[1]], T[t.h[2]], t.arg != 0, u0, u1, s);
      return 0;
    case SPX_OP_NBODY_SELF:
      op_nbody(T[t.h[0]], nullptr, u0, u1, s);
      return 0;
    case SPX_OP_NBODY_PAIR:
      op_nbody(T[t.h[0]], &T[t.h[1]], u0, u1, s);
      return 0;
    case SPX_OP_TRSM_INV:
      if constexpr (kTc) {
        if constexpr (kMode == 2) {
          if (t.prec == SPX_F64_OZAKI) {
            if (phase != 1) {  // split the input (phase 0) or the result (phase 2)
              op_oz_split(T[t.h[1]], u0, u1, &tc.oz->v[0][0]);
              return 0;
            }
            // A <- A V^T: the product reads A's and V's slots, then stores A
            const TileDesc &Vt = T[t.h[0]], &At = T[t.h[1]];
            if (At.lmap < 0 || Vt.lmap < 0) return -1;
            return oz_product_units(g, At, Vt, (double*)At.ptr, At.ld, At.rows, At.cols, false,
                                    t.flags & kFlagFine, kOzStore, u0, u1, tc.st, tc.oz)
                       ? 0
                       : -2;
          }
        }
        const bool ok = t.prec == SPX_BF16
                            ? op_tc_trsm_inv<true>(T[t.h[0]], T[t.h[1]], u0, u1, tc)
                            : op_tc_trsm_inv<false>(T[t.h[0]], T[t.h[1]], u0, u1, tc);
        return ok ? 0 : -2;
      }
      return -1;
    case SPX_OP_TRTRI:
      if (t.prec == SPX_F64_OZAKI && phase == trtri_phases(T[t.h[0]].rows)) {
        if constexpr (kTc) {
          op_oz_split(T[t.h[1]], u0, u1, &tc.oz->v[0][0]);
          return 0;
        }
        return -1;
      }
      op_trtri_units(T[t.h[0]], T[t.h[1]], phase, u0, u1, s);
      return 0;
    case SPX_OP_SPLIT:
    case SPX_OP_SPLIT_T:
      if constexpr (kMode == 2) {
        if (t.op == SPX_OP_SPLIT)
          op_oz_split(T[t.h[0]], u0, u1, &tc.oz->v[0][0]);
        else  // the V staging area is free between products: the column maxima
          op_oz_split_t(T[t.h[0]], u0, u1, reinterpret_cast<unsigned long long*>(&tc.oz->v[0][0]));
        return 0;
      }
      return -1;
    case SPX_OP_NOP:
      return 0;
    case SPX_OP_SPIN:
      if (threadIdx.x == 0) spin_for(g, t.arg);
      __syncthreads();
      return 0;
    default:
      return -1;
  }
}

// Run part `part` of phase `phase`; a serial task runs all of its phases
// and units here, in order.
constexpr int kParked = -100;  // run_part: the task waits on a lock's list (no part finished)
__device__ int acquire_comm(const DevGraph& g, uint32_t u, const TaskDesc& t);

template <int kMode>
__device__ int run_part(const DevGraph& g, const TaskDesc& t, uint32_t phase, uint32_t part,
                        F64Smem& s, TcCtx& tc, uint32_t u, bool locks) {
  const TileDesc* T = g.tiles;
  if (comm_acquire_phase(t)) {
    if (phase == 0) {  // the lock phase (the per-task executors run tasks one by one)
      __shared__ int s_got;
      if (threadIdx.x == 0) s_got = locks ? acquire_comm(g, u, t) : 1;
      __syncthreads();
      return s_got > 0 ? 0 : (s_got == 0 ? kParked : -2);
    }
    --phase;
  }
  if (t.flags & kFlagSerial) {
    const uint32_t nph = op_phases(t.op, t.prec, T, t.h, t.flags & kFlagFine);
    for (uint32_t ph = 0; ph < nph; ++ph) {
      const uint32_t nu = op_phase_units(t.op, t.prec, T, t.h, ph, t.flags & kFlagFine);
      const int r = run_units<kMode>(g, t, ph, 0, nu, s, tc);
      if (r) return r;
      __syncthreads();
    }
    return 0;
  }
  const uint32_t units = op_phase_units(t.op, t.prec, T, t.h, phase, t.flags & kFlagFine);
  const uint32_t parts = phase_parts(units);
  (void)u;
  const uint32_t u0 = (uint32_t)((unsigned long long)part * units / parts);
  const uint32_t u1 = (uint32_t)((unsigned long long)(part + 1) * units / parts);
  return run_units<kMode>(g, t, phase, u0, u1, s, tc);
}

// Push the next phase (np parts) of task u (thread 0).  The CTA that
// finished the phase runs part 0 itself, without a queue round trip, so the
// slot's claim counter starts at 1; a single-part phase (the diagonal steps
// on the critical path) never touches the queue.
__device__ void push_phase(const DevGraph& g, uint32_t u, uint32_t np, uint32_t prio) {
  if (np <= 1) return;
  const uint32_t q = graph_queue(prio);
  const uint32_t slot = atomicAdd(&g.rs->tail[q].v, 1u);
  atomicMax(&g.rs->hiwater, slot + 1u);
  if (slot >= g.qcap) {
    set_error(g.rs, (uint32_t)SPX_ERR_QUEUE_FULL, 0);
    return;
  }
  atomicExch(&g.qclaim[q][slot], 1u);
  __threadfence();
  *(volatile uint32_t*)&g.queue[q][slot] = (u << kPartBits) | (np - 1);
}

// Take the COMMUTATIVE_WRITE locks of task u in ascending handle order
// (records of a task are sorted by handle).  One thread.  False on abort.
__device__ bool lock_comm(const DevGraph& g, uint32_t u) {
  const uint32_t r1 = __ldcg(&g.task_rec[u + 1]);
  for (uint32_t r = __ldcg(&g.task_rec[u]); r < r1; ++r) {
    if (__ldcg(&g.rec_mode[r]) != SPX_COMMUTATIVE_WRITE) continue;
    uint32_t* lk = &g.locks[__ldcg(&g.rec_handle[r])];
    uint32_t spins = 0;
    while (atomicCAS(lk, 0u, u + 1) != 0u) {
      __nanosleep(64);
      if ((++spins & 255u) == 0) {
        if (ld_volatile(&g.rs->abort)) return false;
        if (watchdog_expired(g)) {
          set_error(g.rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
          return false;
        }
      }
    }
  }
  __threadfence();
  return true;
}

__device__ void unlock_comm(const DevGraph& g, uint32_t u) {
  __threadfence();
  const uint32_t r1 = __ldcg(&g.task_rec[u + 1]);
  for (uint32_t r = __ldcg(&g.task_rec[u]); r < r1; ++r)
    if (__ldcg(&g.rec_mode[r]) == SPX_COMMUTATIVE_WRITE)
      atomicExch(&g.locks[__ldcg(&g.rec_handle[r])], 0u);
}

// Short spin lock guarding a tile's wait list (one thread).  False on abort
// or watchdog.
__device__ bool wl_enter(const DevGraph& g, uint32_t h) {
  uint32_t spins = 0;
  while (atomicCAS(&g.wl_lock[h], 0u, 1u) != 0u) {
    if ((++spins & 255u) == 0) {
      if (ld_volatile(&g.rs->abort)) return false;
      if (watchdog_expired(g)) {
        set_error(g.rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
        return false;
      }
    }
  }
  __threadfence();
  return true;
}

__device__ void wl_leave(const DevGraph& g, uint32_t h) {
  __threadfence();
  atomicExch(&g.wl_lock[h], 0u);
}

// Lock phase of a commutative task u (graph runs): take its
// COMMUTATIVE_WRITE locks in ascending handle order, from the record after
// the last lock it was handed (comm_next).  A lock held by another task
// parks u at the end of that tile's FIFO, so the CTA moves on instead of
// spinning; the holder hands the lock to the first parked task when it
// releases it and pushes that task's lock phase again.  The ascending order
// keeps the waits acyclic.  Returns 1 when u holds every lock, 0 when
// parked, -1 on abort / watchdog.  One thread.
__device__ int acquire_comm(const DevGraph& g, uint32_t u, const TaskDesc& t) {
  (void)t;
  const uint32_t r0 = __ldcg(&g.task_rec[u]), r1 = __ldcg(&g.task_rec[u + 1]);
  for (uint32_t r = r0 + ld_volatile(&g.comm_next[u]); r < r1; ++r) {
    if (__ldcg(&g.rec_mode[r]) != SPX_COMMUTATIVE_WRITE) continue;
    const uint32_t h = __ldcg(&g.rec_handle[r]);
    if (!wl_enter(g, h)) return -1;
    if (ld_volatile(&g.locks[h]) == 0u) {
      *(volatile uint32_t*)&g.locks[h] = u + 1;
      wl_leave(g, h);
      continue;
    }
    *(volatile uint32_t*)&g.comm_next[u] = r + 1 - r0;  // resumes after h
    *(volatile uint32_t*)&g.wnext[u] = 0u;
    const uint32_t tail = ld_volatile(&g.wl_tail[h]);
    if (tail) *(volatile uint32_t*)&g.wnext[tail - 1] = u + 1;
    else *(volatile uint32_t*)&g.wl_head[h] = u + 1;
    *(volatile uint32_t*)&g.wl_tail[h] = u + 1;
    wl_leave(g, h);
    return 0;
  }
  __threadfence();
  return 1;
}

// Push the lock phase of task w again (one part).  One thread.
__device__ void push_lock_phase(const DevGraph& g, uint32_t w) {
  const TaskDesc t = load_task(&g.tasks[w]);
  const uint32_t q = graph_queue(t.prio);
  const uint32_t slot = atomicAdd(&g.rs->tail[q].v, 1u);
  atomicMax(&g.rs->hiwater, slot + 1u);
  if (slot >= g.qcap) {
    set_error(g.rs, (uint32_t)SPX_ERR_QUEUE_FULL, 0);
    return;
  }
  __threadfence();
  *(volatile uint32_t*)&g.queue[q][slot] = w << kPartBits;
}

// Release the locks of task u after its last phase: a lock with parked
// tasks goes straight to the first of them.  One thread.
__device__ void release_comm(const DevGraph& g, uint32_t u) {
  __threadfence();
  const uint32_t r0 = __ldcg(&g.task_rec[u]), r1 = __ldcg(&g.task_rec[u + 1]);
  for (uint32_t r = r0; r < r1; ++r) {
    if (__ldcg(&g.rec_mode[r]) != SPX_COMMUTATIVE_WRITE) continue;
    const uint32_t h = __ldcg(&g.rec_handle[r]);
    if (!wl_enter(g, h)) return;
    const uint32_t w = ld_volatile(&g.wl_head[h]);
    if (w) {
      const uint32_t nx = ld_volatile(&g.wnext[w - 1]);
      *(volatile uint32_t*)&g.wl_head[h] = nx;
      if (!nx) *(volatile uint32_t*)&g.wl_tail[h] = 0u;
    }
    *(volatile uint32_t*)&g.locks[h] = w;  // the parked task (+1), or free
    wl_leave(g, h);
    if (w) push_lock_phase(g, w - 1);
  }
}


// ---------------------------------------------------------------------------
// Server mode.  Queues are bounded MPMC rings with one sequence word per cell
// (the cell of ticket t can be written when seq == t and read when
// seq == t + 1; the reader hands it to ticket t + qcap).  Pushers wait
// (bounded) for a slow reader of the previous round, so no entry is lost
// when the ring wraps.
// ---------------------------------------------------------------------------
constexpr uint32_t kSubmit = 0xFFFFFFFDu;  // pop result: a submission was claimed

__device__ bool ring_put(const DevGraph& g, uint32_t q, uint32_t ticket, uint32_t v) {
  const uint32_t cell = ticket % g.qcap;
  uint32_t spins = 0;
  while (ld_volatile(&g.qseq[q][cell]) != ticket) {
    if ((++spins & 1023u) == 0) {
      if (ld_volatile(&g.rs->abort)) return false;
      if (watchdog_expired(g)) {
        set_error(g.rs, (uint32_t)SPX_ERR_QUEUE_FULL, 0);
        return false;
      }
    }
  }
  *(volatile uint32_t*)&g.queue[q][cell] = v;
  __threadfence();
  *(volatile uint32_t*)&g.qseq[q][cell] = ticket + 1;
  return true;
}

// Push np consecutive parts of pool task u (one thread).
__device__ void ring_push_task(const DevGraph& g, uint32_t u, uint32_t p0, uint32_t np,
                               uint32_t prio) {
  if (p0 >= np) return;
  const uint32_t q = prio ? 0u : 1u, cnt = np - p0;
  const uint32_t t0 = atomicAdd(&g.rs->tail[q].v, cnt);
  atomicMax(&g.rs->hiwater, t0 + cnt - ld_volatile(&g.rs->head[q].v));
  for (uint32_t p = 0; p < cnt; ++p)
    if (!ring_put(g, q, t0 + p, (u << kPartBits) | (p0 + p))) return;
}

// Pop a queue entry, claim a submission (kSubmit, entry copied to *sub), or
// leave (kExit): after shutdown with no live request, after idle_ns with
// nothing live, on abort, or when live work makes no progress (watchdog).
__device__ uint32_t pop_server(const DevGraph& g, uint32_t& empties, SubEntry* sub) {
  RunState* rs = g.rs;
  uint32_t backoff = 64, iter = 0;
  unsigned long long idle_start = 0;
  for (;;) {
    if (ld_volatile(&rs->abort)) return kExit;
    for (int q = 0; q < 2; ++q) {
      uint32_t h = ld_volatile(&rs->head[q].v);
      uint32_t t = ld_volatile(&rs->tail[q].v);
      while ((int32_t)(t - h) > 0) {
        const uint32_t prev = atomicCAS(&rs->head[q].v, h, h + 1);
        if (prev == h) {
          const uint32_t cell = h % g.qcap;
          uint32_t spins = 0;
          while (ld_volatile(&g.qseq[q][cell]) != h + 1) {
            if ((++spins & 1023u) == 0) {
              if (ld_volatile(&rs->abort)) return kExit;
              if (watchdog_expired(g)) {
                set_error(rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
                return kExit;
              }
            }
          }
          __threadfence();
          const uint32_t v = ld_volatile(&g.queue[q][cell]);
          __threadfence();
          *(volatile uint32_t*)&g.qseq[q][cell] = h + g.qcap;
          return v;
        }
        h = prev;
        t = ld_volatile(&rs->tail[q].v);
      }
    }
    const uint32_t stail = g.ctl->sub_tail;
    const uint32_t shead = ld_volatile(&rs->sub_head.v);
    if ((int32_t)(stail - shead) > 0) {
      if (atomicCAS(&rs->sub_head.v, shead, shead + 1) == shead) {
        const volatile uint32_t* src = (const volatile uint32_t*)&g.ctl->ring[shead % kSubRing];
        uint32_t* dst = (uint32_t*)sub;
        for (int i = 0; i < (int)(sizeof(SubEntry) / 4); ++i) dst[i] = src[i];
        atomicAdd(&rs->live.v, 1u);
        touch_progress(g);
        return kSubmit;
      }
      continue;
    }
    ++empties;
    const uint32_t live = ld_volatile(&rs->live.v);
    if (live == 0) {
      if (g.ctl->shutdown) return kExit;
      const unsigned long long now = globaltimer();
      if (!idle_start) idle_start = now;
      else if (now - idle_start > g.idle_ns) return kExit;
    } else {
      idle_start = 0;
      if ((++iter & 63u) == 0 && watchdog_expired(g)) {
        set_error(rs, (uint32_t)SPX_ERR_TIMEOUT, 0);
        return kExit;
      }
    }
    __nanosleep(backoff);
    if (backoff < 2048) backoff <<= 1;
  }
}

// Derive the DAG of a claimed request with this CTA, set up its tasks and
// push its ready ones.  All threads.
__device__ void server_admit(const DevGraph& g, const SubEntry& e, uint32_t* sh) {
  DevGraph v = g;
  v.ntasks = e.ntasks;
  v.ntiles = e.ntiles;
  v.nrec = e.nrec;
  v.ecap = e.ecap;
  v.tasks = g.tasks + e.tb;
  v.tiles = g.tiles + e.hb;
  v.rec_handle = g.rec_handle + e.rb;
  v.rec_seq = g.rec_seq + e.rb;
  v.rec_mode = g.rec_mode + e.rb;
  v.task_rec = g.task_rec + e.tb;
  v.hptr = g.hptr + e.hb;
  v.s_task = g.s_task + e.rb;
  v.s_mode = g.s_mode + e.rb;
  v.s_first = g.s_first + e.rb;
  v.rec_pos = g.rec_pos + e.rb;
  v.gid = g.gid + e.rb;
  v.gpos = g.gpos + e.rb;
  v.row_ptr = g.row_ptr + e.tb;
  v.col = g.col + e.eb;
  v.indeg = g.indeg + e.tb;
  const bool ok = derive_dag<kThreads>(v, sh);
  const int tid = threadIdx.x;
  if (!ok) {  // edge buffer too small (cannot happen: it holds every candidate
              // edge): every task becomes ready and drains under the error status
    for (uint32_t u = tid; u < e.ntasks; u += kThreads) g.indeg[e.tb + u] = 0;
    __syncthreads();
  }
  for (uint32_t u = tid; u < e.ntasks; u += kThreads) {
    const uint32_t gu = e.tb + u;
    g.indeg_w[gu] = g.indeg[gu];
    g.remaining[gu] = g.tasks[gu].nparts;
    g.phase[gu] = 0;
    g.task_req[gu] = e.slot;
    g.t_start[gu] = 0xFFFFFFFFu;
    g.t_end[gu] = 0;
  }
  if (tid == 0) {
    ReqDev& r = g.reqs[e.slot];
    r.tb = e.tb; r.ntasks = e.ntasks; r.hb = e.hb; r.ntiles = e.ntiles;
    r.rb = e.rb; r.nrec = e.nrec; r.eb = e.eb; r.ecap = e.ecap;
    r.remaining = e.ntasks;
    r.status = ok ? 0u : (uint32_t)SPX_ERR_QUEUE_FULL;
    r.info = 0;
    r.seq = e.seq;
  }
  __threadfence();
  __syncthreads();
  for (uint32_t u = tid; u < e.ntasks; u += kThreads) {
    const uint32_t gu = e.tb + u;
    if (g.indeg[gu] == 0) ring_push_task(g, gu, 0, g.tasks[gu].nparts, g.tasks[gu].prio);
  }
  __syncthreads();
}

// Release the successors of a finished pool task u of request slot r
// (warp 0): request-local successor ids are offset by the request's task base.
__device__ void release_server(const DevGraph& g, uint32_t u, uint32_t r) {
  const int lane = threadIdx.x & 31;
  const uint32_t tb = g.reqs[r].tb, eb = g.reqs[r].eb;
  const uint32_t r0 = g.row_ptr[u], r1 = g.row_ptr[u + 1];
  for (uint32_t base = r0; base < r1; base += 32) {
    const uint32_t idx = base + lane;
    if (idx < r1) {
      const uint32_t s = tb + g.col[eb + idx];
      if (atomicSub(&g.indeg_w[s], 1u) == 1u) {
        __threadfence();
        ring_push_task(g, s, 0, g.tasks[s].nparts, g.tasks[s].prio);
      }
    }
  }
}

// Last task of request r finished: publish its status to the host.
__device__ void finish_request(const DevGraph& g, uint32_t r) {
  const ReqDev& q = g.reqs[r];
  g.ctl->done_status[r] = (int32_t)ld_volatile(&q.status);
  g.ctl->done_info[r] = q.info;
  __threadfence_system();
  g.ctl->done_seq[r] = q.seq;
  __threadfence_system();
  atomicSub(&g.rs->live.v, 1u);
}

// kMode 2 runs one CTA per SM (its shared memory allows no second), with
// the same register budget as the others.
template <int kMode, bool kServer>
__global__ void __launch_bounds__(kThreads, 2) persistent_kernel(DevGraph g) {
  constexpr bool kTc = kMode >= 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the tensor-core instances align their operand stages to 1024 bytes; they
  // share the space with the FP64 ops' buffers
  unsigned char* base =
      kTc ? (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023) : smem_raw;
  F64Smem& s = *reinterpret_cast<F64Smem*>(base);
  __shared__ TcState tcs;
  TcCtx tc{&tcs, reinterpret_cast<TcBuf*>(base), reinterpret_cast<OzBuf*>(base)};
  if (kTc) {
    tc_setup(tcs, kMode == 2 ? 512u : kTcCtaCols);
    __syncthreads();
  }
  __shared__ uint32_t s_item, s_np, s_adm[2];
  __shared__ int s_flag;
  __shared__ SubEntry s_sub;
  __shared__ uint32_t s_scan[kThreads / 32 + 1];
  const int tid = threadIdx.x;
  RunState* rs = g.rs;
  const long long c_begin = clock64();
  long long busy = 0;
  uint32_t empties = 0;
  uint32_t next = kEmpty;  // thread 0: part 0 of a phase this CTA just opened
  uint32_t rnd = blockIdx.x * 2654435761u + 12345u;  // thread 0: scan start of pop
  if (tid == 0) touch_progress(g);

  for (;;) {
    if (tid == 0) {
      if (next != kEmpty) s_item = next;
      else s_item = kServer ? pop_server(g, empties, &s_sub) : pop(g, empties, rnd, s_adm);
      next = kEmpty;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item == kExit) break;
    if constexpr (!kServer) {
      if (item == kAdmit) {
        if (tid < 32) admit_tasks(g, s_adm[0], s_adm[1]);
        continue;
      }
    }
    if constexpr (kServer) {
      if (item == kSubmit) {
        server_admit(g, s_sub, s_scan);
        continue;
      }
    }
    const uint32_t u = item >> kPartBits, part = item & (kMaxParts - 1);
    const TaskDesc t = load_task(&g.tasks[u]);
    // the phase was written before its parts were pushed (and fenced)
    const uint32_t phase = t.nphases > 1 ? ld_volatile(&g.phase[u]) : 0u;
    const uint32_t req = kServer ? g.task_req[u] : (g.task_group ? g.task_group[u] : 0u);
    // a request (or a member of a batched run) whose task failed drains
    // without running its other tasks
    const bool skip = kServer ? ld_volatile(&g.reqs[req].status) != 0u
                              : (g.task_group && ld_volatile(&g.groups[req].status) != 0u);
    const long long c0 = clock64();
    if (tid == 0) {
      s_flag = 1;
      if ((t.flags & kFlagComm) && (t.flags & kFlagSerial)) s_flag = lock_comm(g, u) ? 1 : 0;
      // a commutative task starts when it holds its locks: its lock phase
      // (possibly parked and pushed again) is not part of its execution
      const bool lockph = comm_acquire_phase(t) && phase == 0;
      const uint32_t tk = atomicAdd(&rs->ticket.v, 1u);
      if (!lockph) atomicMin(&g.t_start[u], tk);
      if (g.trace && part == 0 && phase == (comm_acquire_phase(t) ? 1u : 0u)) {
        g.trace_rec[4 * u + 0] = globaltimer();
        g.trace_rec[4 * u + 2] = smid();
        g.trace_rec[4 * u + 3] = t.nparts;
      }
    }
    __syncthreads();
    if (!s_flag) break;
    // a skipped commutative task still takes (and later releases) its locks
    const bool run = !skip || (comm_acquire_phase(t) && phase == 0);
    const int info = run ? run_part<kMode>(g, t, phase, part, s, tc, u, true) : 0;
    __syncthreads();
    if (info == kParked) continue;  // handed its lock later, pushed again
    const long long dt = clock64() - c0;
    busy += dt;
    if (tid == 0) atomicAdd(&rs->op_cycles[t.op & 31], (unsigned long long)dt);
    if (tid == 0) {
      if (info > 0 && kServer) {
        // the request fails; the server and the other requests go on
        if (atomicCAS(&g.reqs[req].status, 0u, (uint32_t)SPX_NOT_SPD) == 0u)
          g.reqs[req].info = (int)t.arg + info;
      }
      if (info > 0 && !kServer && g.task_group) {
        // the batch member fails; the other members go on
        if (atomicCAS(&g.groups[req].status, 0u, (uint32_t)SPX_NOT_SPD) == 0u)
          g.groups[req].info = (int)t.arg + info;
      }
      if (info > 0 && !kServer && !g.task_group) {
        set_error(rs, (uint32_t)SPX_NOT_SPD, (int)t.arg + info);
        s_flag = 0;
      } else if (info < 0) {
        set_error(rs, (uint32_t)(info == -2 ? SPX_ERR_TIMEOUT : SPX_ERR_BAD_OP), 0);
        s_flag = 0;
      } else {
        __threadfence();
        const uint32_t tk = atomicAdd(&rs->ticket.v, 1u);
        atomicMax(&g.t_end[u], tk);
        if (g.trace) atomicMax(&g.trace_rec[4 * u + 1], globaltimer());
        atomicAdd(&rs->parts_done, 1u);
        s_flag = atomicSub(&g.remaining[u], 1u) == 1u ? 2 : 1;
        if (s_flag == 2 && phase + 1 < t.nphases) {
          // last part of a phase: set up the next phase before pushing it
          const uint32_t np = phase_parts(task_phase_units(t, g.tiles, phase + 1));
          *(volatile uint32_t*)&g.phase[u] = phase + 1;
          atomicExch(&g.remaining[u], np);
          s_np = np;
          s_flag = 3;
        }
        __threadfence();
        touch_progress(g);
      }
    }
    __syncthreads();
    if (s_flag == 0) break;
    if constexpr (kServer) {
      if (s_flag == 3 && tid == 0) {
        ring_push_task(g, u, 1, s_np, t.prio);
        next = u << kPartBits;
      }
      if (s_flag == 2 && tid < 32) {
        release_server(g, u, req);
        __syncwarp();
        if (tid == 0) {
          __threadfence();
          atomicAdd(&rs->done.v, 1u);
          if (atomicSub(&g.reqs[req].remaining, 1u) == 1u) finish_request(g, req);
        }
      }
    } else {
      if (s_flag == 3 && tid == 0) {
        push_phase(g, u, s_np, t.prio);
        next = u << kPartBits;
      }
      if (s_flag == 2) {
        if (tid < 32) {
          if ((t.flags & kFlagComm) && tid == 0) {
            if (comm_acquire_phase(t)) release_comm(g, u);
            else unlock_comm(g, u);
          }
          __syncwarp();
          if (g.sctl) release_stream(g, u);
          else release(g, u);
          __syncwarp();
          if (tid == 0) {
            __threadfence();
            atomicAdd(&rs->done.v, 1u);
            atomicOr(&g.t_end[u], kTaskDone);  // the host may copy the task's results now
          }
        }
      }
    }
  }
  __syncthreads();
  if (kTc) tc_teardown(tcs);
  if (tid == 0) {
    atomicAdd(&rs->busy_cycles, (unsigned long long)busy);
    atomicAdd(&rs->total_cycles, (unsigned long long)(clock64() - c_begin));
    atomicAdd(&rs->ctas, 1u);
    atomicAdd(&rs->empty_pops, empties);
  }
}

// Baseline: one launch per task phase, one CTA per part, insertion order.
template <int kMode>
__global__ void __launch_bounds__(kThreads, 2) task_kernel(DevGraph g, uint32_t u,
                                                                            uint32_t phase) {
  constexpr bool kTc = kMode >= 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base =
      kTc ? (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023) : smem_raw;
  F64Smem& s = *reinterpret_cast<F64Smem*>(base);
  __shared__ TcState tcs;
  TcCtx tc{&tcs, reinterpret_cast<TcBuf*>(base), reinterpret_cast<OzBuf*>(base)};
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = (int)ld_volatile(&g.rs->abort);
  __syncthreads();
  if (s_abort) return;
  if (kTc) {
    tc_setup(tcs, kMode == 2 ? 512u : kTcCtaCols);
    __syncthreads();
  }
  const TaskDesc t = g.tasks[u];
  if (threadIdx.x == 0 && blockIdx.x == 0) touch_progress(g);
  const int info = run_part<kMode>(g, t, phase, blockIdx.x, s, tc, u, false);
  if (threadIdx.x == 0) {
    if (info > 0) set_error(g.rs, (uint32_t)SPX_NOT_SPD, (int)t.arg + info);
    else if (info < 0) set_error(g.rs, (uint32_t)(info == -2 ? SPX_ERR_TIMEOUT : SPX_ERR_BAD_OP), 0);
    else atomicAdd(&g.rs->parts_done, 1u);
  }
  __syncthreads();
  if (kTc) tc_teardown(tcs);
}

}  // namespace
}  // namespace spx
