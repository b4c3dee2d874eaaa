// Internal data layout shared by the host builder (graph.cpp) and the device
// code (derive.cu, mega.cu).  Everything the device reads lives in HBM in the
// structures below; they are plain arrays of fixed-size records so that one
// cudaMemcpyAsync uploads each of them.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx.h"

namespace spx {

constexpr int kMaxHandles = 16;           // operands of one task
constexpr int kPartBits = 8;              // queue entry = task << 8 | part
constexpr uint32_t kMaxParts = 1u << kPartBits;
constexpr uint32_t kMaxTasks = (1u << (32 - kPartBits)) - 2;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // free queue slot
constexpr uint32_t kExit = 0xFFFFFFFEu;   // pop result: leave the loop
// Top bit of a task's end ticket: set once the task has finished (graph
// executors; tickets themselves stay below 2^31).
constexpr uint32_t kTaskDone = 0x80000000u;
// Streaming (tasks inserted while the persistent kernel runs): successor
// slots per task, filled by the admission of each successor; a task's slot
// count gets kSuccClosed when it finishes (later attachments see it done).
constexpr uint32_t kStreamSucc = 64;
constexpr uint32_t kSuccClosed = 0x80000000u;

// Control block of a stream, in device memory: the host's copy engine raises
// published after the tasks below it (their descriptors, records and
// predecessor lists) were written, on the same stream, and sets end when no
// task will follow.
struct StreamCtl {
  uint32_t published;
  uint32_t end;
};
// Work queues of a graph run, popped in this order: critical-path tasks
// (priority >= 2), high priority, normal.  The server keeps two ring queues
// (critical and high share the first).
constexpr int kQueues = 3;
__host__ __device__ inline uint32_t graph_queue(uint32_t prio) {
  return prio >= 2 ? 0u : (prio == 1 ? 1u : 2u);
}
constexpr int kThreads = 256;             // threads per persistent CTA
constexpr int kBlk = 64;                  // edge of a FP64 sub-tile part

// kFlagComm: the task has a COMMUTATIVE_WRITE access: a leading phase of one
// part takes the tiles' locks (see comm_acquire_phase), the op's phases
// follow, and the last one releases them.  kFlagSerial: one CTA runs every
// phase and every unit of the task in order (no-split graphs, and the
// server's commutative tasks, which take the locks at their single part);
// the arithmetic per unit is the same as when the units are spread over
// CTAs.  kFlagFine:
// the task is on the critical path (inserted with priority >= 2): its POTRF,
// TRSM and FP64 SYRK / GEMM phases use smaller units so that more SMs share
// it.
// kFlagAtomic: the written operand is an ATOMIC_WRITE (the op adds into it
// with atomic additions).
enum TaskFlags : uint8_t { kFlagComm = 1, kFlagSerial = 2, kFlagFine = 4, kFlagAtomic = 8 };

// One registered tile (a data handle of the STF model).
struct TileDesc {
  void* ptr;      // element (0,0), row-major
  void* lowp;     // optional low-precision copy (nullptr if none)
  int32_t rows, cols, ld, lowp_ld;
  int32_t lmap;   // tensor map holding the low-precision copy, -1 if none
  int32_t lr0, lc0;  // position of the copy's (0,0) in that map
  int32_t dtype;  // SPX_DT_* of the tile's elements
};
static_assert(sizeof(TileDesc) == 48, "TileDesc layout");

// One task: op, operands (handles in op order), parts, argument.
struct TaskDesc {
  uint8_t op, prec, flags, prio;  // prio: 0 = normal, 1 = high, 2 = critical path
  uint32_t nparts;   // parts of phase 0
  uint32_t h[3];
  uint32_t nphases;  // phases run one after another (1 for serial tasks)
  int64_t arg;
};
static_assert(sizeof(TaskDesc) == 32, "TaskDesc layout");

// ---------------------------------------------------------------------------
// Server mode (continuous batching): one resident persistent kernel, task
// graphs submitted while it runs.  Each submitted graph (a request) gets
// ranges of pool arrays; its CSR keeps request-local task ids and edge
// offsets, mapped to pool ids at release.
// ---------------------------------------------------------------------------
constexpr int kSubRing = 1024;      // submission ring entries (host-mapped)
constexpr int kMaxRequests = 1024;  // request slots

// One submission (host -> device), written to host-mapped memory.
struct SubEntry {
  uint32_t seq, slot;
  uint32_t tb, ntasks;  // task range [tb, tb + ntasks] (ntasks + 1 entries)
  uint32_t hb, ntiles;  // tile range (ntiles + 1 entries)
  uint32_t rb, nrec;    // access-record range (nrec + 1 entries)
  uint32_t eb, ecap;    // edge range
  uint32_t pad[6];
};
static_assert(sizeof(SubEntry) == 64, "SubEntry layout");

// Host-mapped control block of a server.
struct HostCtl {
  volatile uint32_t sub_tail;   // submissions published by the host
  volatile uint32_t shutdown;   // 1: exit once no request is live
  uint32_t pad0[30];
  SubEntry ring[kSubRing];
  volatile uint32_t done_seq[kMaxRequests];   // seq of the finished request in a slot
  volatile int32_t done_status[kMaxRequests];
  volatile int32_t done_info[kMaxRequests];
};

// Device record of a live request.
struct ReqDev {
  uint32_t tb, ntasks, hb, ntiles, rb, nrec, eb, ecap;
  uint32_t remaining;  // tasks not finished
  uint32_t status;     // 0, or the first failure of one of its tasks
  uint32_t seq;
  int32_t info;
  uint32_t pad[4];
};
static_assert(sizeof(ReqDev) == 64, "ReqDev layout");

// Run state of one execution; hot counters on separate 128-byte lines.
struct alignas(128) Line {
  uint32_t v;
  uint32_t pad[31];
};

struct RunState {
  Line head[kQueues];    // next queue slot to pop (0 = most urgent)
  Line tail[kQueues];    // next queue slot to fill
  Line done;             // finished tasks
  Line ticket;           // global ticket counter
  Line progress;         // %globaltimer >> 10 at the last finished part
  Line sub_head;         // server: submissions claimed by the device
  Line live;             // server: requests claimed and not finished
  Line admit_claim;      // stream: tasks claimed for admission
  Line admitted;         // stream: tasks whose admission finished
  // control words, read by every popping CTA
  alignas(128) uint32_t status;  // SPX_OK or an error / SPX_NOT_SPD
  int32_t info;          // failed POTRF column (1-based)
  uint32_t abort;        // set on any error: every CTA drains
  // statistics
  alignas(128) uint32_t empty_pops;  // pops that found both queues empty
  uint32_t parts_done;
  uint32_t hiwater;
  uint32_t ctas;
  unsigned long long busy_cycles;
  unsigned long long total_cycles;
  unsigned long long op_cycles[32];  // busy cycles by op (SPX_NUM_OPS <= 32)
};

// Status of one member graph of a batched run.
struct GroupState {
  uint32_t status;  // SPX_OK or SPX_NOT_SPD
  int32_t info;     // failed POTRF column (1-based)
};

// Pointers and sizes handed to the device kernels by value.
struct DevGraph {
  uint32_t ntasks, ntiles, nrec, ecap;
  uint32_t qcap;               // entries per priority queue
  uint32_t trace;
  unsigned long long watchdog_ns;
  const TaskDesc* tasks;       // [ntasks]
  const TileDesc* tiles;       // [ntiles]
  const CUtensorMap* maps;     // [nmaps] low-precision matrices (TMA)
  // access records in insertion order (records of one task are contiguous
  // and sorted by handle)
  const uint32_t* rec_handle;  // [nrec]
  const uint32_t* rec_seq;     // [nrec] position on the handle's list
  const uint8_t* rec_mode;     // [nrec]
  const uint32_t* task_rec;    // [ntasks+1] first record of each task
  // derivation scratch
  uint32_t* hptr;              // [ntiles+1] start of each handle's list
  uint32_t* s_task;            // [nrec] per-handle lists, concatenated
  uint8_t* s_mode;             // [nrec]
  uint8_t* s_first;            // [nrec] 1 at the first entry of a list
  uint32_t* rec_pos;           // [nrec] record -> position in the lists
  uint32_t* gid;               // [nrec] group index of each list entry
  uint32_t* gpos;              // [nrec+1] first entry of each group
  uint32_t* ucount;            // [ntasks] unique successors per task
  // derived DAG
  uint32_t* row_ptr;           // [ntasks+1]
  uint32_t* col;               // [ecap]
  uint32_t* indeg;             // [ntasks]
  // execution state
  uint32_t* indeg_w;           // [ntasks] remaining predecessors
  uint32_t* remaining;         // [ntasks] parts of the current phase not finished
  uint32_t* phase;             // [ntasks] current phase of a multi-phase task
  uint32_t* queue[kQueues];    // [qcap] each (the server uses the first two)
  // graph runs: an entry is one phase of a task, (task << kPartBits) |
  // (parts - 1); qclaim counts the parts claimed from each slot (atomicAdd,
  // so a wide phase is handed out without a compare-and-swap loop)
  uint32_t* qclaim[kQueues];   // [qcap] each, zero at the start of a run
  uint32_t* locks;             // [ntiles] owner task + 1, 0 = free
  // commutative tasks of graph runs: a FIFO of parked tasks per tile (task
  // + 1, 0 = none) behind a short spin lock, and per task the next record
  // to lock when it is handed a lock it waited for; all zero at the start
  uint32_t* wl_lock;           // [ntiles]
  uint32_t* wl_head;           // [ntiles]
  uint32_t* wl_tail;           // [ntiles]
  uint32_t* wnext;             // [ntasks]
  uint32_t* comm_next;         // [ntasks]
  uint32_t* t_start;           // [ntasks] tickets
  uint32_t* t_end;             // [ntasks]
  unsigned long long* trace_rec;  // [4*ntasks] when trace
  RunState* rs;
  // batched graph runs (spx_batch_execute): the member graph of each task and
  // each member's status; nullptr otherwise.  A POTRF failure then fails its
  // member only: that member's later tasks are skipped (popped and released
  // without running), the other members go on.
  const uint32_t* task_group;  // [ntasks]
  GroupState* groups;          // [members], zero at the start of a run
  // server mode only (server = 1): ring queues, requests, host control
  uint32_t server;
  uint32_t pad_;
  unsigned long long idle_ns;  // exit after this long with nothing live
  uint32_t* qseq[2];           // [qcap] ring cell sequence numbers
  uint32_t* task_req;          // [pool tasks] request slot of a task
  ReqDev* reqs;                // [kMaxRequests]
  HostCtl* ctl;                // device address of the host-mapped block
  // stream mode (sctl != nullptr): tasks arrive while the kernel runs; their
  // predecessors come from the host (pred_ptr / pred, in task order) and are
  // attached on admission to the predecessors' successor slots
  StreamCtl* sctl;             // the stream's control block
  uint32_t* succ_cnt;          // [task capacity] slots taken | kSuccClosed
  uint32_t* succ;              // [task capacity * kStreamSucc], kEmpty = not written yet
  const uint32_t* pred_ptr;    // [task capacity + 1]
  const uint32_t* pred;        // [predecessor capacity]
};


// Phases and work units of a task.  A task runs its phases one after
// another; the units of a phase are independent 64-granular pieces that any
// CTAs may run in parallel (parts = min(units, kMaxParts); part p covers
// units [p*U/P, (p+1)*U/P)).  When the last part of a phase finishes, the
// parts of the next phase are pushed; after the last phase the task releases
// its successors.  Shared by the host (part and queue-entry counts) and the
// device.
//   POTRF (nb = diagonal 64-blocks): for j = 0..nb-1, phase 3j factors block
//     (j,j) (1 unit), phase 3j+1 solves the rows below it (64-row units),
//     phase 3j+2 updates the lower triangle below it (64 x 64 block pairs);
//     3nb-2 phases.
//   TRSM (A m x n, nbc column blocks): for j = 0..nbc-1, phase 2j solves
//     column block j (64-row units), phase 2j+1 updates the column blocks
//     l > j (64 x 64 units).
//   Fine tasks (kFlagFine) use 16-row units for the row solves, the TRSM
//     updates and the FP64 GEMMs (16 x 64 blocks), and 32 x 32 block pairs
//     for the POTRF and SYRK updates: one SM
//     does about 2 FP64 FMA per clock, so a 64 x 64 x 64 unit alone takes
//     tens of microseconds, and the critical path is a chain of such units.
//   Fine TRSM with n <= 512 (row form): one phase of kTrsmRows-row units,
//     each solving all column blocks of its rows (rows are independent); the
//     2 nbc - 1 phase boundaries of the column form, each waiting for CTAs
//     to pick up its parts, were most of a critical panel solve's time.
//   TRSM_INV (A_ik <- A_ik V^T, tensor cores): one phase, 128-row blocks of
//     A_ik (each block runs its 128-column output blocks right to left: output
//     column c needs input columns <= c only, V being lower triangular, so
//     the block is updated in place).
//   SYRK: one phase, lower 64-block pairs.  GEMMs: one phase, 64x64 output
//     blocks.  TRMM: one phase, the units of GEMM_FWD.  TRTRI (V <- L^{-1},
//     by blocks): phase 0 inverts the 64 x 64 diagonal blocks of L, one unit
//     each, and zeroes V to their right; then, for block sizes s = 64, 128,
//     ... (level l, s = 64 * 2^(l-1)), the diagonal s-blocks pair up (top T,
//     bottom B) into the inverse of their 2s-block: phase 2l - 1 forms
//     W^T = (L_BT V_TT)^T into the zero upper block V_TB (16 x 64 units),
//     phase 2l forms V_BT = -V_BB W (16 x 64 units); the last phase zeroes the
//     upper part again (64-row units).  1 + 2 levels (+ 1) phases, all of
//     them parallel, instead of the 2 nb of a substitution.
//   Block solves (L n x n, X n x r): TRSM_L_FWD, for j = 0..nb-1, phase 2j
//     solves row block j of X with L_jj (one unit per column block of X),
//     phase 2j+1 subtracts L_ij X_j from the rows below it; TRSM_LT_BWD does
//     the same from the last row block up, with L_jj^T and the rows above.
//     The update units, and those of GEMM_FWD / GEMM_BWD, are row blocks x
//     column blocks of X: 16-row blocks of all r columns when X is narrow
//     (r <= 16: a 64-row block would leave most SMs idle on the solve's
//     critical path and waste lanes), 64 x 64 blocks otherwise.
__host__ __device__ inline uint32_t cdiv64(int a) { return (uint32_t)((a + kBlk - 1) / kBlk); }

__host__ __device__ inline uint32_t cdiv128(int a) { return (uint32_t)((a + 127) / 128); }
__host__ __device__ inline uint32_t cdiv16(int a) { return (uint32_t)((a + 15) / 16); }
__host__ __device__ inline uint32_t cdiv32(int a) { return (uint32_t)((a + 31) / 32); }

constexpr int kNarrowRows = 16;  // rows of a narrow right-hand-side unit
__host__ __device__ inline bool rhs_narrow(int cols) { return cols <= 16; }
__host__ __device__ inline uint32_t rhs_unit_rows(int cols) {
  return rhs_narrow(cols) ? (uint32_t)kNarrowRows : (uint32_t)kBlk;
}
__host__ __device__ inline uint32_t rhs_col_blocks(int cols) {
  return rhs_narrow(cols) ? 1u : cdiv64(cols);
}
__host__ __device__ inline uint32_t rhs_row_units(int rows, int cols) {
  const uint32_t rb = rhs_unit_rows(cols);
  return ((uint32_t)rows + rb - 1) / rb;
}

// TRTRI by blocks (see above): levels = ceil(log2(64-blocks)).
__host__ __device__ inline uint32_t trtri_levels(int n) {
  uint32_t lv = 0;
  while ((uint32_t)kBlk << lv < (uint32_t)n) ++lv;
  return lv;
}
__host__ __device__ inline uint32_t trtri_phases(int n) {
  const uint32_t lv = trtri_levels(n);
  return 1u + 2u * lv + (lv ? 1u : 0u);
}
// Units of TRTRI level phase (1 .. 2 levels) for an n x n L, and the pair
// (p, s, sB: top block [p, p+s), bottom block [p+s, p+s+sB)) and local unit of
// unit u when pair_of != nullptr.
__host__ __device__ inline uint32_t trtri_level_units(int n, uint32_t phase, uint32_t u = 0,
                                                      int* pair_of = nullptr) {
  const uint32_t lvl = (phase + 1) / 2;  // 1-based
  const bool pa = phase % 2 == 1;        // W^T = (L_BT V_TT)^T, else V_BT = -V_BB W
  const int s = kBlk << (lvl - 1);
  uint32_t total = 0;
  for (int p = 0; p + s < n; p += 2 * s) {
    const int sb = n - p - s < s ? n - p - s : s;
    const uint32_t cnt = pa ? (uint32_t)(s / 16) * cdiv64(sb) : cdiv16(sb) * (uint32_t)(s / kBlk);
    if (pair_of && u >= total && u < total + cnt) {
      pair_of[0] = p;
      pair_of[1] = s;
      pair_of[2] = sb;
      pair_of[3] = (int)(u - total);
    }
    total += cnt;
  }
  return total;
}

// Units of a split-prec (SPX_F64_OZAKI) product, run by the one-CTA-per-SM
// kernel: output blocks of 128 rows x 64 columns, a unit being up to
// kOzGroup consecutive column blocks of one row block (their K loops and
// epilogues pipelined on one CTA), one block per unit for critical-path
// tasks (fine).  lower: only the blocks that reach the lower triangle (64 j <
// 128 (i + 1)).  Returns the number of units; with unit < that number and
// blk != nullptr, also its row block, first column block and block count.
// Eight blocks (a whole 512-wide row block): the pipeline refills once per
// row block (measured against four: 48.7 vs 51.0 ms on the n = 8192 GEMM DAG,
// 93.4 vs 94.6 ms on the n = 16384 factorization; two were slower).
constexpr int kOzGroup = 8;
__host__ __device__ inline uint32_t oz_units(int rows, int cols, bool lower, bool fine,
                                             uint32_t unit, uint32_t* blk) {
  const uint32_t nbr = cdiv128(rows), nbc = cdiv64(cols), g = fine ? 1u : (uint32_t)kOzGroup;
  uint32_t total = 0;
  for (uint32_t i = 0; i < nbr; ++i) {
    const uint32_t nb = lower && 2 * (i + 1) < nbc ? 2 * (i + 1) : nbc;
    const uint32_t cnt = (nb + g - 1) / g;
    if (blk && unit >= total && unit < total + cnt) {
      const uint32_t j0 = (unit - total) * g;
      blk[0] = i;
      blk[1] = j0;
      blk[2] = nb - j0 < g ? nb - j0 : g;
    }
    total += cnt;
  }
  return total;
}

// Row form of the TRSM of critical-path tasks: units of kTrsmRows rows, the
// rows held in shared memory (n <= kTrsmRowMaxN).
constexpr int kTrsmRows = 4;
constexpr int kTrsmRowMaxN = 512;
__host__ __device__ inline bool trsm_row_form(int n, bool fine) {
  return fine && n <= kTrsmRowMaxN;
}

// Low-precision tasks (prec = SPX_TF32 / SPX_BF16): SYRK and GEMM_NT_SUB run
// on the tensor cores in 128 x 128 output units (SYRK: lower block pairs);
// TRSM runs its FP64 phases and then one more phase that writes the
// low-precision copy of its result (64-row units).
__host__ __device__ inline uint32_t op_phases(int op, int prec, const TileDesc* t,
                                              const uint32_t* h, bool fine = false) {
  switch (op) {
    case SPX_OP_POTRF: return 3 * cdiv64(t[h[0]].rows) - 2;
    case SPX_OP_POTRF_PANEL:  // POTRF's, one more solving A_ik's last block; split prec: the split
      return 3 * cdiv64(t[h[0]].rows) - 1 + (prec == SPX_F64_OZAKI ? 1u : 0u);
    case SPX_OP_TRSM:
      return (trsm_row_form(t[h[1]].cols, fine) ? 1u : 2 * cdiv64(t[h[1]].cols) - 1) +
             (prec != SPX_F64 ? 1u : 0u);
    case SPX_OP_TRSM_L_FWD:
    case SPX_OP_TRSM_LT_BWD: return 2 * cdiv64(t[h[0]].rows) - 1;
    case SPX_OP_TRTRI:  // split prec: one more phase splits V into its slot
      return trtri_phases(t[h[0]].rows) + (prec == SPX_F64_OZAKI ? 1u : 0u);
    case SPX_OP_TRSM_INV:  // split prec: split A, product into A, split the result
      return prec == SPX_F64_OZAKI ? 3u : 1u;
    default: return 1;
  }
}

// Units of phase `phase` of a block solve with an n x n factor and an
// n x cols right-hand side (forward or backward).
__host__ __device__ inline uint32_t solve_phase_units(bool fwd, int n, int cols, uint32_t phase) {
  const uint32_t nb = cdiv64(n), j = phase / 2;
  if (phase % 2 == 0) return rhs_col_blocks(cols);
  const int rest = fwd ? n - kBlk * (int)(j + 1) : kBlk * (int)(nb - 1 - j);
  return rhs_row_units(rest, cols) * rhs_col_blocks(cols);
}

__host__ __device__ inline uint32_t op_phase_units(int op, int prec, const TileDesc* t,
                                                   const uint32_t* h, uint32_t phase,
                                                   bool fine) {
  switch (op) {
    case SPX_OP_POTRF: {
      const int n = t[h[0]].rows, below = n - kBlk * (int)(phase / 3 + 1);
      if (phase % 3 == 0) return 1u;
      if (phase % 3 == 1) return fine ? cdiv16(below) : cdiv64(below);
      const uint32_t q = fine ? cdiv32(below) : cdiv64(below);
      return q * (q + 1) / 2;
    }
    case SPX_OP_POTRF_PANEL: {  // POTRF's units, then those of the rows of A_ik
      const int n = t[h[0]].rows, qm = t[h[1]].rows;
      const int rest = n - kBlk * (int)(phase / 3 + 1), below = rest > 0 ? rest : 0;
      const uint32_t nb = cdiv64(n), qrb = fine ? cdiv16(qm) : cdiv64(qm);
      if (phase >= 3 * nb - 1) return cdiv64(qm);  // split of A_ik
      if (phase % 3 == 0) return 1u;
      if (phase % 3 == 1) return (fine ? cdiv16(below) : cdiv64(below)) + qrb;
      const uint32_t q = fine ? cdiv32(below) : cdiv64(below);
      return q * (q + 1) / 2 + qrb * (nb - 1 - phase / 3);
    }
    case SPX_OP_TRSM: {
      const uint32_t nbr = cdiv64(t[h[1]].rows), nbc = cdiv64(t[h[1]].cols), j = phase / 2;
      if (trsm_row_form(t[h[1]].cols, fine))  // the solve, then the low-precision copy
        return phase == 0 ? ((uint32_t)t[h[1]].rows + kTrsmRows - 1) / kTrsmRows : nbr;
      if (phase >= 2 * nbc - 1) return nbr;  // low-precision copy
      const uint32_t rb = fine ? cdiv16(t[h[1]].rows) : nbr;
      return phase % 2 == 0 ? rb : rb * (nbc - 1 - j);
    }
    case SPX_OP_SYRK: {
      if (prec == SPX_F64_OZAKI) return oz_units(t[h[1]].rows, t[h[1]].rows, true, fine, 0, nullptr);
      const uint32_t nb = prec != SPX_F64 ? cdiv128(t[h[1]].rows)
                                          : (fine ? cdiv32(t[h[1]].rows) : cdiv64(t[h[1]].rows));
      return nb * (nb + 1) / 2;
    }
    case SPX_OP_GEMM_NT_SUB:
      if (prec == SPX_F64_OZAKI) return oz_units(t[h[2]].rows, t[h[2]].cols, false, fine, 0, nullptr);
      if (prec != SPX_F64) return cdiv128(t[h[2]].rows) * cdiv128(t[h[2]].cols);
      return (fine ? cdiv16(t[h[2]].rows) : cdiv64(t[h[2]].rows)) * cdiv64(t[h[2]].cols);
    case SPX_OP_GEMM_NN_ADD:
      if (prec == SPX_F64_OZAKI) return oz_units(t[h[2]].rows, t[h[2]].cols, false, fine, 0, nullptr);
      return (fine ? cdiv16(t[h[2]].rows) : cdiv64(t[h[2]].rows)) * cdiv64(t[h[2]].cols);
    case SPX_OP_SPLIT: return cdiv64(t[h[0]].rows);    // 64 rows per unit
    case SPX_OP_SPLIT_T: return cdiv64(t[h[0]].cols);  // 64 columns per unit
    case SPX_OP_GEMM_FWD:
    case SPX_OP_GEMM_BWD:
      return rhs_row_units(t[h[2]].rows, t[h[2]].cols) * rhs_col_blocks(t[h[2]].cols);
    case SPX_OP_TRSM_L_FWD:
    case SPX_OP_TRSM_LT_BWD:
      return solve_phase_units(op == SPX_OP_TRSM_L_FWD, t[h[0]].rows, t[h[1]].cols, phase);
    case SPX_OP_COPY:
    case SPX_OP_AXPY: return cdiv64(t[h[1]].rows);
    case SPX_OP_TRMM:
      return rhs_row_units(t[h[2]].rows, t[h[2]].cols) * rhs_col_blocks(t[h[2]].cols);
    case SPX_OP_TRSM_INV:  // 128-row blocks of A_ik (tensor cores)
      if (prec == SPX_F64_OZAKI)
        return phase == 1 ? oz_units(t[h[1]].rows, t[h[1]].cols, false, fine, 0, nullptr)
                          : cdiv64(t[h[1]].rows);
      return cdiv128(t[h[1]].rows);
    case SPX_OP_NBODY_SELF:  // 64-particle target blocks
      return cdiv64(t[h[0]].rows);
    case SPX_OP_NBODY_PAIR:  // target blocks of P (sources Q), then of Q (sources P)
      return cdiv64(t[h[0]].rows) + cdiv64(t[h[1]].rows);
    case SPX_OP_TRTRI: {  // diagonal inverses, level products, zeroing (64-block units)
      const int n = t[h[0]].rows;
      if (phase == 0 || phase + 1 >= trtri_phases(n)) return cdiv64(n);  // (split: 64-row units)
      return trtri_level_units(n, phase);
    }
    default: return 1;
  }
}

__host__ __device__ inline uint32_t phase_parts(uint32_t units) {
  return units < kMaxParts ? units : kMaxParts;
}

// A commutative task that is not serial starts with a phase of one part that
// acquires its tile locks (or parks the task on a lock's wait list); the
// op's phase p is the task's phase p + 1.
__host__ __device__ inline bool comm_acquire_phase(const TaskDesc& t) {
  return (t.flags & kFlagComm) && !(t.flags & kFlagSerial);
}

__host__ __device__ inline uint32_t task_phases(const TaskDesc& t, const TileDesc* tiles) {
  return op_phases(t.op, t.prec, tiles, t.h, t.flags & kFlagFine) +
         (comm_acquire_phase(t) ? 1u : 0u);
}

__host__ __device__ inline uint32_t task_phase_units(const TaskDesc& t, const TileDesc* tiles,
                                                     uint32_t phase) {
  if (comm_acquire_phase(t)) {
    if (phase == 0) return 1u;
    --phase;
  }
  return op_phase_units(t.op, t.prec, tiles, t.h, phase, t.flags & kFlagFine);
}

// Launchers implemented in the .cu files (all asynchronous on stream).
cudaError_t launch_derive(const DevGraph& g, cudaStream_t st);
cudaError_t launch_init(const DevGraph& g, cudaStream_t st);  // reset run state only
// mode: 0 FP64 ops only, 1 tensor-core tile ops, 2 the split-FP64 products.
cudaError_t launch_persistent(const DevGraph& g, int num_ctas, int mode, cudaStream_t st);
cudaError_t launch_per_task(const DevGraph& g, const TaskDesc* host_tasks,
                            const TileDesc* host_tiles, int mode, cudaStream_t st);
// The launches of one task's phases on st (per-task executors).
cudaError_t launch_task(const DevGraph& g, uint32_t u, const TaskDesc& t,
                        const TileDesc* host_tiles, int mode, cudaStream_t st);
cudaError_t launch_server(const DevGraph& g, int num_ctas, int mode, cudaStream_t st);  // mode as launch_persistent
cudaError_t launch_ring_init(const DevGraph& g, cudaStream_t st);
int persistent_max_ctas(int* per_sm);
size_t persistent_smem_bytes();

}  // namespace spx
