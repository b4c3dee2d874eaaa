// Host side of the C ABI: the graph builder (task insertion), device memory
// management, and the execute / wait / inspect calls.
//
// Insertion follows the paper's model (section "Task insertion"; section
// "Internal implementation"): a task names tiles by address with an access
// mode; each tile (data handle) keeps the ordered list of the tasks that use
// it.  Here insertion is O(1) per access: it appends an access record
// (task, handle, mode, position on the handle's list) and updates three
// counters per handle that size the device edge buffer exactly.  Dependency
// derivation itself (groups, edges, de-duplication, CSR, in-degrees) runs on
// the device (derive.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "spx.h"
#include "graph_access.h"
#include "spx_internal.h"
#include "tmap.h"

using namespace spx;

namespace {

enum State { kBuilding = 0, kFrozen = 1, kRunning = 2, kDone = 3, kStreaming = 4 };

// Per-handle state of the host-side STF derivation (streaming): the members
// of the last group of accesses and of the group before it.
struct StreamGroup {
  int mode = -1;
  std::vector<uint32_t> last, prev;
};

// Predecessors of a task with the given access records, by the same rule as
// the device derivation: a READ / COMMUTATIVE_WRITE / ATOMIC_WRITE joins a
// last group of the same mode and depends on the group before it; any other
// access starts a group and depends on every member of the last one.
// Updates the handle states; returns the predecessors sorted and unique.
std::vector<uint32_t> stf_preds(std::vector<StreamGroup>& sg, uint32_t v, const uint32_t* handle,
                                const uint8_t* mode, uint32_t nrec) {
  std::vector<uint32_t> preds;
  for (uint32_t i = 0; i < nrec; ++i) {
    StreamGroup& s = sg[handle[i]];
    const int m = mode[i];
    const bool join = s.mode == m && (m == SPX_READ || m == SPX_COMMUTATIVE_WRITE ||
                                      m == SPX_ATOMIC_WRITE);
    if (join) {
      preds.insert(preds.end(), s.prev.begin(), s.prev.end());
      s.last.push_back(v);
    } else {
      preds.insert(preds.end(), s.last.begin(), s.last.end());
      s.prev.swap(s.last);
      s.last.assign(1, v);
      s.mode = m;
    }
  }
  std::sort(preds.begin(), preds.end());
  preds.erase(std::unique(preds.begin(), preds.end()), preds.end());
  return preds;
}

struct HandleState {
  uint32_t count = 0;      // accesses so far (next position on the list)
  int last_mode = -1;      // mode of the last group
  uint32_t last_size = 0;  // members of the last group
  uint32_t prev_size = 0;  // members of the group before it
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Layout of the single device allocation (and of the pinned upload mirror
// for its first region).  Offsets in bytes, 256-aligned.
struct Layout {
  size_t tasks, tiles, maps, rec_handle, rec_seq, rec_mode, task_rec, task_group, upload_end;
  size_t queue[kQueues], t_start, ff_end;
  size_t rs, locks, t_end, trace, phase, qclaim[kQueues], groups, wl_lock, wl_head, wl_tail, wnext,
      comm_next, zero_end;
  size_t hptr, s_task, s_mode, s_first, rec_pos, gid, gpos, ucount, row_ptr, col, indeg,
      indeg_w, remaining, total;
};

Layout make_layout(size_t N, size_t H, size_t M, size_t E, size_t Q, size_t NM, bool trace,
                   size_t NG) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1), 256);
    return at;
  };
  L.tasks = take(N * sizeof(TaskDesc));
  L.tiles = take(H * sizeof(TileDesc));
  L.maps = take(NM * sizeof(CUtensorMap));
  L.rec_handle = take(M * 4);
  L.rec_seq = take(M * 4);
  L.rec_mode = take(M);
  L.task_rec = take((N + 1) * 4);
  L.task_group = take(NG ? N * 4 : 0);
  L.upload_end = o;
  for (int q = 0; q < kQueues; ++q) L.queue[q] = take(Q * 4);
  L.t_start = take(N * 4);
  L.ff_end = o;
  L.rs = take(sizeof(RunState));
  L.locks = take(H * 4);
  L.t_end = take(N * 4);
  L.trace = take(trace ? N * 32 : 0);
  L.phase = take(N * 4);
  for (int q = 0; q < kQueues; ++q) L.qclaim[q] = take(Q * 4);
  L.groups = take(NG * sizeof(GroupState));
  L.wl_lock = take(H * 4);
  L.wl_head = take(H * 4);
  L.wl_tail = take(H * 4);
  L.wnext = take(N * 4);
  L.comm_next = take(N * 4);
  L.zero_end = o;
  L.hptr = take((H + 1) * 4);
  L.s_task = take(M * 4);
  L.s_mode = take(M);
  L.s_first = take(M);
  L.rec_pos = take(M * 4);
  L.gid = take(M * 4);
  L.gpos = take((M + 1) * 4);
  L.ucount = take(N * 4);
  L.row_ptr = take((N + 1) * 4);
  L.col = take(E * 4);
  L.indeg = take(N * 4);
  L.indeg_w = take(N * 4);
  L.remaining = take(N * 4);
  L.total = o;
  return L;
}


}  // namespace

struct spx_graph {
  spx_graph_config_t cfg{};
  int state = kBuilding;
  bool derived = false;     // device DAG valid
  bool uploaded = false;    // device copy of the inserted graph valid
  int last_status = 0;
  int last_info = 0;

  // inserted graph (host)
  std::vector<TileDesc> tiles;
  std::vector<int> tile_dtype;
  std::vector<CUtensorMap> maps;      // low-precision matrices
  // kind 0: low-precision matrix; 1: split store (the map with 128-row
  // boxes; the next map, kind 2, is the same store with 64-row boxes).  For
  // a split store ld = the slot pitch b and cols_ = the number of slots.
  struct MapInfo { uintptr_t base; size_t bytes; int ld, elem, dtype, cols_, kind; };
  std::vector<MapInfo> map_info;
  int tc_mode = 0;  // kernel family: 1 some task on the tensor cores, 2 some split-FP64 task
  std::unordered_map<uintptr_t, uint32_t> key_to_handle;
  std::vector<HandleState> hstate;
  std::vector<TaskDesc> tasks;
  std::vector<uint32_t> rec_handle, rec_seq, task_rec{0};
  std::vector<uint8_t> rec_mode;
  unsigned long long cand_edges = 0;
  unsigned long long items[kQueues] = {0, 0, 0};  // queue parts per graph queue

  // device
  int device = -1;
  void* dmem = nullptr;
  size_t dcap = 0;
  void* pinned = nullptr;   // upload mirror
  size_t pcap = 0;
  RunState* host_rs = nullptr;  // pinned copy of the run state
  cudaEvent_t done_ev = nullptr;
  cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};  // derive start, run start, run end
  cudaStream_t last_stream = nullptr;
  Layout lay{};
  DevGraph dg{};
  long long nedges = -1;
  // CUDA-graph replay of the re-execution sequence (cfg.cuda_graph)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // SPX_EXEC_STREAMS: predecessor lists (host), four streams, events
  std::vector<uint32_t> pred_ptr, pred;
  // streaming (spx_stream_begin .. spx_stream_end)
  std::vector<StreamGroup> sg;                 // per handle
  std::vector<std::vector<uint32_t>> spred;    // predecessors per task (relays included)
  std::vector<uint32_t> sout, salias;          // attachments per task; its relay (or ~0)
  uint32_t s_cap_tasks = 0, s_cap_tiles = 0, s_pub = 0, s_tiles_up = 0;
  size_t s_cap_recs = 0, s_cap_preds = 0, s_npreds = 0, s_preds_up = 0, s_recs_up = 0;
  unsigned long long s_items = 0, s_qcap = 0;
  int s_fail = 0;                              // first error of the stream
  StreamCtl s_ctl_host{};                      // the values last sent to the device
  StreamCtl* s_ctl = nullptr;                  // the kernel's copy (device memory)
  cudaStream_t s_up = nullptr;                 // uploads while the kernel runs
  cudaStream_t done_stream = nullptr;          // completion snapshots (spx_graph_tasks_done)
  std::vector<uint32_t> done_buf;
  size_t s_off_cnt = 0, s_off_succ = 0, s_off_pptr = 0, s_off_pred = 0;
  cudaStream_t xs[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr, join_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> task_ev;
  // batched execution (spx_batch_execute).  The first graph of a batch owns
  // the merged graph that runs it (batch); every member points to the
  // merged graph of its last batched run (batch_of).  The merged graph keeps
  // its members, the member of each of its tasks and a pinned copy of the
  // members' statuses.
  spx_graph* batch = nullptr;
  spx_graph* batch_of = nullptr;
  uint32_t batch_index = 0;
  std::vector<spx_graph*> members;
  std::vector<uint32_t> task_group;
  GroupState* host_groups = nullptr;
  size_t host_groups_cap = 0;
};

namespace {

int cuda_fail(cudaError_t e) {
  (void)cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return SPX_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SPX_ERR_NO_DEVICE;
  return SPX_ERR_CUDA;
}

// Operand count, shape and mode checks of the built-in ops.
// Operand count of each built-in op (-1: any, 1..16).
const int kWantNh[SPX_NUM_OPS] = {1, 2, 2, 3, 3, 2, 3, 2, 3, -1, -1, 2, 2, 3, 2, 2, 1, 2, 2, 1, 1};

int check_operands(int op, const std::vector<TileDesc>& t, const std::vector<int>& dt,
                   const unsigned* h, const int* m, int nh) {
  if (op == SPX_OP_NOP || op == SPX_OP_SPIN) return SPX_OK;
  if (nh != kWantNh[op]) return SPX_ERR_INVALID_ARG;
  // FP64 throughout, except: the solve updates (GEMM_FWD, GEMM_BWD, TRMM)
  // also run with all operands FP32 on at most 16 right-hand-side columns,
  // and COPY / AXPY convert between FP64 and FP32 in either direction.
  const bool f32_ok = op == SPX_OP_GEMM_FWD || op == SPX_OP_GEMM_BWD || op == SPX_OP_TRMM;
  const bool conv_ok = op == SPX_OP_COPY || op == SPX_OP_AXPY;
  const bool all_f32 = f32_ok && dt[h[0]] == SPX_DT_F32;
  for (int i = 0; i < nh; ++i) {
    const int d = dt[h[i]];
    if (conv_ok ? d != SPX_DT_F64 && d != SPX_DT_F32 : d != (all_f32 ? SPX_DT_F32 : SPX_DT_F64))
      return SPX_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (h[i] == h[j]) return SPX_ERR_INVALID_ARG;
  }
  const int w = nh - 1;  // written operand is the last one
  const bool atomic_ok = op == SPX_OP_GEMM_NN_ADD || op == SPX_OP_AXPY;
  auto writes = [](int md) {
    return md == SPX_WRITE || md == SPX_COMMUTATIVE_WRITE || md == SPX_MAYBE_WRITE;
  };
  if (!writes(m[w]) && !(m[w] == SPX_ATOMIC_WRITE && atomic_ok)) return SPX_ERR_INVALID_ARG;
  if ((op == SPX_OP_NBODY_PAIR || op == SPX_OP_POTRF_PANEL) && !writes(m[0]))
    return SPX_ERR_INVALID_ARG;  // both operands written
  auto R = [&](int i) { return t[h[i]].rows; };
  auto C = [&](int i) { return t[h[i]].cols; };
  bool ok = true;
  switch (op) {
    case SPX_OP_POTRF: ok = R(0) == C(0); break;
    case SPX_OP_POTRF_PANEL: ok = R(0) == C(0) && C(1) == C(0); break;
    case SPX_OP_TRSM: ok = R(0) == C(0) && C(1) == R(0); break;
    case SPX_OP_SYRK: ok = R(1) == C(1) && R(0) == R(1); break;
    case SPX_OP_GEMM_NT_SUB: ok = R(0) == R(2) && R(1) == C(2) && C(0) == C(1); break;
    case SPX_OP_GEMM_NN_ADD: ok = R(0) == R(2) && C(1) == C(2) && C(0) == R(1); break;
    case SPX_OP_TRSM_L_FWD:
    case SPX_OP_TRSM_LT_BWD: ok = R(0) == C(0) && R(1) == R(0); break;
    case SPX_OP_GEMM_FWD: ok = R(0) == R(2) && C(0) == R(1) && C(1) == C(2); break;
    case SPX_OP_GEMM_BWD: ok = R(0) == R(1) && C(0) == R(2) && C(1) == C(2); break;
    case SPX_OP_COPY:
    case SPX_OP_AXPY: ok = R(0) == R(1) && C(0) == C(1); break;
    case SPX_OP_TRMM: ok = R(0) == C(0) && C(0) == R(1) && R(2) == R(0) && C(2) == C(1); break;
    case SPX_OP_TRTRI: ok = R(0) == C(0) && R(1) == R(0) && C(1) == C(0); break;
    case SPX_OP_TRSM_INV: ok = R(0) == C(0) && C(1) == R(0) && C(1) % 32 == 0; break;
    case SPX_OP_NBODY_SELF: ok = C(0) == 8; break;
    case SPX_OP_NBODY_PAIR: ok = C(0) == 8 && C(1) == 8; break;
    case SPX_OP_SPLIT:
    case SPX_OP_SPLIT_T: break;  // the slot's shape is checked with the split store
    default: ok = false;
  }
  if (all_f32 && C(nh - 1) > 16) ok = false;
  return ok ? SPX_OK : SPX_ERR_INVALID_ARG;
}

// Find the registered low-precision matrix that holds tile h's copy and
// record the copy's position in it.
bool resolve_lowp(spx_graph* g, uint32_t h) {
  TileDesc& t = g->tiles[h];
  if (!t.lowp) return false;
  if (t.lmap >= 0) return true;
  const uintptr_t p = (uintptr_t)t.lowp;
  for (size_t m = 0; m < g->map_info.size(); ++m) {
    const auto& mi = g->map_info[m];
    if (mi.kind == 2 || p < mi.base || p >= mi.base + mi.bytes) continue;
    if (mi.kind == 1) {  // a split slot: its index is the TMA slot coordinate
      const size_t slot = (size_t)ozaki_slot_bytes(mi.ld), off = p - mi.base;
      if (off % slot || t.lowp_ld != mi.ld || t.rows > mi.ld || t.cols > mi.ld) return false;
      t.lmap = (int)m;
      t.lr0 = (int)(off / slot);
      t.lc0 = 0;
      return true;
    }
    const size_t off = p - mi.base, row_bytes = (size_t)mi.ld * mi.elem;
    if (off % mi.elem || t.lowp_ld != mi.ld) return false;
    t.lmap = (int)m;
    t.lr0 = (int)(off / row_bytes);
    t.lc0 = (int)((off % row_bytes) / mi.elem);
    return true;
  }
  return false;
}

// Low-precision tasks: TRSM writes the copy of its result; SYRK / GEMM_NT_SUB
// read the copies of their factor operands through TMA.  The copies must lie
// in a matrix registered with spx_lowp_register of the task's type, with the
// K extent a whole number of 128-byte chunks (or ending the matrix).
int check_lowp(spx_graph* g, int op, int prec, const unsigned* h) {
  const int want = prec == SPX_BF16 ? SPX_DT_BF16 : SPX_DT_F32;
  int ins[2] = {-1, -1};
  switch (op) {
    case SPX_OP_TRSM: ins[0] = (int)h[1]; break;
    case SPX_OP_POTRF_PANEL:  // split prec only: A_ik is split after its solve
      if (prec != SPX_F64_OZAKI) return SPX_ERR_INVALID_ARG;
      ins[0] = (int)h[1];
      break;
    case SPX_OP_TRSM_INV:
      ins[0] = (int)h[1];
      if (prec == SPX_F64_OZAKI) ins[1] = (int)h[0];  // V's digits feed the product
      break;
    case SPX_OP_TRTRI:  // split prec only: V is split after the inversion
      if (prec != SPX_F64_OZAKI) return SPX_ERR_INVALID_ARG;
      ins[0] = (int)h[1];
      break;
    case SPX_OP_SYRK: ins[0] = (int)h[0]; break;
    case SPX_OP_GEMM_NT_SUB: ins[0] = (int)h[0]; ins[1] = (int)h[1]; break;
    case SPX_OP_GEMM_NN_ADD:  // split prec only, K within one slot
      if (prec != SPX_F64_OZAKI) return SPX_ERR_INVALID_ARG;
      ins[0] = (int)h[0];
      ins[1] = (int)h[1];
      break;
    case SPX_OP_SPLIT:
    case SPX_OP_SPLIT_T:
      if (prec != SPX_F64_OZAKI) return SPX_ERR_INVALID_ARG;
      ins[0] = (int)h[0];
      break;
    default: return SPX_ERR_INVALID_ARG;
  }
  for (int i : ins) {
    if (i < 0) continue;
    if (!resolve_lowp(g, (uint32_t)i)) return SPX_ERR_INVALID_ARG;
    const TileDesc& t = g->tiles[i];
    const auto& mi = g->map_info[t.lmap];
    if ((mi.kind == 1) != (prec == SPX_F64_OZAKI)) return SPX_ERR_INVALID_ARG;
    if (mi.kind == 1) continue;  // slot shape checked by resolve_lowp
    if (mi.dtype != want) return SPX_ERR_INVALID_ARG;
    const int chunk = 128 / mi.elem;  // K elements per TMA box
    if (t.lc0 % chunk) return SPX_ERR_INVALID_ARG;
    // a partial last K chunk must run past the matrix edge (read as zeros)
    if (op != SPX_OP_TRSM && op != SPX_OP_TRSM_INV && t.cols % chunk &&
        t.lc0 + t.cols != mi.cols_)
      return SPX_ERR_INVALID_ARG;
  }
  return SPX_OK;
}

int ensure_device(spx_graph* g) {
  if (g->device >= 0) return SPX_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  int n = 0;
  e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return SPX_ERR_NO_DEVICE;
  e = cudaEventCreateWithFlags(&g->done_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&g->tev[i]);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaHostAlloc((void**)&g->host_rs, sizeof(RunState), cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_fail(e);
  std::memset(g->host_rs, 0, sizeof(RunState));
  g->device = dev;
  return SPX_OK;
}

void set_dev(spx_graph* g, const Layout& L, size_t N, size_t H, size_t M, size_t E, size_t Q,
             size_t NG);

// Size the device allocation for the inserted graph and upload it.
int prepare_device(spx_graph* g, cudaStream_t st) {
  int rc = ensure_device(g);
  if (rc != SPX_OK) return rc;
  const size_t N = g->tasks.size(), H = g->tiles.size(), M = g->rec_handle.size();
  // edge offsets and counts are 32-bit on the device
  if (g->cand_edges > 0xFFFFFFFFull) return SPX_ERR_INVALID_ARG;
  const size_t E = std::max<unsigned long long>(g->cand_edges, 1);
  size_t Q = std::max<unsigned long long>(
      std::max(std::max(g->items[0], g->items[1]), g->items[2]), 1);
  if (g->cfg.queue_capacity > 0) Q = (size_t)g->cfg.queue_capacity;
  if (Q > 0xFFFFFFF0ull) return SPX_ERR_INVALID_ARG;
  const size_t NG = g->task_group.empty() ? 0 : g->members.size();
  const Layout L = make_layout(N, H, M, E, Q, g->maps.size(), g->cfg.trace != 0, NG);
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  if (L.total > g->dcap) {
    if (g->dmem) {
      cudaError_t e = cudaStreamSynchronize(g->last_stream ? g->last_stream : st);
      if (e != cudaSuccess) return cuda_fail(e);
      cudaFree(g->dmem);
      g->dmem = nullptr;
      g->dcap = 0;
    }
    const size_t want = L.total + L.total / 4;
    cudaError_t e = cudaMalloc(&g->dmem, want);
    if (e != cudaSuccess) return cuda_fail(e);
    g->dcap = want;
  }
  if (L.upload_end > g->pcap) {
    if (g->pinned) {
      cudaStreamSynchronize(g->last_stream ? g->last_stream : st);
      cudaFreeHost(g->pinned);
      g->pinned = nullptr;
      g->pcap = 0;
    }
    const size_t want = L.upload_end + L.upload_end / 4;
    cudaError_t e = cudaHostAlloc(&g->pinned, want, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e);
    g->pcap = want;
  } else if (g->last_stream) {
    // the previous upload may still be reading the mirror
    cudaError_t e = cudaStreamSynchronize(g->last_stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  char* P = (char*)g->pinned;
  std::memcpy(P + L.tasks, g->tasks.data(), N * sizeof(TaskDesc));
  std::memcpy(P + L.tiles, g->tiles.data(), H * sizeof(TileDesc));
  if (!g->maps.empty()) std::memcpy(P + L.maps, g->maps.data(), g->maps.size() * sizeof(CUtensorMap));
  std::memcpy(P + L.rec_handle, g->rec_handle.data(), M * 4);
  std::memcpy(P + L.rec_seq, g->rec_seq.data(), M * 4);
  std::memcpy(P + L.rec_mode, g->rec_mode.data(), M);
  std::memcpy(P + L.task_rec, g->task_rec.data(), (N + 1) * 4);
  if (NG) std::memcpy(P + L.task_group, g->task_group.data(), N * 4);
  cudaError_t e = cudaMemcpyAsync(g->dmem, g->pinned, L.upload_end, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);

  set_dev(g, L, N, H, M, E, Q, NG);
  g->lay = L;
  g->uploaded = true;
  g->derived = false;
  g->pred_ptr.clear();  // the four-stream executor reads the new DAG back
  g->nedges = -1;
  return SPX_OK;
}

// Device pointers and sizes of the graph's allocation laid out by L.
void set_dev(spx_graph* g, const Layout& L, size_t N, size_t H, size_t M, size_t E, size_t Q,
             size_t NG) {
  char* D = (char*)g->dmem;
  DevGraph& d = g->dg;
  d = DevGraph{};
  d.ntasks = (uint32_t)N;
  d.ntiles = (uint32_t)H;
  d.nrec = (uint32_t)M;
  d.ecap = (uint32_t)E;
  d.qcap = (uint32_t)Q;
  d.trace = g->cfg.trace ? 1u : 0u;
  d.watchdog_ns = g->cfg.watchdog_ns ? g->cfg.watchdog_ns : 10000000000ull;
  d.tasks = (const TaskDesc*)(D + L.tasks);
  d.tiles = (const TileDesc*)(D + L.tiles);
  d.maps = (const CUtensorMap*)(D + L.maps);
  d.rec_handle = (const uint32_t*)(D + L.rec_handle);
  d.rec_seq = (const uint32_t*)(D + L.rec_seq);
  d.rec_mode = (const uint8_t*)(D + L.rec_mode);
  d.task_rec = (const uint32_t*)(D + L.task_rec);
  for (int q = 0; q < kQueues; ++q) {
    d.queue[q] = (uint32_t*)(D + L.queue[q]);
    d.qclaim[q] = (uint32_t*)(D + L.qclaim[q]);
  }
  d.t_start = (uint32_t*)(D + L.t_start);
  d.rs = (RunState*)(D + L.rs);
  d.locks = (uint32_t*)(D + L.locks);
  d.t_end = (uint32_t*)(D + L.t_end);
  d.trace_rec = g->cfg.trace ? (unsigned long long*)(D + L.trace) : nullptr;
  d.hptr = (uint32_t*)(D + L.hptr);
  d.s_task = (uint32_t*)(D + L.s_task);
  d.s_mode = (uint8_t*)(D + L.s_mode);
  d.s_first = (uint8_t*)(D + L.s_first);
  d.rec_pos = (uint32_t*)(D + L.rec_pos);
  d.gid = (uint32_t*)(D + L.gid);
  d.gpos = (uint32_t*)(D + L.gpos);
  d.ucount = (uint32_t*)(D + L.ucount);
  d.row_ptr = (uint32_t*)(D + L.row_ptr);
  d.col = (uint32_t*)(D + L.col);
  d.indeg = (uint32_t*)(D + L.indeg);
  d.indeg_w = (uint32_t*)(D + L.indeg_w);
  d.remaining = (uint32_t*)(D + L.remaining);
  d.phase = (uint32_t*)(D + L.phase);
  d.task_group = NG ? (const uint32_t*)(D + L.task_group) : nullptr;
  d.groups = NG ? (GroupState*)(D + L.groups) : nullptr;
  d.wl_lock = (uint32_t*)(D + L.wl_lock);
  d.wl_head = (uint32_t*)(D + L.wl_head);
  d.wl_tail = (uint32_t*)(D + L.wl_tail);
  d.wnext = (uint32_t*)(D + L.wnext);
  d.comm_next = (uint32_t*)(D + L.comm_next);
}

// Queues to "empty", tickets, locks and run state to zero.
int reset_run_state(spx_graph* g, cudaStream_t st) {
  const Layout& L = g->lay;
  char* D = (char*)g->dmem;
  cudaError_t e = cudaMemsetAsync(D + L.queue[0], 0xFF, L.ff_end - L.queue[0], st);
  if (e == cudaSuccess) e = cudaMemsetAsync(D + L.rs, 0, L.zero_end - L.rs, st);
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// Streaming: tasks inserted while the persistent kernel runs.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoAlias = 0xFFFFFFFFu;

// Queue entries a task may push (one per phase).
uint32_t task_entries(const TaskDesc& t) { return t.nphases ? t.nphases : 1u; }

// A predecessor for a new successor: p itself, or, once p's successor slots
// are all but full, the newest relay behind it: a NOP task that depends on p
// and takes p's later successors (the relay is appended to the task list).
uint32_t stream_attach_target(spx_graph* g, uint32_t p) {
  while (g->salias[p] != kNoAlias) p = g->salias[p];
  if (g->sout[p] + 1 < kStreamSucc) return p;
  TaskDesc r{};
  r.op = SPX_OP_NOP;
  r.prio = 1;
  r.flags = kFlagSerial;
  r.nphases = 1;
  r.nparts = 1;
  const uint32_t rid = (uint32_t)g->tasks.size();
  g->tasks.push_back(r);
  g->task_rec.push_back((uint32_t)g->rec_handle.size());
  g->spred.push_back({p});
  g->sout.push_back(0);
  g->salias.push_back(kNoAlias);
  g->sout[p] += 1;
  g->s_npreds += 1;
  g->s_items += 1;
  g->salias[p] = rid;
  return rid;
}

// Host-side derivation of the newly inserted task v (and of the relays it
// needs); checks the stream's capacities.
int stream_add_task(spx_graph* g, uint32_t v) {
  const uint32_t r0 = g->task_rec[v], r1 = g->task_rec[v + 1];
  std::vector<uint32_t> preds =
      stf_preds(g->sg, v, g->rec_handle.data() + r0, g->rec_mode.data() + r0, r1 - r0);
  g->spred.resize(g->tasks.size());
  g->sout.resize(g->tasks.size(), 0);
  g->salias.resize(g->tasks.size(), kNoAlias);
  for (uint32_t& p : preds) {
    p = stream_attach_target(g, p);
    g->sout[p] += 1;
  }
  g->s_npreds += preds.size();
  g->s_items += task_entries(g->tasks[v]);
  g->spred[v] = std::move(preds);
  if (g->tasks.size() > g->s_cap_tasks || g->s_npreds > g->s_cap_preds ||
      g->s_items > g->s_qcap) {
    g->s_fail = SPX_ERR_QUEUE_FULL;
    return g->s_fail;
  }
  return SPX_OK;
}

// Upload the tasks inserted since the last publication (with their tiles,
// records and predecessor lists) on the upload stream, wait for the copies,
// then raise the published count the kernel polls.
int stream_publish(spx_graph* g) {
  const size_t N = g->tasks.size(), H = g->tiles.size(), M = g->rec_handle.size();
  if (N == g->s_pub && H == g->s_tiles_up) return SPX_OK;
  const Layout& L = g->lay;
  char* D = (char*)g->dmem;
  cudaStream_t up = g->s_up;
  cudaError_t e = cudaSuccess;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(D + off, src, bytes, cudaMemcpyHostToDevice, up);
  };
  put(L.tiles + g->s_tiles_up * sizeof(TileDesc), g->tiles.data() + g->s_tiles_up,
      (H - g->s_tiles_up) * sizeof(TileDesc));
  put(L.rec_handle + g->s_recs_up * 4, g->rec_handle.data() + g->s_recs_up, (M - g->s_recs_up) * 4);
  put(L.rec_mode + g->s_recs_up, g->rec_mode.data() + g->s_recs_up, M - g->s_recs_up);
  put(L.task_rec + (size_t)g->s_pub * 4, g->task_rec.data() + g->s_pub, (N + 1 - g->s_pub) * 4);
  put(L.tasks + (size_t)g->s_pub * sizeof(TaskDesc), g->tasks.data() + g->s_pub,
      (N - g->s_pub) * sizeof(TaskDesc));
  // predecessor lists in task order, offsets continuing the published ones
  std::vector<uint32_t> ptr, pred;
  ptr.reserve(N - g->s_pub);
  size_t at = g->s_preds_up;
  for (size_t v = g->s_pub; v < N; ++v) {
    pred.insert(pred.end(), g->spred[v].begin(), g->spred[v].end());
    at += g->spred[v].size();
    ptr.push_back((uint32_t)at);
  }
  put(g->s_off_pptr + (size_t)(g->s_pub + 1) * 4, ptr.data(), ptr.size() * 4);
  put(g->s_off_pred + g->s_preds_up * 4, pred.data(), pred.size() * 4);
  // the count the kernel polls, written after the data on the same stream
  // (copies from pageable memory return once the source has been staged)
  g->s_ctl_host.published = (uint32_t)N;
  put((size_t)((char*)&g->s_ctl->published - D), &g->s_ctl_host.published, 4);
  if (e != cudaSuccess) return cuda_fail(e);
  g->s_pub = (uint32_t)N;
  g->s_tiles_up = (uint32_t)H;
  g->s_recs_up = M;
  g->s_preds_up = at;
  return SPX_OK;
}

// Tell the kernel that no task follows (it drains and exits).
void stream_close(spx_graph* g) {
  g->s_ctl_host.end = 1u;
  cudaMemcpyAsync(&g->s_ctl->end, &g->s_ctl_host.end, 4, cudaMemcpyHostToDevice, g->s_up);
  g->state = kRunning;
}

}  // namespace

extern "C" {

void spx_config_default(spx_graph_config_t* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->executor = SPX_EXEC_PERSISTENT;
  cfg->watchdog_ns = 10000000000ull;
}

int spx_abi_version(void) { return 1; }

const char* spx_strerror(int code) {
  switch (code) {
    case SPX_OK: return "ok";
    case SPX_NOT_SPD: return "matrix is not positive definite (info = failing column)";
    case SPX_ERR_INVALID_ARG: return "invalid argument";
    case SPX_ERR_BAD_HANDLE: return "unknown tile handle or task id";
    case SPX_ERR_STATE: return "call not allowed in the graph's current state";
    case SPX_ERR_OOM: return "out of memory";
    case SPX_ERR_QUEUE_FULL: return "device work queue capacity exceeded";
    case SPX_ERR_TIMEOUT: return "timeout (device watchdog or host wait)";
    case SPX_ERR_CUDA: return "CUDA runtime error";
    case SPX_ERR_BAD_OP: return "device met an unknown task op";
    case SPX_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown status code";
  }
}

int spx_graph_create(spx_graph_t* out, const spx_graph_config_t* cfg) {
  if (!out) return SPX_ERR_INVALID_ARG;
  *out = nullptr;
  spx_graph* g = new (std::nothrow) spx_graph();
  if (!g) return SPX_ERR_OOM;
  spx_config_default(&g->cfg);
  if (cfg) {
    if (cfg->num_ctas < 0 || cfg->queue_capacity < 0 || cfg->priorities < 0 ||
        cfg->priorities > 1 ||
        (cfg->executor != SPX_EXEC_PERSISTENT && cfg->executor != SPX_EXEC_PER_TASK &&
         cfg->executor != SPX_EXEC_STREAMS)) {
      delete g;
      return SPX_ERR_INVALID_ARG;
    }
    g->cfg = *cfg;
    if (!g->cfg.watchdog_ns) g->cfg.watchdog_ns = 10000000000ull;
  }
  *out = g;
  return SPX_OK;
}

int spx_tile_register(spx_graph_t g, void* dev_ptr, int rows, int cols, int ld, int dtype,
                      void* lowp_ptr, int lowp_ld, unsigned* out_handle) {
  if (!g || !dev_ptr || !out_handle || rows < 1 || cols < 1 || ld < cols ||
      dtype < SPX_DT_F64 || dtype > SPX_DT_BF16 || (lowp_ptr && lowp_ld < cols))
    return SPX_ERR_INVALID_ARG;
  if (g->state != kBuilding && g->state != kStreaming) return SPX_ERR_STATE;
  const uintptr_t key = (uintptr_t)dev_ptr;
  auto it = g->key_to_handle.find(key);
  if (it != g->key_to_handle.end()) {
    const TileDesc& t = g->tiles[it->second];
    if (t.rows != rows || t.cols != cols || t.ld != ld || g->tile_dtype[it->second] != dtype)
      return SPX_ERR_INVALID_ARG;
    *out_handle = it->second;
    return SPX_OK;
  }
  if (g->state == kStreaming) return SPX_ERR_STATE;  // tiles come before the stream
  const uint32_t h = (uint32_t)g->tiles.size();
  g->tiles.push_back(
      TileDesc{dev_ptr, lowp_ptr, rows, cols, ld, lowp_ptr ? lowp_ld : 0, -1, 0, 0, dtype});
  g->tile_dtype.push_back(dtype);
  g->hstate.emplace_back();
  g->key_to_handle.emplace(key, h);
  g->uploaded = false;
  *out_handle = h;
  return SPX_OK;
}

int spx_lowp_register(spx_graph_t g, void* dev_ptr, int rows, int cols, int ld, int dtype,
                      unsigned* out_map) {
  if (!g || !dev_ptr || rows < 1 || cols < 1 || ld < cols ||
      (dtype != SPX_DT_BF16 && dtype != SPX_DT_F32))
    return SPX_ERR_INVALID_ARG;
  if (g->state != kBuilding) return SPX_ERR_STATE;
  const int elem = dtype == SPX_DT_BF16 ? 2 : 4;
  for (size_t m = 0; m < g->map_info.size(); ++m)
    if (g->map_info[m].base == (uintptr_t)dev_ptr) {
      if (out_map) *out_map = (unsigned)m;
      return SPX_OK;
    }
  CUtensorMap map;
  const int rc = make_tmap(&map, dev_ptr, rows, cols, ld, dtype);
  if (rc != SPX_OK) return rc;
  g->maps.push_back(map);
  g->map_info.push_back({(uintptr_t)dev_ptr, (size_t)rows * ld * elem, ld, elem, dtype, cols, 0});
  g->uploaded = false;
  if (out_map) *out_map = (unsigned)(g->maps.size() - 1);
  return SPX_OK;
}

long long spx_ozaki_slot_bytes(int b) { return ozaki_slot_bytes(b); }

int spx_ozaki_register(spx_graph_t g, void* dev_ptr, int nslots, int b, unsigned* out_map) {
  if (!g || !dev_ptr || nslots < 1 || !ozaki_slot_bytes(b)) return SPX_ERR_INVALID_ARG;
  if (g->state != kBuilding) return SPX_ERR_STATE;
  for (size_t m = 0; m < g->map_info.size(); ++m)
    if (g->map_info[m].base == (uintptr_t)dev_ptr) {
      const auto& mi = g->map_info[m];
      if (mi.kind != 1 || mi.ld != b || mi.cols_ != nslots) return SPX_ERR_INVALID_ARG;
      if (out_map) *out_map = (unsigned)m;
      return SPX_OK;
    }
  CUtensorMap ma, mb;
  int rc = make_tmap_ozaki(&ma, dev_ptr, nslots, b, 128);
  if (rc == SPX_OK) rc = make_tmap_ozaki(&mb, dev_ptr, nslots, b, 64);
  if (rc != SPX_OK) return rc;
  const size_t bytes = (size_t)nslots * (size_t)ozaki_slot_bytes(b);
  g->maps.push_back(ma);
  g->maps.push_back(mb);
  g->map_info.push_back({(uintptr_t)dev_ptr, bytes, b, 2, SPX_DT_BF16, nslots, 1});
  g->map_info.push_back({(uintptr_t)dev_ptr, bytes, b, 2, SPX_DT_BF16, nslots, 2});
  g->uploaded = false;
  if (out_map) *out_map = (unsigned)(g->maps.size() - 2);
  return SPX_OK;
}

int spx_task_insert(spx_graph_t g, int op, const unsigned* handles, const int* modes, int nh,
                    int priority, int prec, unsigned* out_task) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state != kBuilding && g->state != kStreaming) return SPX_ERR_STATE;
  if (g->state == kStreaming) {
    if (g->s_fail) return g->s_fail;
    // the running kernel's family is fixed; the capacities hold
    const int mode = prec == SPX_F64 ? 0 : prec == SPX_F64_OZAKI ? 2 : 1;
    if (mode > g->tc_mode || (mode == 1 && g->tc_mode == 2)) return SPX_ERR_INVALID_ARG;
    if (g->tasks.size() + 1 > g->s_cap_tasks || g->rec_handle.size() + (size_t)nh > g->s_cap_recs)
      return SPX_ERR_QUEUE_FULL;
  }
  if (op < 0 || op >= SPX_NUM_OPS || nh < 1 || nh > kMaxHandles || !handles || !modes ||
      priority < 0 || prec < SPX_F64 || prec > SPX_F64_OZAKI)
    return SPX_ERR_INVALID_ARG;
  if (g->tasks.size() >= kMaxTasks) return SPX_ERR_INVALID_ARG;
  for (int i = 0; i < nh; ++i) {
    if (handles[i] >= g->tiles.size()) return SPX_ERR_BAD_HANDLE;
    if (modes[i] < SPX_READ || modes[i] > SPX_MAYBE_WRITE) return SPX_ERR_INVALID_ARG;
  }
  int rc = check_operands(op, g->tiles, g->tile_dtype, handles, modes, nh);
  if (rc != SPX_OK) return rc;
  if ((op == SPX_OP_TRSM_INV || op == SPX_OP_SPLIT || op == SPX_OP_SPLIT_T) && prec == SPX_F64)
    return SPX_ERR_INVALID_ARG;  // tensor cores / split store only
  if (op == SPX_OP_GEMM_NN_ADD && prec == SPX_F64_OZAKI && modes[2] == SPX_ATOMIC_WRITE)
    return SPX_ERR_INVALID_ARG;  // the split product's update is not atomic
  if (prec != SPX_F64) {
    rc = check_lowp(g, op, prec, handles);
    if (rc != SPX_OK) return rc;
  }

  // Merge repeated handles (the same mode twice stays, else WRITE) and order
  // this task's accesses by handle (the lock order on the device).
  uint32_t hh[kMaxHandles];
  int mm[kMaxHandles];
  int k = 0;
  for (int i = 0; i < nh; ++i) {
    int j = 0;
    while (j < k && hh[j] != handles[i]) ++j;
    if (j < k) {
      if (mm[j] != modes[i]) mm[j] = SPX_WRITE;
    } else {
      hh[k] = handles[i];
      mm[k] = modes[i];
      ++k;
    }
  }
  for (int i = 1; i < k; ++i)
    for (int j = i; j > 0 && hh[j - 1] > hh[j]; --j) {
      std::swap(hh[j - 1], hh[j]);
      std::swap(mm[j - 1], mm[j]);
    }

  TaskDesc t{};
  t.op = (uint8_t)op;
  t.prec = (uint8_t)prec;
  t.prio = (uint8_t)(priority > 2 ? 2 : priority);
  t.flags = priority >= 2 ? kFlagFine : 0;
  for (int i = 0; i < k; ++i) {
    if (mm[i] == SPX_COMMUTATIVE_WRITE) t.flags |= kFlagComm;
    // the written operand of GEMM_NN_ADD / AXPY accumulated atomically
    if (mm[i] == SPX_ATOMIC_WRITE && hh[i] == handles[nh - 1] &&
        (op == SPX_OP_GEMM_NN_ADD || op == SPX_OP_AXPY))
      t.flags |= kFlagAtomic;
  }
  for (int i = 0; i < 3; ++i) t.h[i] = i < nh ? handles[i] : 0;
  uint32_t items = 1;  // queue entries over all phases
  if (g->cfg.no_split) {
    t.flags |= kFlagSerial;
    t.nphases = 1;
    t.nparts = 1;
  } else {
    t.nphases = task_phases(t, g->tiles.data());
    t.nparts = phase_parts(task_phase_units(t, g->tiles.data(), 0));
    items = 0;
    for (uint32_t ph = 0; ph < t.nphases; ++ph)
      items += phase_parts(task_phase_units(t, g->tiles.data(), ph));
    if (t.flags & kFlagComm)  // an acquire entry again for each lock handed over
      for (int i = 0; i < k; ++i) items += mm[i] == SPX_COMMUTATIVE_WRITE ? 1u : 0u;
  }
  t.arg = 0;

  const uint32_t tid = (uint32_t)g->tasks.size();
  for (int i = 0; i < k; ++i) {
    HandleState& s = g->hstate[hh[i]];
    const int m = mm[i];
    if (s.last_mode == m && m != SPX_WRITE && m != SPX_MAYBE_WRITE) {
      g->cand_edges += s.prev_size;
      s.last_size += 1;
    } else {
      g->cand_edges += s.last_size;
      s.prev_size = s.last_size;
      s.last_size = 1;
      s.last_mode = m;
    }
    g->rec_handle.push_back(hh[i]);
    g->rec_seq.push_back(s.count++);
    g->rec_mode.push_back((uint8_t)m);
  }
  g->task_rec.push_back((uint32_t)g->rec_handle.size());
  g->tasks.push_back(t);
  g->items[graph_queue(t.prio)] += items;
  if (prec != SPX_F64) {
    const int mode = prec == SPX_F64_OZAKI ? 2 : 1;
    if (mode > g->tc_mode) g->tc_mode = mode;
  }
  g->uploaded = false;
  if (out_task) *out_task = tid;
  if (g->state == kStreaming) return stream_add_task(g, tid);
  return SPX_OK;
}

int spx_task_set_arg(spx_graph_t g, unsigned task, long long arg) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (task >= g->tasks.size()) return SPX_ERR_BAD_HANDLE;
  if (g->state != kBuilding && !(g->state == kStreaming && task >= g->s_pub))
    return SPX_ERR_STATE;
  g->tasks[task].arg = arg;
  g->uploaded = false;
  return SPX_OK;
}

int spx_task_set_scalar(spx_graph_t g, unsigned task, double alpha) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (task >= g->tasks.size()) return SPX_ERR_BAD_HANDLE;
  if (g->state != kBuilding && !(g->state == kStreaming && task >= g->s_pub))
    return SPX_ERR_STATE;
  if (g->tasks[task].op != SPX_OP_AXPY || !(alpha == alpha) || alpha == 0.0 ||
      alpha - alpha != 0.0)
    return SPX_ERR_INVALID_ARG;
  long long bits;
  std::memcpy(&bits, &alpha, sizeof bits);  // the device reads the FP64 bits
  g->tasks[task].arg = bits;
  g->uploaded = false;
  return SPX_OK;
}

int spx_graph_assign_priorities(spx_graph_t g) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state == kRunning) return SPX_ERR_STATE;
  const size_t N = g->tasks.size(), H = g->tiles.size();
  if (N == 0) return SPX_ERR_STATE;
  // weight: phases of the task (its dependent steps; serial tasks one)
  std::vector<double> w(N), tl(N), bl(N);
  for (size_t u = 0; u < N; ++u) {  // the op's phases (a commutative task's lock phase aside)
    const TaskDesc& t = g->tasks[u];
    w[u] = (t.flags & kFlagSerial) ? 1.0 : std::max<uint32_t>(op_phases(t.op, t.prec, g->tiles.data(), t.h), 1);
  }
  auto groups = [](int m) {
    return m == SPX_READ || m == SPX_COMMUTATIVE_WRITE || m == SPX_ATOMIC_WRITE;
  };
  struct Fwd { int mode = -1; double last = 0.0, prev = 0.0; };
  std::vector<Fwd> f(H);
  for (size_t u = 0; u < N; ++u) {  // top levels, insertion order
    double t = 0.0;
    for (uint32_t r = g->task_rec[u]; r < g->task_rec[u + 1]; ++r) {
      const Fwd& s = f[g->rec_handle[r]];
      const int m = g->rec_mode[r];
      if (s.mode < 0) continue;
      t = std::max(t, (s.mode == m && groups(m)) ? s.prev : s.last);
    }
    tl[u] = t;
    const double end = t + w[u];
    for (uint32_t r = g->task_rec[u]; r < g->task_rec[u + 1]; ++r) {
      Fwd& s = f[g->rec_handle[r]];
      const int m = g->rec_mode[r];
      if (s.mode == m && groups(m)) {
        s.last = std::max(s.last, end);
      } else {
        s.prev = s.mode < 0 ? 0.0 : s.last;
        s.last = end;
        s.mode = m;
      }
    }
  }
  struct Bwd { int mode = -1; double cur = 0.0, next = 0.0; };
  std::vector<Bwd> b(H);
  for (size_t k = N; k-- > 0;) {  // bottom levels, reverse insertion order
    double s_max = 0.0;
    for (uint32_t r = g->task_rec[k]; r < g->task_rec[k + 1]; ++r) {
      const Bwd& s = b[g->rec_handle[r]];
      const int m = g->rec_mode[r];
      if (s.mode < 0) continue;
      s_max = std::max(s_max, (s.mode == m && groups(m)) ? s.next : s.cur);
    }
    bl[k] = w[k] + s_max;
    for (uint32_t r = g->task_rec[k]; r < g->task_rec[k + 1]; ++r) {
      Bwd& s = b[g->rec_handle[r]];
      const int m = g->rec_mode[r];
      if (s.mode == m && groups(m)) {
        s.cur = std::max(s.cur, bl[k]);
      } else {
        s.next = s.mode < 0 ? 0.0 : s.cur;
        s.cur = bl[k];
        s.mode = m;
      }
    }
  }
  double cp = 0.0;
  for (size_t u = 0; u < N; ++u) cp = std::max(cp, tl[u] + bl[u]);
  g->items[0] = g->items[1] = g->items[2] = 0;
  for (size_t u = 0; u < N; ++u) {
    TaskDesc& t = g->tasks[u];
    const double slack = cp - tl[u] - bl[u];
    const int cls = slack <= 1e-9 * cp ? 2 : (slack <= 0.1 * cp ? 1 : 0);
    t.prio = (uint8_t)cls;
    uint32_t items = 1;
    if (!(t.flags & kFlagSerial)) {
      t.flags = (uint8_t)((t.flags & ~kFlagFine) | (cls == 2 ? kFlagFine : 0));
      t.nphases = task_phases(t, g->tiles.data());  // the TRSM row form has fewer
      t.nparts = phase_parts(task_phase_units(t, g->tiles.data(), 0));
      items = 0;
      for (uint32_t ph = 0; ph < t.nphases; ++ph)
        items += phase_parts(task_phase_units(t, g->tiles.data(), ph));
      if (t.flags & kFlagComm)
        for (uint32_t r = g->task_rec[u]; r < g->task_rec[u + 1]; ++r)
          items += g->rec_mode[r] == SPX_COMMUTATIVE_WRITE ? 1u : 0u;
    }
    g->items[graph_queue(t.prio)] += items;
  }
  g->uploaded = false;
  g->derived = false;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  return SPX_OK;
}

int spx_graph_derive(spx_graph_t g, void* stream) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state == kRunning || g->state == kStreaming) return SPX_ERR_STATE;
  if (g->tasks.empty()) return SPX_ERR_STATE;
  if (g->cfg.priorities == 1 && g->state == kBuilding) {
    const int rc = spx_graph_assign_priorities(g);
    if (rc != SPX_OK) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = SPX_OK;
  if (!g->uploaded) rc = prepare_device(g, st);
  if (rc != SPX_OK) return rc;
  rc = reset_run_state(g, st);
  if (rc != SPX_OK) return rc;
  cudaError_t e = launch_derive(g->dg, st);
  if (e != cudaSuccess) return cuda_fail(e);
  g->derived = true;
  g->nedges = -1;
  g->last_stream = st;
  if (g->state == kBuilding) g->state = kFrozen;
  return SPX_OK;
}

// The sequence that re-runs an uploaded (and, for the persistent executor,
// derived) graph: run-state reset, queue initialisation, executor, status
// copy.  Enqueued on st, or captured into a CUDA graph.
int enqueue_rerun(spx_graph* g, cudaStream_t st) {
  int rc = reset_run_state(g, st);
  if (rc != SPX_OK) return rc;
  cudaError_t e;
  if (g->cfg.executor == SPX_EXEC_PER_TASK) {
    e = launch_per_task(g->dg, g->tasks.data(), g->tiles.data(), g->tc_mode, st);
  } else {
    e = launch_init(g->dg, st);
    if (e == cudaSuccess) e = launch_persistent(g->dg, g->cfg.num_ctas, g->tc_mode, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->host_rs, g->dg.rs, sizeof(RunState), cudaMemcpyDeviceToHost, st);
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

int build_replay(spx_graph* g) {
  cudaError_t e = cudaSuccess;
  if (!g->cap_stream) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  const int rc = enqueue_rerun(g, g->cap_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->cap_stream, &graph);
  if (rc != SPX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaGraphInstantiate(&g->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->gexec = nullptr;
    return cuda_fail(e);
  }
  return SPX_OK;
}

// SPX_EXEC_STREAMS set-up: the derived DAG read back once as predecessor
// lists, the four streams, and the events (created once, reused).
int prepare_streams(spx_graph* g, cudaStream_t st) {
  const size_t N = g->tasks.size();
  cudaError_t e = cudaSuccess;
  if (g->pred_ptr.size() != N + 1) {
    e = cudaStreamSynchronize(st);  // the derivation has to finish first
    if (e != cudaSuccess) return cuda_fail(e);
    long long ne = 0;
    int rc = spx_graph_sizes(g, nullptr, &ne, nullptr, nullptr);
    if (rc != SPX_OK) return rc;
    std::vector<uint32_t> rp(N + 1), col((size_t)std::max<long long>(ne, 1));
    e = cudaMemcpy(rp.data(), g->dg.row_ptr, (N + 1) * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ne > 0)
      e = cudaMemcpy(col.data(), g->dg.col, (size_t)ne * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    g->pred_ptr.assign(N + 1, 0);
    for (size_t u = 0; u < N; ++u)
      for (uint32_t k = rp[u]; k < rp[u + 1]; ++k) ++g->pred_ptr[col[k] + 1];
    for (size_t v = 0; v < N; ++v) g->pred_ptr[v + 1] += g->pred_ptr[v];
    g->pred.assign((size_t)std::max<long long>(ne, 1), 0);
    std::vector<uint32_t> fill(g->pred_ptr.begin(), g->pred_ptr.end() - 1);
    for (size_t u = 0; u < N; ++u)
      for (uint32_t k = rp[u]; k < rp[u + 1]; ++k) g->pred[fill[col[k]]++] = (uint32_t)u;
  }
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    if (!g->xs[i]) e = cudaStreamCreateWithFlags(&g->xs[i], cudaStreamNonBlocking);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    if (!g->join_ev[i]) e = cudaEventCreateWithFlags(&g->join_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess && !g->fork_ev) e = cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming);
  while (e == cudaSuccess && g->task_ev.size() < N) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) g->task_ev.push_back(ev);
  }
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

// Per-task launches over four streams (see SPX_EXEC_STREAMS), joined on st.
cudaError_t launch_streams(spx_graph* g, cudaStream_t st) {
  persistent_max_ctas(nullptr);
  const size_t N = g->tasks.size();
  auto stream_of = [&](size_t u) {
    return (g->tasks[u].flags & kFlagComm) ? 0 : (int)(u % 4);
  };
  cudaError_t e = cudaEventRecord(g->fork_ev, st);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(g->xs[i], g->fork_ev, 0);
  for (size_t u = 0; u < N && e == cudaSuccess; ++u) {
    const int si = stream_of(u);
    for (uint32_t k = g->pred_ptr[u]; k < g->pred_ptr[u + 1] && e == cudaSuccess; ++k)
      if (stream_of(g->pred[k]) != si) e = cudaStreamWaitEvent(g->xs[si], g->task_ev[g->pred[k]], 0);
    if (e == cudaSuccess)
      e = launch_task(g->dg, (uint32_t)u, g->tasks[u], g->tiles.data(), g->tc_mode, g->xs[si]);
    if (e == cudaSuccess) e = cudaEventRecord(g->task_ev[u], g->xs[si]);
  }
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = cudaEventRecord(g->join_ev[i], g->xs[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g->join_ev[i], 0);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

int spx_graph_execute(spx_graph_t g, void* stream) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state == kRunning || g->state == kDone || g->state == kStreaming) return SPX_ERR_STATE;
  if (g->tasks.empty()) return SPX_ERR_STATE;
  g->batch_of = nullptr;  // runs alone from now on
  if (g->cfg.priorities == 1 && g->state == kBuilding) {
    const int prc = spx_graph_assign_priorities(g);
    if (prc != SPX_OK) return prc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = SPX_OK;
  cudaError_t e = cudaSuccess;
  if (!g->uploaded) {
    rc = prepare_device(g, st);
    if (rc != SPX_OK) return rc;
  }
  const bool replay = g->cfg.cuda_graph && g->state == kFrozen &&
                      g->cfg.executor != SPX_EXEC_STREAMS &&
                      (g->cfg.executor == SPX_EXEC_PER_TASK || g->derived);
  if (replay) {
    if (!g->gexec) {
      rc = build_replay(g);
      if (rc != SPX_OK) return rc;
    }
    e = cudaEventRecord(g->tev[0], st);
    if (e == cudaSuccess) e = cudaEventRecord(g->tev[1], st);
    if (e == cudaSuccess) e = cudaGraphLaunch(g->gexec, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->tev[2], st);
    if (e == cudaSuccess) e = cudaEventRecord(g->done_ev, st);
    if (e != cudaSuccess) return cuda_fail(e);
    g->last_stream = st;
    g->state = kRunning;
    return SPX_OK;
  }
  e = cudaEventRecord(g->tev[0], st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (g->cfg.executor == SPX_EXEC_PER_TASK) {
    rc = reset_run_state(g, st);
    if (rc != SPX_OK) return rc;
    e = cudaEventRecord(g->tev[1], st);
    if (e == cudaSuccess) e = launch_per_task(g->dg, g->tasks.data(), g->tiles.data(), g->tc_mode, st);
  } else if (g->cfg.executor == SPX_EXEC_STREAMS) {
    rc = g->derived ? reset_run_state(g, st) : spx_graph_derive(g, stream);
    if (rc == SPX_OK) rc = prepare_streams(g, st);
    if (rc != SPX_OK) return rc;
    e = cudaEventRecord(g->tev[1], st);
    if (e == cudaSuccess) e = launch_streams(g, st);
  } else {
    if (!g->derived) {
      rc = spx_graph_derive(g, stream);  // also resets the run state
      if (rc != SPX_OK) return rc;
    } else {
      rc = reset_run_state(g, st);
      if (rc == SPX_OK) {
        e = launch_init(g->dg, st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
      if (rc != SPX_OK) return rc;
    }
    e = cudaEventRecord(g->tev[1], st);
    if (e == cudaSuccess) e = launch_persistent(g->dg, g->cfg.num_ctas, g->tc_mode, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(g->tev[2], st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemcpyAsync(g->host_rs, g->dg.rs, sizeof(RunState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && g->dg.groups)
    e = cudaMemcpyAsync(g->host_groups, g->dg.groups, g->members.size() * sizeof(GroupState),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(g->done_ev, st);
  if (e != cudaSuccess) return cuda_fail(e);
  g->last_stream = st;
  g->state = kRunning;
  return SPX_OK;
}

int spx_graph_host_preds(spx_graph_t g, unsigned* pred_ptr, unsigned* pred, long long cap,
                         long long* total) {
  if (!g || !pred_ptr || (cap > 0 && !pred)) return SPX_ERR_INVALID_ARG;
  std::vector<StreamGroup> sg(g->tiles.size());
  const size_t N = g->tasks.size();
  long long at = 0;
  pred_ptr[0] = 0;
  for (size_t v = 0; v < N; ++v) {
    const uint32_t r0 = g->task_rec[v], r1 = g->task_rec[v + 1];
    const std::vector<uint32_t> p = stf_preds(sg, (uint32_t)v, g->rec_handle.data() + r0,
                                              g->rec_mode.data() + r0, r1 - r0);
    for (uint32_t x : p) {
      if (at < cap) pred[at] = x;
      ++at;
    }
    pred_ptr[v + 1] = (unsigned)std::min<long long>(at, 0xFFFFFFFFll);
  }
  if (total) *total = at;
  return at > cap ? SPX_ERR_QUEUE_FULL : SPX_OK;
}

int spx_stream_begin(spx_graph_t g, void* stream, int max_tasks, int max_tiles,
                     long long max_records, long long max_preds) {
  if (!g || max_tasks < 1 || max_tiles < 1 || max_records < 1 || max_preds < 1 ||
      (unsigned)max_tasks > kMaxTasks)
    return SPX_ERR_INVALID_ARG;
  if (g->state != kBuilding) return SPX_ERR_STATE;
  if (g->cfg.executor != SPX_EXEC_PERSISTENT || g->cfg.cuda_graph || g->cfg.no_split)
    return SPX_ERR_INVALID_ARG;
  int rc = ensure_device(g);
  if (rc != SPX_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)max_tasks, H = (size_t)max_tiles, M = (size_t)max_records,
               P = (size_t)max_preds;
  if (g->tasks.size() > N || g->tiles.size() > H || g->rec_handle.size() > M)
    return SPX_ERR_INVALID_ARG;
  // A tile's copy position is resolved at its first low-precision / split
  // use; tile descriptors are uploaded as they are registered, so resolve
  // them all now (no tile with a copy may be registered while streaming).
  for (uint32_t h = 0; h < g->tiles.size(); ++h)
    if (g->tiles[h].lowp && !resolve_lowp(g, h)) return SPX_ERR_INVALID_ARG;
  // queue entries: one per phase of a task (bounded by the tasks' phases;
  // 48 per task covers tiles up to 512 and the split ops)
  const size_t Q = N * 48;
  if (Q > 0xFFFFFFF0ull) return SPX_ERR_INVALID_ARG;
  const Layout L = make_layout(N, H, M, 1, Q, g->maps.size(), g->cfg.trace != 0, 0);
  size_t o = L.total;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1), 256);
    return at;
  };
  g->s_off_cnt = take(N * 4);
  g->s_off_succ = take(N * kStreamSucc * 4);
  g->s_off_pptr = take((N + 1) * 4);
  g->s_off_pred = take(P * 4);
  const size_t off_ctl = take(sizeof(StreamCtl));
  cudaError_t e = cudaSuccess;
  if (g->dmem && o > g->dcap) {
    if (g->last_stream) cudaStreamSynchronize(g->last_stream);
    cudaFree(g->dmem);
    g->dmem = nullptr;
    g->dcap = 0;
  }
  if (!g->dmem) {
    e = cudaMalloc(&g->dmem, o);
    if (e != cudaSuccess) return cuda_fail(e);
    g->dcap = o;
  }
  if (!g->s_up) {
    e = cudaStreamCreateWithFlags(&g->s_up, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  g->s_ctl = (StreamCtl*)((char*)g->dmem + off_ctl);
  g->s_ctl_host = StreamCtl{};
  g->lay = L;
  set_dev(g, L, N, H, M, 1, Q, 0);
  char* D = (char*)g->dmem;
  DevGraph& d = g->dg;
  d.sctl = g->s_ctl;
  d.succ_cnt = (uint32_t*)(D + g->s_off_cnt);
  d.succ = (uint32_t*)(D + g->s_off_succ);
  d.pred_ptr = (const uint32_t*)(D + g->s_off_pptr);
  d.pred = (const uint32_t*)(D + g->s_off_pred);
  g->uploaded = false;  // the graph's run layout is the stream's now
  g->derived = false;
  g->nedges = -1;
  g->pred_ptr.clear();
  // run state, queues, successor slots; the tile maps are fixed from here on
  rc = reset_run_state(g, g->s_up);
  if (rc != SPX_OK) return rc;
  e = cudaMemsetAsync(D + g->s_off_cnt, 0, N * 4, g->s_up);
  if (e == cudaSuccess) e = cudaMemsetAsync(D + g->s_off_succ, 0xFF, N * kStreamSucc * 4, g->s_up);
  if (e == cudaSuccess) e = cudaMemsetAsync(D + g->s_off_pptr, 0, 4, g->s_up);
  if (e == cudaSuccess) e = cudaMemsetAsync(D + off_ctl, 0, sizeof(StreamCtl), g->s_up);
  if (e == cudaSuccess && !g->maps.empty())
    e = cudaMemcpyAsync(D + L.maps, g->maps.data(), g->maps.size() * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice, g->s_up);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->s_up);
  if (e != cudaSuccess) return cuda_fail(e);
  // host-side derivation of the tasks inserted so far
  g->s_cap_tasks = (uint32_t)N;
  g->s_cap_tiles = (uint32_t)H;
  g->s_cap_recs = M;
  g->s_cap_preds = P;
  g->s_qcap = Q;
  g->s_pub = g->s_tiles_up = 0;
  g->s_recs_up = g->s_preds_up = g->s_npreds = 0;
  g->s_items = 0;
  g->s_fail = 0;
  g->sg.assign(g->tiles.size(), StreamGroup{});
  g->spred.assign(g->tasks.size(), {});
  g->sout.assign(g->tasks.size(), 0);
  g->salias.assign(g->tasks.size(), kNoAlias);
  g->state = kStreaming;
  const size_t n0 = g->tasks.size();
  for (size_t v = 0; v < n0 && rc == SPX_OK; ++v) rc = stream_add_task(g, (uint32_t)v);
  if (rc == SPX_OK) rc = stream_publish(g);
  if (rc != SPX_OK) {
    g->state = kBuilding;
    return rc;
  }
  // the kernel: admits published tasks and runs them until the stream ends
  e = cudaEventRecord(g->tev[0], st);
  if (e == cudaSuccess) e = cudaEventRecord(g->tev[1], st);
  if (e == cudaSuccess) e = launch_persistent(g->dg, g->cfg.num_ctas, g->tc_mode, st);
  if (e == cudaSuccess) e = cudaEventRecord(g->tev[2], st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->host_rs, g->dg.rs, sizeof(RunState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(g->done_ev, st);
  if (e != cudaSuccess) {
    stream_close(g);
    return cuda_fail(e);
  }
  g->last_stream = st;
  return SPX_OK;
}

int spx_stream_flush(spx_graph_t g) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state != kStreaming) return SPX_ERR_STATE;
  if (g->s_fail) return g->s_fail;
  return stream_publish(g);
}

int spx_stream_copy_h2d(spx_graph_t g, void* dev_dst, size_t dpitch, const void* host_src,
                        size_t spitch, size_t width_bytes, size_t rows) {
  if (!g || !dev_dst || !host_src || width_bytes > dpitch || width_bytes > spitch)
    return SPX_ERR_INVALID_ARG;
  if (g->state != kStreaming) return SPX_ERR_STATE;
  if (g->s_fail) return g->s_fail;
  if (!rows || !width_bytes) return SPX_OK;
  // on the upload stream: ahead of the next publication's count
  const cudaError_t e = cudaMemcpy2DAsync(dev_dst, dpitch, host_src, spitch, width_bytes, rows,
                                          cudaMemcpyHostToDevice, g->s_up);
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

int spx_stream_end(spx_graph_t g) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state != kStreaming) return SPX_ERR_STATE;
  const int rc = g->s_fail ? g->s_fail : stream_publish(g);
  stream_close(g);
  return rc;
}

int spx_graph_wait(spx_graph_t g, unsigned long long timeout_ns, int* info) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (info) *info = 0;
  if (g->state == kDone) {
    if (info) *info = g->last_info;
    return g->last_status;
  }
  if (g->state != kRunning) return SPX_ERR_STATE;
  if (g->batch_of) {
    // a member of a batched run: wait for the merged graph, then give every
    // member its own status (a run-wide error, else the member's)
    spx_graph* B = g->batch_of;
    const int rc = spx_graph_wait(B, timeout_ns, nullptr);
    if (rc == SPX_ERR_TIMEOUT && B->state == kRunning) return rc;
    for (spx_graph* m : B->members) {
      if (!m || m->batch_of != B || m->state != kRunning) continue;
      m->state = kDone;
      if (B->last_status != SPX_OK) {
        m->last_status = B->last_status;
        m->last_info = B->last_info;
      } else {
        m->last_status = (int)(int32_t)B->host_groups[m->batch_index].status;
        m->last_info = B->host_groups[m->batch_index].info;
      }
    }
    if (info) *info = g->last_info;
    return g->last_status;
  }
  const auto t0 = std::chrono::steady_clock::now();
  long spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(g->done_ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      g->state = kDone;
      g->last_status = cuda_fail(e);
      return g->last_status;
    }
    if (timeout_ns) {
      const auto dt = std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if ((unsigned long long)dt > timeout_ns) return SPX_ERR_TIMEOUT;
    }
    if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  g->state = kDone;
  const RunState& r = *g->host_rs;
  g->last_status = (int)(int32_t)r.status;  // SPX_OK, SPX_NOT_SPD or a negative code
  g->last_info = r.info;
  if (info) *info = g->last_info;
  return g->last_status;
}

int spx_graph_sizes(spx_graph_t g, long long* ntasks, long long* nedges, long long* naccesses,
                    long long* ntiles) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (ntasks) *ntasks = (long long)g->tasks.size();
  if (naccesses) *naccesses = (long long)g->rec_handle.size();
  if (ntiles) *ntiles = (long long)g->tiles.size();
  if (nedges) {
    *nedges = -1;
    if (g->derived && g->state != kRunning) {
      if (g->nedges < 0) {
        uint32_t e = 0;
        cudaError_t err = cudaStreamSynchronize(g->last_stream);
        if (err == cudaSuccess)
          err = cudaMemcpy(&e, g->dg.row_ptr + g->tasks.size(), 4, cudaMemcpyDeviceToHost);
        if (err != cudaSuccess) return cuda_fail(err);
        g->nedges = e;
      }
      *nedges = g->nedges;
    }
  }
  return SPX_OK;
}

int spx_graph_edges(spx_graph_t g, unsigned* row_ptr, unsigned* col, unsigned* indeg) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (!g->derived || g->state == kRunning) return SPX_ERR_STATE;
  long long ne = 0;
  int rc = spx_graph_sizes(g, nullptr, &ne, nullptr, nullptr);
  if (rc != SPX_OK) return rc;
  const size_t N = g->tasks.size();
  cudaError_t e = cudaSuccess;
  if (row_ptr) e = cudaMemcpy(row_ptr, g->dg.row_ptr, (N + 1) * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && col && ne > 0)
    e = cudaMemcpy(col, g->dg.col, (size_t)ne * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && indeg) e = cudaMemcpy(indeg, g->dg.indeg, N * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

int spx_graph_tickets(spx_graph_t g, unsigned* start, unsigned* end) {
  if (!g || (!start && !end)) return SPX_ERR_INVALID_ARG;
  if (g->state != kDone) return SPX_ERR_STATE;
  const size_t N = g->tasks.size();
  cudaError_t e = cudaSuccess;
  if (start) e = cudaMemcpy(start, g->dg.t_start, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && end) e = cudaMemcpy(end, g->dg.t_end, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && end)
    for (size_t i = 0; i < N; ++i) end[i] &= ~kTaskDone;  // the ticket alone
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

int spx_graph_tasks_done(spx_graph_t g, const unsigned* tasks, int count, int* done) {
  if (!g || count < 0 || (count && (!tasks || !done))) return SPX_ERR_INVALID_ARG;
  if (g->state != kRunning && g->state != kStreaming && g->state != kDone) return SPX_ERR_STATE;
  if (g->cfg.executor != SPX_EXEC_PERSISTENT || g->batch_of) return SPX_ERR_STATE;
  const size_t N = g->tasks.size();
  for (int i = 0; i < count; ++i)
    if (tasks[i] >= N) return SPX_ERR_BAD_HANDLE;
  if (!g->done_stream) {
    const cudaError_t e = cudaStreamCreateWithFlags(&g->done_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  g->done_buf.resize(N);
  // a snapshot of the end tickets, read by the copy engine while the kernel runs
  cudaError_t e = cudaMemcpyAsync(g->done_buf.data(), g->dg.t_end, N * 4, cudaMemcpyDeviceToHost,
                                  g->done_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->done_stream);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < count; ++i)
    done[i] = g->state == kDone || (g->done_buf[tasks[i]] & kTaskDone) ? 1 : 0;
  return SPX_OK;
}

int spx_graph_trace(spx_graph_t g, unsigned long long* rec) {
  if (!g || !rec) return SPX_ERR_INVALID_ARG;
  if (g->state != kDone || !g->cfg.trace) return SPX_ERR_STATE;
  cudaError_t e = cudaMemcpy(rec, g->dg.trace_rec, g->tasks.size() * 32, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SPX_OK : cuda_fail(e);
}

int spx_graph_task_ops(spx_graph_t g, int* ops, int* priorities) {
  if (!g || (!ops && !priorities)) return SPX_ERR_INVALID_ARG;
  for (size_t i = 0; i < g->tasks.size(); ++i) {
    if (ops) ops[i] = g->tasks[i].op;
    if (priorities) priorities[i] = g->tasks[i].prio;
  }
  return SPX_OK;
}

int spx_graph_stats(spx_graph_t g, long long* out, int n) {
  if (!g || !out || n < 0) return SPX_ERR_INVALID_ARG;
  if (g->batch_of && g->state == kDone) g = g->batch_of;  // the batched run
  if (g->state != kDone) return SPX_ERR_STATE;
  const RunState& r = *g->host_rs;
  long long v[9 + SPX_NUM_OPS] = {
      (long long)r.parts_done,  (long long)r.hiwater,      (long long)r.empty_pops,
      (long long)r.ctas,        (long long)r.busy_cycles,  (long long)r.total_cycles,
      (long long)g->dg.qcap,    (long long)(r.tail[0].v + r.tail[1].v), (long long)r.tail[2].v};
  for (int op = 0; op < SPX_NUM_OPS; ++op) v[9 + op] = (long long)r.op_cycles[op];
  for (int i = 0; i < n && i < 9 + SPX_NUM_OPS; ++i) out[i] = v[i];
  return SPX_OK;
}

int spx_graph_write_dot(spx_graph_t g, const char* path) {
  if (!g || !path) return SPX_ERR_INVALID_ARG;
  if (!g->derived || g->state == kRunning) return SPX_ERR_STATE;
  const size_t N = g->tasks.size();
  long long ne = 0;
  int rc = spx_graph_sizes(g, nullptr, &ne, nullptr, nullptr);
  if (rc != SPX_OK) return rc;
  std::vector<unsigned> rp(N + 1), col((size_t)std::max<long long>(ne, 1));
  rc = spx_graph_edges(g, rp.data(), col.data(), nullptr);
  if (rc != SPX_OK) return rc;
  FILE* f = std::fopen(path, "w");
  if (!f) return SPX_ERR_INVALID_ARG;
  static const char* names[SPX_NUM_OPS] = {"POTRF", "TRSM", "SYRK", "GEMM", "GEMM_NN",
                                           "TRSM_FWD", "GEMM_FWD", "TRSM_BWD", "GEMM_BWD",
                                           "NOP", "SPIN", "COPY", "AXPY", "TRMM", "TRTRI",
                                           "TRSM_INV", "NBODY_SELF", "NBODY_PAIR",
                                           "POTRF_PANEL", "SPLIT", "SPLIT_T"};
  std::fprintf(f, "digraph spx {\n");
  for (size_t u = 0; u < N; ++u)
    std::fprintf(f, "  t%zu [label=\"%s #%zu\"];\n", u, names[g->tasks[u].op], u);
  for (size_t u = 0; u < N; ++u)
    for (unsigned p = rp[u]; p < rp[u + 1]; ++p) std::fprintf(f, "  t%zu -> t%u;\n", u, col[p]);
  std::fprintf(f, "}\n");
  std::fclose(f);
  return SPX_OK;
}

int spx_graph_timing(spx_graph_t g, float* prep_ms, float* run_ms) {
  if (g && g->batch_of && g->state == kDone) g = g->batch_of;  // the batched run
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state != kDone || !g->tev[0]) return SPX_ERR_STATE;
  float a = 0.f, b = 0.f;
  cudaError_t e = cudaEventElapsedTime(&a, g->tev[0], g->tev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&b, g->tev[1], g->tev[2]);
  if (e != cudaSuccess) return cuda_fail(e);
  if (prep_ms) *prep_ms = a;
  if (run_ms) *run_ms = b;
  return SPX_OK;
}

int spx_graph_reset(spx_graph_t g) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state != kDone) return SPX_ERR_STATE;
  g->state = kFrozen;
  return SPX_OK;
}

int spx_graph_clear(spx_graph_t g) {
  if (!g) return SPX_ERR_INVALID_ARG;
  if (g->state == kRunning || g->state == kStreaming) return SPX_ERR_STATE;
  g->sg.clear();
  g->spred.clear();
  g->sout.clear();
  g->salias.clear();
  g->batch_of = nullptr;
  g->tiles.clear();
  g->tile_dtype.clear();
  g->maps.clear();
  g->map_info.clear();
  g->tc_mode = 0;
  g->key_to_handle.clear();
  g->hstate.clear();
  g->tasks.clear();
  g->rec_handle.clear();
  g->rec_seq.clear();
  g->rec_mode.clear();
  g->task_rec.assign(1, 0);
  g->cand_edges = 0;
  g->items[0] = g->items[1] = g->items[2] = 0;
  g->uploaded = false;
  g->derived = false;
  g->nedges = -1;
  g->state = kBuilding;
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  return SPX_OK;
}

int spx_batch_execute(spx_graph_t* gs, int ng, void* stream) {
  if (!gs || ng < 1) return SPX_ERR_INVALID_ARG;
  for (int i = 0; i < ng; ++i) {
    if (!gs[i]) return SPX_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (gs[j] == gs[i]) return SPX_ERR_INVALID_ARG;
    if (gs[i]->state == kRunning || gs[i]->state == kDone) return SPX_ERR_STATE;
    if (gs[i]->tasks.empty()) return SPX_ERR_STATE;
  }
  spx_graph* owner = gs[0];
  if (owner->batch && owner->batch->state == kRunning) return SPX_ERR_STATE;
  if (!owner->batch) {
    spx_graph_config_t cfg = owner->cfg;
    cfg.executor = SPX_EXEC_PERSISTENT;
    cfg.cuda_graph = 0;
    const int rc = spx_graph_create(&owner->batch, &cfg);
    if (rc != SPX_OK) return rc;
  }
  spx_graph* B = owner->batch;
  for (spx_graph* m : B->members)  // the previous batch's members run alone now
    if (m && m->batch_of == B) m->batch_of = nullptr;
  spx_graph_clear(B);
  B->members.assign(gs, gs + ng);
  B->task_group.clear();
  // Merge: every member's tiles (one handle per address), low-precision
  // matrices and tasks, members in order, tasks in insertion order.
  std::vector<unsigned> hmap;
  for (int i = 0; i < ng; ++i) {
    const spx_graph* m = gs[i];
    for (const auto& mi : m->map_info) {
      if (mi.kind == 2) continue;  // registered with its kind-1 twin
      const int rows = (int)(mi.bytes / ((size_t)mi.ld * mi.elem));
      const int rc =
          mi.kind == 1 ? spx_ozaki_register(B, (void*)mi.base, mi.cols_, mi.ld, nullptr)
                       : spx_lowp_register(B, (void*)mi.base, rows, mi.cols_, mi.ld, mi.dtype, nullptr);
      if (rc != SPX_OK) return rc;
    }
    hmap.assign(m->tiles.size(), 0);
    for (size_t h = 0; h < m->tiles.size(); ++h) {
      const TileDesc& t = m->tiles[h];
      const int rc = spx_tile_register(B, t.ptr, t.rows, t.cols, t.ld, m->tile_dtype[h], t.lowp,
                                       t.lowp ? t.lowp_ld : 0, &hmap[h]);
      if (rc != SPX_OK) return rc;
    }
    for (size_t u = 0; u < m->tasks.size(); ++u) {
      const TaskDesc& t = m->tasks[u];
      const uint32_t r0 = m->task_rec[u], r1 = m->task_rec[u + 1];
      unsigned hh[kMaxHandles];
      int mm[kMaxHandles];
      int nh = 0;
      if (kWantNh[t.op] < 0) {  // NOP / SPIN: the merged accesses
        for (uint32_t r = r0; r < r1; ++r, ++nh) {
          hh[nh] = hmap[m->rec_handle[r]];
          mm[nh] = m->rec_mode[r];
        }
      } else {                   // the op's operands in order, with their modes
        nh = kWantNh[t.op];
        for (int j = 0; j < nh; ++j) {
          hh[j] = hmap[t.h[j]];
          mm[j] = SPX_READ;
          for (uint32_t r = r0; r < r1; ++r)
            if (m->rec_handle[r] == t.h[j]) mm[j] = m->rec_mode[r];
        }
      }
      unsigned tid = 0;
      int rc = spx_task_insert(B, t.op, hh, mm, nh, t.prio, t.prec, &tid);
      if (rc == SPX_OK) rc = spx_task_set_arg(B, tid, t.arg);
      if (rc != SPX_OK) return rc;
      B->task_group.push_back((uint32_t)i);
    }
  }
  if (B->host_groups_cap < (size_t)ng) {
    if (B->host_groups) cudaFreeHost(B->host_groups);
    B->host_groups = nullptr;
    B->host_groups_cap = 0;
    const cudaError_t e =
        cudaHostAlloc((void**)&B->host_groups, ng * sizeof(GroupState), cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e);
    B->host_groups_cap = (size_t)ng;
  }
  const int rc = spx_graph_execute(B, stream);
  if (rc != SPX_OK) return rc;
  for (int i = 0; i < ng; ++i) {
    gs[i]->batch_of = B;
    gs[i]->batch_index = (uint32_t)i;
    gs[i]->state = kRunning;
  }
  return SPX_OK;
}

void spx_graph_destroy(spx_graph_t g) {
  if (!g) return;
  if (g->state == kStreaming) stream_close(g);  // the kernel drains what was published
  if (g->state == kRunning) spx_graph_wait(g, 0, nullptr);
  if (g->batch_of) {  // leave the merged graph's member list
    for (spx_graph*& m : g->batch_of->members)
      if (m == g) m = nullptr;
  }
  if (g->batch) {     // the merged graph this graph owns: detach its members
    if (g->batch->state == kRunning) spx_graph_wait(g->batch, 0, nullptr);
    for (spx_graph* m : g->batch->members)
      if (m && m != g && m->batch_of == g->batch) {
        if (m->state == kRunning) spx_graph_wait(m, 0, nullptr);
        m->batch_of = nullptr;
      }
    g->batch->members.clear();
    spx_graph_destroy(g->batch);
    g->batch = nullptr;
  }
  if (g->host_groups) cudaFreeHost(g->host_groups);
  if (g->s_up) cudaStreamSynchronize(g->s_up);
  if (g->last_stream) cudaStreamSynchronize(g->last_stream);
  if (g->dmem) cudaFree(g->dmem);
  if (g->pinned) cudaFreeHost(g->pinned);
  if (g->host_rs) cudaFreeHost(g->host_rs);
  if (g->s_up) cudaStreamDestroy(g->s_up);
  if (g->done_stream) cudaStreamDestroy(g->done_stream);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  for (int i = 0; i < 4; ++i) {
    if (g->xs[i]) cudaStreamDestroy(g->xs[i]);
    if (g->join_ev[i]) cudaEventDestroy(g->join_ev[i]);
  }
  if (g->fork_ev) cudaEventDestroy(g->fork_ev);
  for (cudaEvent_t ev : g->task_ev) cudaEventDestroy(ev);
  if (g->done_ev) cudaEventDestroy(g->done_ev);
  for (int i = 0; i < 3; ++i)
    if (g->tev[i]) cudaEventDestroy(g->tev[i]);
  delete g;
}

}  // extern "C"

int spx_graph_view(spx_graph_t g, spx::GraphView* v) {
  if (!g || !v) return SPX_ERR_INVALID_ARG;
  if (g->state == kRunning) return SPX_ERR_STATE;
  v->tasks = g->tasks.data();
  v->ntasks = g->tasks.size();
  v->tiles = g->tiles.data();
  v->ntiles = g->tiles.size();
  v->maps = g->maps.data();
  v->nmaps = g->maps.size();
  v->rec_handle = g->rec_handle.data();
  v->rec_seq = g->rec_seq.data();
  v->rec_mode = g->rec_mode.data();
  v->nrec = g->rec_handle.size();
  v->task_rec = g->task_rec.data();
  v->cand_edges = g->cand_edges;
  v->items = g->items[0] + g->items[1] + g->items[2];
  return SPX_OK;
}
