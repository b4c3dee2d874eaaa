// Continuous-batching server: one resident persistent kernel runs the tasks
// of every live request graph, and new graphs are admitted while it runs.
//
// A request is an ordinary spx graph that was built (tasks inserted) but not
// executed.  spx_server_submit copies its arrays into ranges of the server's
// device pools (task ids and tile handles inside the copy are rebased to the
// pool), then publishes a submission entry in a host-mapped ring.  An idle
// CTA of the resident kernel claims it, derives the request's DAG on the
// device and pushes its ready tasks into the shared work queues, where they
// interleave with the tasks of every other live request.  When a request's
// last task finishes, the kernel writes its status to host-mapped memory;
// spx_server_poll reads it and frees the request's pool ranges.
//
// The resident kernel exits after idle_ns with nothing live (and is
// relaunched by the next submit or poll), or on spx_server_stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "graph_access.h"
#include "spx.h"
#include "spx_internal.h"

using namespace spx;

namespace {

// First-fit allocator of index ranges in a pool.
class RangeAlloc {
 public:
  void reset(size_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t n, size_t* at) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *at = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t at, size_t n) {
    auto it = free_.emplace(at, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Live {
  uint32_t slot;
  size_t tb, nt, hb, nh, rb, nr, eb, ne, mb, nm;
  unsigned long long items;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

int cuda_err(cudaError_t e) {
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SPX_ERR_OOM : SPX_ERR_CUDA;
}

}  // namespace

struct spx_server {
  spx_server_config_t cfg{};
  void* dmem = nullptr;
  HostCtl* ctl = nullptr;       // host view
  HostCtl* ctl_dev = nullptr;   // device view of the same memory
  DevGraph dg{};
  cudaStream_t run_stream = nullptr, copy_stream = nullptr;
  cudaEvent_t run_done = nullptr;
  bool launched = false;
  RangeAlloc tasks, tiles, recs, edges, maps;
  std::vector<uint32_t> free_slots;
  std::unordered_map<unsigned long long, Live> live;
  unsigned long long next_seq = 1, live_items = 0;
  uint32_t sub_tail = 0;
  std::vector<char> stage;      // host staging of one submission
  void* pinned = nullptr;
  size_t pinned_cap = 0;
};

namespace {

int ensure_running(spx_server* s) {
  if (s->launched) {
    const cudaError_t q = cudaEventQuery(s->run_done);
    if (q == cudaErrorNotReady) return SPX_OK;
    if (q != cudaSuccess) return cuda_err(q);
    // exited: error, or idle exit
    uint32_t status = 0;
    cudaError_t e = cudaMemcpy(&status, &s->dg.rs->status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    if (status) return (int)(int32_t)status;
    s->launched = false;
  }
  cudaError_t e = launch_server(s->dg, s->cfg.num_ctas, s->cfg.tensor_cores, s->run_stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->run_done, s->run_stream);
  if (e != cudaSuccess) return cuda_err(e);
  s->launched = true;
  return SPX_OK;
}

}  // namespace

extern "C" {

void spx_server_config_default(spx_server_config_t* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->max_tasks = 1 << 21;
  c->max_tiles = 1 << 20;
  c->max_records = 1 << 23;
  c->max_edges = 1 << 23;
  c->max_maps = 256;
  c->queue_capacity = 1 << 22;
  c->watchdog_ns = 10000000000ull;
  c->idle_ns = 2000000000ull;
}

int spx_server_create(spx_server_t* out, const spx_server_config_t* cfg) {
  if (!out) return SPX_ERR_INVALID_ARG;
  *out = nullptr;
  spx_server* s = new (std::nothrow) spx_server();
  if (!s) return SPX_ERR_OOM;
  spx_server_config_default(&s->cfg);
  if (cfg) {
    spx_server_config_t c = *cfg;
    spx_server_config_t d;
    spx_server_config_default(&d);
    if (!c.max_tasks) c.max_tasks = d.max_tasks;
    if (!c.max_tiles) c.max_tiles = d.max_tiles;
    if (!c.max_records) c.max_records = d.max_records;
    if (!c.max_edges) c.max_edges = d.max_edges;
    if (!c.max_maps) c.max_maps = d.max_maps;
    if (!c.queue_capacity) c.queue_capacity = d.queue_capacity;
    if (!c.watchdog_ns) c.watchdog_ns = d.watchdog_ns;
    if (!c.idle_ns) c.idle_ns = d.idle_ns;
    s->cfg = c;
  }
  const spx_server_config_t& c = s->cfg;
  if (c.max_tasks < 2 || c.max_tasks > (long long)kMaxTasks || c.max_tiles < 2 ||
      c.max_records < 2 || c.max_edges < 1 || c.queue_capacity < 64 ||
      c.queue_capacity > 0x40000000ll || c.num_ctas < 0 || c.tensor_cores < 0 ||
      c.tensor_cores > 2) {
    delete s;
    return SPX_ERR_INVALID_ARG;
  }
  const size_t T = c.max_tasks, H = c.max_tiles, M = c.max_records, E = c.max_edges,
               NM = c.max_maps, Q = c.queue_capacity;
  // one device arena
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = al(o + std::max<size_t>(bytes, 1)); return at; };
  const size_t o_tasks = take(T * sizeof(TaskDesc)), o_tiles = take(H * sizeof(TileDesc)),
               o_maps = take(NM * sizeof(CUtensorMap)), o_rh = take(M * 4), o_rs = take(M * 4),
               o_rm = take(M), o_trec = take(T * 4), o_q0 = take(Q * 4), o_q1 = take(Q * 4),
               o_s0 = take(Q * 4), o_s1 = take(Q * 4), o_tst = take(T * 4), o_run = take(sizeof(RunState)),
               o_tend = take(T * 4), o_phase = take(T * 4), o_hptr = take(H * 4),
               o_stask = take(M * 4), o_smode = take(M), o_sfirst = take(M), o_rpos = take(M * 4),
               o_gid = take(M * 4), o_gpos = take(M * 4), o_rowp = take(T * 4), o_col = take(E * 4),
               o_indeg = take(T * 4), o_indw = take(T * 4), o_rem = take(T * 4), o_treq = take(T * 4),
               o_reqs = take(kMaxRequests * sizeof(ReqDev)), o_locks = take(H * 4);
  int rc = SPX_OK;
  cudaError_t e = cudaMalloc(&s->dmem, o);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->ctl, sizeof(HostCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->ctl_dev, s->ctl, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->run_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->run_done, cudaEventDisableTiming);
  if (e != cudaSuccess) rc = cuda_err(e);
  if (rc != SPX_OK) {
    spx_server_destroy(s);
    return rc;
  }
  std::memset((void*)s->ctl, 0, sizeof(HostCtl));
  char* D = (char*)s->dmem;
  DevGraph& d = s->dg;
  d = DevGraph{};
  d.qcap = (uint32_t)Q;
  d.watchdog_ns = c.watchdog_ns;
  d.idle_ns = c.idle_ns;
  d.server = 1;
  d.tasks = (const TaskDesc*)(D + o_tasks);
  d.tiles = (const TileDesc*)(D + o_tiles);
  d.maps = (const CUtensorMap*)(D + o_maps);
  d.rec_handle = (const uint32_t*)(D + o_rh);
  d.rec_seq = (const uint32_t*)(D + o_rs);
  d.rec_mode = (const uint8_t*)(D + o_rm);
  d.task_rec = (const uint32_t*)(D + o_trec);
  d.queue[0] = (uint32_t*)(D + o_q0);
  d.queue[1] = (uint32_t*)(D + o_q1);
  d.qseq[0] = (uint32_t*)(D + o_s0);
  d.qseq[1] = (uint32_t*)(D + o_s1);
  d.t_start = (uint32_t*)(D + o_tst);
  d.rs = (RunState*)(D + o_run);
  d.t_end = (uint32_t*)(D + o_tend);
  d.phase = (uint32_t*)(D + o_phase);
  d.hptr = (uint32_t*)(D + o_hptr);
  d.s_task = (uint32_t*)(D + o_stask);
  d.s_mode = (uint8_t*)(D + o_smode);
  d.s_first = (uint8_t*)(D + o_sfirst);
  d.rec_pos = (uint32_t*)(D + o_rpos);
  d.gid = (uint32_t*)(D + o_gid);
  d.gpos = (uint32_t*)(D + o_gpos);
  d.row_ptr = (uint32_t*)(D + o_rowp);
  d.col = (uint32_t*)(D + o_col);
  d.indeg = (uint32_t*)(D + o_indeg);
  d.indeg_w = (uint32_t*)(D + o_indw);
  d.remaining = (uint32_t*)(D + o_rem);
  d.task_req = (uint32_t*)(D + o_treq);
  d.reqs = (ReqDev*)(D + o_reqs);
  d.locks = (uint32_t*)(D + o_locks);
  d.ctl = s->ctl_dev;
  d.ntasks = (uint32_t)T;
  d.ntiles = (uint32_t)H;
  d.nrec = (uint32_t)M;
  d.ecap = (uint32_t)E;
  e = cudaMemsetAsync(d.rs, 0, sizeof(RunState), s->run_stream);
  if (e == cudaSuccess) e = launch_ring_init(d, s->run_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->run_stream);
  if (e != cudaSuccess) {
    rc = cuda_err(e);
    spx_server_destroy(s);
    return rc;
  }
  s->tasks.reset(T);
  s->tiles.reset(H);
  s->recs.reset(M);
  s->edges.reset(E);
  s->maps.reset(NM);
  for (int i = kMaxRequests - 1; i >= 0; --i) s->free_slots.push_back((uint32_t)i);
  *out = s;
  return SPX_OK;
}

int spx_server_submit(spx_server_t s, spx_graph_t g, unsigned long long* out_request) {
  if (!s || !g || !out_request) return SPX_ERR_INVALID_ARG;
  GraphView v;
  int rc = spx_graph_view(g, &v);
  if (rc != SPX_OK) return rc;
  if (v.ntasks == 0) return SPX_ERR_STATE;
  for (size_t i = 0; i < v.ntasks; ++i) {
    if (v.tasks[i].flags & kFlagComm) return SPX_ERR_INVALID_ARG;  // no commutative writes
    if (v.tasks[i].prec != SPX_F64 && !s->cfg.tensor_cores) return SPX_ERR_INVALID_ARG;
    // the split-FP64 products need the one-CTA-per-SM instance (tensor_cores = 2)
    if (v.tasks[i].prec == SPX_F64_OZAKI && s->cfg.tensor_cores != 2) return SPX_ERR_INVALID_ARG;
  }
  const unsigned long long items = v.items;
  if (s->free_slots.empty() || s->live_items + items > (unsigned long long)s->cfg.queue_capacity)
    return SPX_ERR_OOM;
  if (v.cand_edges > 0xFFFFFFFFull) return SPX_ERR_INVALID_ARG;  // 32-bit edge offsets
  Live L{};
  L.nt = v.ntasks + 1;
  L.nh = v.ntiles + 1;
  L.nr = v.nrec + 1;
  L.ne = std::max<size_t>(v.cand_edges, 1);
  L.nm = v.nmaps;
  bool ok = s->tasks.alloc(L.nt, &L.tb);
  if (ok && !(ok = s->tiles.alloc(L.nh, &L.hb))) s->tasks.release(L.tb, L.nt);
  if (ok && !(ok = s->recs.alloc(L.nr, &L.rb))) {
    s->tasks.release(L.tb, L.nt);
    s->tiles.release(L.hb, L.nh);
  }
  if (ok && !(ok = s->edges.alloc(L.ne, &L.eb))) {
    s->tasks.release(L.tb, L.nt);
    s->tiles.release(L.hb, L.nh);
    s->recs.release(L.rb, L.nr);
  }
  if (ok && L.nm && !(ok = s->maps.alloc(L.nm, &L.mb))) {
    s->tasks.release(L.tb, L.nt);
    s->tiles.release(L.hb, L.nh);
    s->recs.release(L.rb, L.nr);
    s->edges.release(L.eb, L.ne);
  }
  if (!ok) return SPX_ERR_OOM;
  L.slot = s->free_slots.back();
  L.items = items;
  // stage the rebased copy in pinned memory
  const size_t b_tasks = v.ntasks * sizeof(TaskDesc), b_tiles = v.ntiles * sizeof(TileDesc),
               b_maps = v.nmaps * sizeof(CUtensorMap), b_rec = v.nrec * 4, b_mode = v.nrec,
               b_trec = (v.ntasks + 1) * 4;
  const size_t need = al(b_tasks) + al(b_tiles) + al(b_maps) + 2 * al(b_rec) + al(b_mode) + al(b_trec);
  if (need > s->pinned_cap) {
    if (s->pinned) cudaFreeHost(s->pinned);
    s->pinned = nullptr;
    s->pinned_cap = 0;
    cudaError_t e = cudaHostAlloc(&s->pinned, need * 2, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_err(e);
    s->pinned_cap = need * 2;
  }
  char* P = (char*)s->pinned;
  size_t off = 0;
  TaskDesc* pt = (TaskDesc*)(P + off);
  off += al(b_tasks);
  for (size_t i = 0; i < v.ntasks; ++i) {
    pt[i] = v.tasks[i];
    // the server takes a commutative task's locks at its single part
    if (pt[i].flags & kFlagComm) {
      pt[i].flags |= kFlagSerial;
      pt[i].nphases = 1;
      pt[i].nparts = 1;
    }
    for (int k = 0; k < 3; ++k) pt[i].h[k] += (uint32_t)L.hb;
  }
  TileDesc* ptl = (TileDesc*)(P + off);
  off += al(b_tiles);
  for (size_t i = 0; i < v.ntiles; ++i) {
    ptl[i] = v.tiles[i];
    if (ptl[i].lmap >= 0) ptl[i].lmap += (int32_t)L.mb;
  }
  char* pm = P + off;
  off += al(b_maps);
  if (b_maps) std::memcpy(pm, v.maps, b_maps);
  char* prh = P + off;
  off += al(b_rec);
  std::memcpy(prh, v.rec_handle, b_rec);
  char* prs = P + off;
  off += al(b_rec);
  std::memcpy(prs, v.rec_seq, b_rec);
  char* prm = P + off;
  off += al(b_mode);
  std::memcpy(prm, v.rec_mode, b_mode);
  char* ptr_ = P + off;
  std::memcpy(ptr_, v.task_rec, b_trec);
  const DevGraph& d = s->dg;
  cudaStream_t cs = s->copy_stream;
  cudaError_t e = cudaMemcpyAsync((void*)(d.tasks + L.tb), pt, b_tasks, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.tiles + L.hb), ptl, b_tiles, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && b_maps) e = cudaMemcpyAsync((void*)(d.maps + L.mb), pm, b_maps, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.rec_handle + L.rb), prh, b_rec, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.rec_seq + L.rb), prs, b_rec, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.rec_mode + L.rb), prm, b_mode, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.task_rec + L.tb), ptr_, b_trec, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_err(e);
  s->free_slots.pop_back();
  const unsigned long long seq = s->next_seq++;
  s->live[seq] = L;
  s->live_items += items;
  SubEntry& se = s->ctl->ring[s->sub_tail % kSubRing];
  SubEntry ent{};
  ent.seq = (uint32_t)seq;
  ent.slot = L.slot;
  ent.tb = (uint32_t)L.tb;
  ent.ntasks = (uint32_t)v.ntasks;
  ent.hb = (uint32_t)L.hb;
  ent.ntiles = (uint32_t)v.ntiles;
  ent.rb = (uint32_t)L.rb;
  ent.nrec = (uint32_t)v.nrec;
  ent.eb = (uint32_t)L.eb;
  ent.ecap = (uint32_t)L.ne;
  std::memcpy((void*)&se, &ent, sizeof(SubEntry));
  std::atomic_thread_fence(std::memory_order_seq_cst);
  s->sub_tail += 1;
  s->ctl->sub_tail = s->sub_tail;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  rc = ensure_running(s);
  if (rc != SPX_OK) return rc;
  *out_request = seq;
  return SPX_OK;
}

int spx_server_poll(spx_server_t s, unsigned long long request, int* status, int* info) {
  if (!s) return SPX_ERR_INVALID_ARG;
  auto it = s->live.find(request);
  if (it == s->live.end()) return SPX_ERR_BAD_HANDLE;
  const Live& L = it->second;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (s->ctl->done_seq[L.slot] != (uint32_t)request) {
    const int rc = ensure_running(s);  // relaunch after an idle exit
    return rc != SPX_OK ? rc : 0;
  }
  if (status) *status = s->ctl->done_status[L.slot];
  if (info) *info = s->ctl->done_info[L.slot];
  s->tasks.release(L.tb, L.nt);
  s->tiles.release(L.hb, L.nh);
  s->recs.release(L.rb, L.nr);
  s->edges.release(L.eb, L.ne);
  if (L.nm) s->maps.release(L.mb, L.nm);
  s->free_slots.push_back(L.slot);
  s->live_items -= L.items;
  s->live.erase(it);
  return 1;
}

int spx_server_stop(spx_server_t s) {
  if (!s) return SPX_ERR_INVALID_ARG;
  s->ctl->shutdown = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  int rc = SPX_OK;
  if (s->launched) {
    cudaError_t e = cudaStreamSynchronize(s->run_stream);
    if (e != cudaSuccess) return cuda_err(e);
    uint32_t status = 0;
    e = cudaMemcpy(&status, &s->dg.rs->status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    rc = (int)(int32_t)status;
    s->launched = false;
  }
  s->ctl->shutdown = 0;
  return rc;
}

int spx_server_stats(spx_server_t s, long long* out, int n) {
  if (!s || !out || n < 0) return SPX_ERR_INVALID_ARG;
  if (s->launched && cudaEventQuery(s->run_done) == cudaErrorNotReady) return SPX_ERR_STATE;
  RunState r;
  cudaError_t e = cudaMemcpy(&r, s->dg.rs, sizeof(RunState), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(e);
  const long long v[6] = {(long long)r.parts_done, (long long)r.done.v, (long long)r.sub_head.v,
                          (long long)r.live.v, (long long)r.busy_cycles, (long long)r.total_cycles};
  for (int i = 0; i < n && i < 6; ++i) out[i] = v[i];
  return SPX_OK;
}

void spx_server_destroy(spx_server_t s) {
  if (!s) return;
  if (s->launched) spx_server_stop(s);
  if (s->dmem) cudaFree(s->dmem);
  if (s->ctl) cudaFreeHost((void*)s->ctl);
  if (s->pinned) cudaFreeHost(s->pinned);
  if (s->run_done) cudaEventDestroy(s->run_done);
  if (s->run_stream) cudaStreamDestroy(s->run_stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  delete s;
}

}  // extern "C"
