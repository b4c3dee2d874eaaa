// Dependency derivation on the device: access records -> successor CSR and
// in-degree counters in HBM.
//
// Model (Specx paper, section "Internal implementation"): each address used
// as a dependency has a data handle holding the ordered list of the tasks that
// use it; a finished task releases the next entry (or, for commutative
// accesses, every commutative entry at the same point) of each list.  The
// explicit DAG equivalent: on each handle's list, consecutive READs form one
// group, consecutive COMMUTATIVE_WRITEs form one group, every WRITE is a group
// of its own, and every member of a group depends on every member of the
// group before it.  Edges are de-duplicated across handles.
//
// Steps (one CTA of 1024 threads; block barriers between steps):
//   1. histogram of accesses per handle, exclusive scan -> list offsets;
//   2. scatter each access to its slot (offset + position on the list, a
//      position the host assigned in O(1) at insertion) -> per-handle lists
//      in insertion order;
//   3. group starts (first entry of a list, a WRITE, or a mode change),
//      scan -> group index of every entry and first entry of every group;
//   4. per task: k-way merge of the next-group ranges of its k accesses
//      (each range is sorted by task id) -> unique successors ascending;
//      counted first, scanned into row_ptr, then written with in-degree
//      atomics;
//   5. execution state: remaining predecessors, remaining parts, and the
//      initial ready tasks (in-degree 0) written to the two priority queues.
#include <cuda_runtime.h>
#include <stdint.h>

#include "derive_steps.cuh"
#include "spx_internal.h"

namespace spx {
namespace {

// Execution state and initial ready queues (step 5): one entry per ready
// task, (task << kPartBits) | (parts - 1).  Uses ucount as
// scratch.  Every thread of the CTA must call it.
__device__ void init_run(const DevGraph& g, uint32_t* sh) {
  const uint32_t N = g.ntasks;
  const int tid = threadIdx.x;
  for (uint32_t u = tid; u < N; u += kDeriveThreads) {
    g.indeg_w[u] = g.indeg[u];
    g.remaining[u] = g.tasks[u].nparts;
  }
  for (int q = 0; q < kQueues; ++q) {
    __syncthreads();
    for (uint32_t u = tid; u < N; u += kDeriveThreads) {
      const TaskDesc& t = g.tasks[u];
      const bool in_q = g.indeg[u] == 0 && graph_queue(t.prio) == (uint32_t)q;
      g.ucount[u] = in_q ? 1u : 0u;
    }
    __syncthreads();
    const uint32_t total = block_excl_scan(g.ucount, N, sh);
    if (total > g.qcap) {
      if (tid == 0) {
        g.rs->status = (uint32_t)SPX_ERR_QUEUE_FULL;
        g.rs->abort = 1;
      }
      return;
    }
    for (uint32_t u = tid; u < N; u += kDeriveThreads) {
      const TaskDesc& t = g.tasks[u];
      const bool in_q = g.indeg[u] == 0 && graph_queue(t.prio) == (uint32_t)q;
      if (in_q) g.queue[q][g.ucount[u]] = (u << kPartBits) | (t.nparts - 1);
    }
    if (tid == 0) {
      g.rs->tail[q].v = total;
      if (total > g.rs->hiwater) g.rs->hiwater = total;
    }
  }
}

__global__ void __launch_bounds__(kDeriveThreads, 1) derive_kernel(DevGraph g) {
  __shared__ uint32_t sh[kDeriveThreads / 32 + 1];
  if (!derive_dag(g, sh)) {  // cannot happen: ecap counts every candidate edge
    if (threadIdx.x == 0) {
      g.rs->status = (uint32_t)SPX_ERR_QUEUE_FULL;
      g.rs->abort = 1;
    }
    return;
  }

  // 5. execution state
  init_run(g, sh);
}

__global__ void __launch_bounds__(kDeriveThreads, 1) init_kernel(DevGraph g) {
  __shared__ uint32_t sh[kDeriveThreads / 32 + 1];
  init_run(g, sh);
}

}  // namespace

cudaError_t launch_derive(const DevGraph& g, cudaStream_t st) {
  derive_kernel<<<1, kDeriveThreads, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_init(const DevGraph& g, cudaStream_t st) {
  init_kernel<<<1, kDeriveThreads, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
