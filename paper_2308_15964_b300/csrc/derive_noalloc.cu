// Allocation-free variant of the dependency derivation, for callers that
// cannot allocate device memory: code that runs where cudaMalloc is not
// allowed or not wanted, such as a host callback, an embedding runtime that
// owns all device memory through its own pool, or a process that must not
// touch the allocator once it has started serving.  The caller passes the
// access records and the output arrays; the derivation's scratch lives in a
// fixed array in this library's device memory (a file-scope __device__
// array), which every GPU that loads the library holds until the process
// exits.
//
// The array is shared by every call: two calls that overlap on the GPU
// (different streams, or different host threads) race on it and produce
// garbage.  Each call re-initialises every scratch word it reads, so
// consecutive calls on one stream are independent.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "derive_steps.cuh"
#include "spx.h"
#include "spx_internal.h"

namespace spx {
namespace {

constexpr uint32_t kNaMaxRec = SPX_NOALLOC_MAX_RECORDS;
constexpr uint32_t kNaMaxHandles = SPX_NOALLOC_MAX_HANDLES;

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
// Scratch layout (byte offsets): list offsets per handle, the concatenated
// per-handle lists (task, mode, first flag), record positions, group
// indices and group starts.
constexpr size_t kOffHptr = 0;
constexpr size_t kOffSTask = kOffHptr + na_align((kNaMaxHandles + 1) * 4ull);
constexpr size_t kOffRecPos = kOffSTask + na_align(kNaMaxRec * 4ull);
constexpr size_t kOffGid = kOffRecPos + na_align(kNaMaxRec * 4ull);
constexpr size_t kOffGpos = kOffGid + na_align(kNaMaxRec * 4ull);
constexpr size_t kOffSMode = kOffGpos + na_align((kNaMaxRec + 1) * 4ull);
constexpr size_t kOffSFirst = kOffSMode + na_align(kNaMaxRec);
constexpr size_t kScratchBytes = kOffSFirst + na_align(kNaMaxRec);  // about 5.3 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array per device, looked up once per device.
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Checks the caller's records before any scratch write depends on them:
// offsets start at 0, end at nrec, give 1..16 records per task; handles and
// modes in range; each handle's positions are exactly 0..count-1 and follow
// task order.  Sets *status to SPX_ERR_INVALID_ARG and returns false
// otherwise.  Uses hptr and gid as scratch.
__device__ bool validate(const DevGraph& g, uint32_t* sh, int* status) {
  __shared__ int bad;
  const uint32_t N = g.ntasks, H = g.ntiles, M = g.nrec;
  const int tid = threadIdx.x;
  if (tid == 0) bad = (g.task_rec[0] != 0 || g.task_rec[N] != M) ? 1 : 0;
  for (uint32_t i = tid; i <= H; i += kDeriveThreads) g.hptr[i] = 0;
  for (uint32_t p = tid; p < M; p += kDeriveThreads) g.gid[p] = 0;
  __syncthreads();
  for (uint32_t u = tid; u < N; u += kDeriveThreads) {
    const uint32_t r0 = g.task_rec[u], r1 = g.task_rec[u + 1];
    if (r1 <= r0 || r1 - r0 > (uint32_t)kMaxHandles || r1 > M) bad = 1;
  }
  for (uint32_t r = tid; r < M; r += kDeriveThreads) {
    if (g.rec_handle[r] >= H || g.rec_mode[r] > SPX_MAYBE_WRITE) bad = 1;
    else atomicAdd(&g.hptr[g.rec_handle[r]], 1u);
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) *status = SPX_ERR_INVALID_ARG;
    return false;
  }
  block_excl_scan(g.hptr, H + 1, sh);
  __syncthreads();
  // every (handle, position) slot taken exactly once
  for (uint32_t r = tid; r < M; r += kDeriveThreads) {
    const uint32_t h = g.rec_handle[r];
    const uint32_t seq = g.rec_seq[r];
    if (seq >= g.hptr[h + 1] - g.hptr[h]) bad = 1;
    else atomicAdd(&g.gid[g.hptr[h] + seq], 1u);
  }
  __syncthreads();
  for (uint32_t p = tid; p < M && !bad; p += kDeriveThreads)
    if (g.gid[p] != 1u) bad = 1;
  __syncthreads();
  if (!bad) {
    // positions follow task order on each handle: scatter task ids, compare
    for (uint32_t u = tid; u < N; u += kDeriveThreads)
      for (uint32_t r = g.task_rec[u]; r < g.task_rec[u + 1]; ++r)
        g.s_task[g.hptr[g.rec_handle[r]] + g.rec_seq[r]] = u;
    __syncthreads();
    for (uint32_t h = tid; h < H; h += kDeriveThreads)
      for (uint32_t p = g.hptr[h] + 1; p < g.hptr[h + 1]; ++p)
        if (g.s_task[p] <= g.s_task[p - 1]) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) *status = SPX_ERR_INVALID_ARG;
    return false;
  }
  return true;
}

__global__ void __launch_bounds__(kDeriveThreads, 1) derive_noalloc_kernel(DevGraph g, int* status) {
  __shared__ uint32_t sh[kDeriveThreads / 32 + 1];
  if (threadIdx.x == 0) *status = 0;
  __syncthreads();
  if (!validate(g, sh, status)) return;
  __syncthreads();
  if (!derive_dag(g, sh)) {
    if (threadIdx.x == 0) *status = SPX_ERR_INVALID_ARG;  // col_cap < edges; row_ptr[n] = edges
  }
}

}  // namespace
}  // namespace spx

extern "C" int spx_graph_derive_noalloc(const unsigned* dev_task_rec, const unsigned* dev_rec_handle,
                                        const unsigned* dev_rec_seq,
                                        const unsigned char* dev_rec_mode, int ntasks,
                                        int nhandles, long long nrec, unsigned* dev_row_ptr,
                                        unsigned* dev_col, long long col_cap, unsigned* dev_indeg,
                                        int* dev_status, void* stream) {
  using namespace spx;
  if (!dev_task_rec || !dev_rec_handle || !dev_rec_seq || !dev_rec_mode || !dev_row_ptr ||
      !dev_indeg || !dev_status || (!dev_col && col_cap > 0) || ntasks < 1 || nhandles < 1 ||
      nrec < ntasks || col_cap < 0)
    return SPX_ERR_INVALID_ARG;
  if (nrec > (long long)kNaMaxRec || nhandles > (int)kNaMaxHandles) return SPX_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPX_ERR_NO_DEVICE;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        (void)cudaGetLastError();
        return SPX_ERR_CUDA;
      }
    }
    base = g_noalloc_addr[dev];
  }
  unsigned char* S = (unsigned char*)base;
  DevGraph g{};
  g.ntasks = (uint32_t)ntasks;
  g.ntiles = (uint32_t)nhandles;
  g.nrec = (uint32_t)nrec;
  g.ecap = (uint32_t)(col_cap > 0xFFFFFFFFll ? 0xFFFFFFFFll : col_cap);
  g.task_rec = dev_task_rec;
  g.rec_handle = dev_rec_handle;
  g.rec_seq = dev_rec_seq;
  g.rec_mode = dev_rec_mode;
  g.hptr = (uint32_t*)(S + kOffHptr);
  g.s_task = (uint32_t*)(S + kOffSTask);
  g.rec_pos = (uint32_t*)(S + kOffRecPos);
  g.gid = (uint32_t*)(S + kOffGid);
  g.gpos = (uint32_t*)(S + kOffGpos);
  g.s_mode = (uint8_t*)(S + kOffSMode);
  g.s_first = (uint8_t*)(S + kOffSFirst);
  g.row_ptr = dev_row_ptr;
  g.col = dev_col;
  g.indeg = dev_indeg;
  derive_noalloc_kernel<<<1, kDeriveThreads, 0, (cudaStream_t)stream>>>(g, dev_status);
  return cudaGetLastError() == cudaSuccess ? SPX_OK : SPX_ERR_CUDA;
}
