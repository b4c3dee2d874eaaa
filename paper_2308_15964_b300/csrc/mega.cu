// Host side of the executors: occupancy, launch sizes and the launches of the
// persistent kernel (graph runs and the resident server) and of the
// one-launch-per-task baseline.  The kernels are in mega_kernels.cuh, each
// instantiation compiled in its own mega_k_*.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mega_launch.h"
#include "spx_internal.h"
#include "tile_f64.cuh"
#include "tile_tc.cuh"
#include "tile_oz.cuh"

namespace spx {
namespace {

// Kernel families: 0 FP64 only (two CTAs per SM), 1 tensor-core tile ops
// (two CTAs per SM, 256 TMEM columns each), 2 the split-FP64 products (one
// CTA per SM, all 512 TMEM columns, three 48 KB operand stages).
int g_max_ctas_per_sm[3] = {-1, -1, -1};
int g_api_ctas_per_sm[3] = {-1, -1, -1};  // what the occupancy calculator guarantees
int g_sms = -1;

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

constexpr size_t smem_bytes(int mode) {
  return mode == 0   ? sizeof(F64Smem)
         : mode == 1 ? cmax(sizeof(F64Smem), sizeof(TcBuf)) + 1024
                     : cmax(cmax(sizeof(F64Smem), sizeof(TcBuf)), sizeof(OzBuf)) + 1024;
}

// Every kernel prefers the largest shared-memory carveout.  (A kernel that
// allocates tensor memory is held to one CTA per SM by the occupancy rules
// of this GPU, whatever its shared memory; the FP64 kernel runs two.)
void configure(int mode) {
  const void* graph_fn =
      mode == 0 ? mega_fn_graph_f64() : mode == 1 ? mega_fn_graph_tc() : mega_fn_graph_oz();
  const void* fns[3] = {graph_fn,
                        mode == 0 ? mega_fn_server_f64() : mode == 1 ? mega_fn_server_tc() : mega_fn_server_oz(),
                        mode == 0 ? mega_fn_task_f64() : mode == 1 ? mega_fn_task_tc() : mega_fn_task_oz()};
  for (const void* f : fns) {
    if (!f) continue;
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(mode));
    cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, graph_fn, kThreads, smem_bytes(mode));
  g_api_ctas_per_sm[mode] = occ > 0 ? occ : 1;
  if (mode == 1 && occ == 1) {
    // The occupancy calculator answers 1 for any kernel that allocates tensor
    // memory.  Two CTAs of this one (256 of the 512 TMEM columns each) fit in
    // the SM's registers and shared memory, and the GPU runs them (ncu on the
    // stand-alone tensor-core kernel: two blocks per SM, one wave).  No CTA of
    // the persistent kernel waits for another to start, so a CTA that did not
    // fit would only start after the work, find nothing left and exit.
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaFuncGetAttributes(&fa, graph_fn);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const size_t per_cta = smem_bytes(mode) + fa.sharedSizeBytes + 1024;
    if (2 * per_cta <= (size_t)smem_sm && 2 * fa.numRegs * kThreads <= regs_sm) occ = 2;
  }
  if (mode == 2) occ = 1;  // all of the SM's TMEM and most of its shared memory
  g_max_ctas_per_sm[mode] = occ > 0 ? occ : 1;
}

}  // namespace

size_t persistent_smem_bytes() { return smem_bytes(0); }

int persistent_max_ctas(int* per_sm) {
  if (g_max_ctas_per_sm[0] < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    configure(0);
    configure(1);
    configure(2);
  }
  if (per_sm) *per_sm = g_max_ctas_per_sm[0];
  return g_sms * g_max_ctas_per_sm[0];
}

cudaError_t launch_persistent(const DevGraph& g, int num_ctas, int mode, cudaStream_t st) {
  persistent_max_ctas(nullptr);
  const int maxc = g_sms * g_max_ctas_per_sm[mode];
  int n = num_ctas > 0 ? num_ctas : maxc;
  if (n > maxc) n = maxc;  // every CTA resident: no CTA waits behind a spinning one
  return mode == 0   ? mega_launch_graph_f64(n, smem_bytes(0), st, g)
         : mode == 1 ? mega_launch_graph_tc(n, smem_bytes(1), st, g)
                     : mega_launch_graph_oz(n, smem_bytes(2), st, g);
}

cudaError_t launch_server(const DevGraph& g, int num_ctas, int mode, cudaStream_t st) {
  persistent_max_ctas(nullptr);
  // The server kernel exits when idle and is launched again by the next
  // submission: it keeps to the occupancy the calculator guarantees, so that
  // no CTA of an exited launch can start late beside the next one.
  const int maxc = g_sms * g_api_ctas_per_sm[mode];
  int n = num_ctas > 0 ? num_ctas : maxc;
  if (n > maxc) n = maxc;
  return mode == 0   ? mega_launch_server_f64(n, smem_bytes(0), st, g)
         : mode == 1 ? mega_launch_server_tc(n, smem_bytes(1), st, g)
                     : mega_launch_server_oz(n, smem_bytes(2), st, g);
}

__global__ void ring_init_kernel(uint32_t* s0, uint32_t* s1, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    s0[i] = i;
    s1[i] = i;
  }
}

cudaError_t launch_ring_init(const DevGraph& g, cudaStream_t st) {
  ring_init_kernel<<<256, 256, 0, st>>>(g.qseq[0], g.qseq[1], g.qcap);
  return cudaGetLastError();
}

cudaError_t launch_task(const DevGraph& g, uint32_t u, const TaskDesc& t,
                        const TileDesc* host_tiles, int mode, cudaStream_t st) {
  for (uint32_t ph = 0; ph < t.nphases; ++ph) {
    const uint32_t np =
        (t.flags & kFlagSerial)
            ? 1u
            : phase_parts(task_phase_units(t, host_tiles, ph));
    if (mode == 2) mega_launch_task_oz((int)np, smem_bytes(2), st, g, u, ph);
    else if (mode == 1) mega_launch_task_tc((int)np, smem_bytes(1), st, g, u, ph);
    else mega_launch_task_f64((int)np, smem_bytes(0), st, g, u, ph);
  }
  return cudaSuccess;
}

cudaError_t launch_per_task(const DevGraph& g, const TaskDesc* host_tasks,
                            const TileDesc* host_tiles, int mode, cudaStream_t st) {
  persistent_max_ctas(nullptr);
  for (uint32_t u = 0; u < g.ntasks; ++u) launch_task(g, u, host_tasks[u], host_tiles, mode, st);
  return cudaGetLastError();
}

}  // namespace spx
