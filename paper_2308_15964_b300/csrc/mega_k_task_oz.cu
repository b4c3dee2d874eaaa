// One instantiation of the executor kernels: the one-launch-per-task baseline kernel, one CTA per SM with the split-FP64 products.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_task_oz() { return (const void*)task_kernel<2>; }

cudaError_t mega_launch_task_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                               uint32_t task, uint32_t phase) {
  task_kernel<2><<<ctas, kThreads, smem, st>>>(g, task, phase);
  return cudaGetLastError();
}

}  // namespace spx
