// One instantiation of the executor kernels: the one-launch-per-task baseline kernel with tensor-core tile ops.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_task_tc() { return (const void*)task_kernel<1>; }

cudaError_t mega_launch_task_tc(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                               uint32_t task, uint32_t phase) {
  task_kernel<1><<<ctas, kThreads, smem, st>>>(g, task, phase);
  return cudaGetLastError();
}

}  // namespace spx
