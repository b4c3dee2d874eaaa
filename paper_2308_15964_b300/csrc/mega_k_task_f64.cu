// One instantiation of the executor kernels: the one-launch-per-task baseline kernel with FP64 tile ops.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_task_f64() { return (const void*)task_kernel<0>; }

cudaError_t mega_launch_task_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                               uint32_t task, uint32_t phase) {
  task_kernel<0><<<ctas, kThreads, smem, st>>>(g, task, phase);
  return cudaGetLastError();
}

}  // namespace spx
