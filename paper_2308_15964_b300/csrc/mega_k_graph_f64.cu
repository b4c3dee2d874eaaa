// One instantiation of the executor kernels: the persistent kernel with FP64 tile ops, for graph runs.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_graph_f64() { return (const void*)persistent_kernel<0, false>; }

cudaError_t mega_launch_graph_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g) {
  persistent_kernel<0, false><<<ctas, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
