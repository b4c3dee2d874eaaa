// One instantiation of the executor kernels: the persistent kernel with tensor-core tile ops, for graph runs.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_graph_tc() { return (const void*)persistent_kernel<1, false>; }

cudaError_t mega_launch_graph_tc(int ctas, size_t smem, cudaStream_t st, const DevGraph& g) {
  persistent_kernel<1, false><<<ctas, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
