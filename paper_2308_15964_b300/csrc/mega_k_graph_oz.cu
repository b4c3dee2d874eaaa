// One instantiation of the executor kernels: the persistent kernel, one CTA per SM with the split-FP64 products, for graph runs.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_graph_oz() { return (const void*)persistent_kernel<2, false>; }

cudaError_t mega_launch_graph_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g) {
  persistent_kernel<2, false><<<ctas, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
