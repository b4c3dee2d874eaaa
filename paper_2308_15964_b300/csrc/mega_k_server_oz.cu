// One instantiation of the executor kernels: the resident server kernel, one CTA per SM, with
// the split-FP64 products (and the tensor-core and FP64 tile ops).
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_server_oz() { return (const void*)persistent_kernel<2, true>; }

cudaError_t mega_launch_server_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g) {
  persistent_kernel<2, true><<<ctas, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
