// One instantiation of the executor kernels: the resident server kernel with FP64 tile ops.
// Each instantiation sits in its own file so that they compile in parallel.
#include "mega_kernels.cuh"
#include "mega_launch.h"

namespace spx {

const void* mega_fn_server_f64() { return (const void*)persistent_kernel<0, true>; }

cudaError_t mega_launch_server_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g) {
  persistent_kernel<0, true><<<ctas, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace spx
