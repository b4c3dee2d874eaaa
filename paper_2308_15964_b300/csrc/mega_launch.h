// Launchers of the executor kernel instantiations (mega_k_*.cu): the kernel
// pointer (for attributes and occupancy) and a launch of ctas x kThreads
// threads with smem bytes of dynamic shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_internal.h"

namespace spx {

const void* mega_fn_graph_f64();
const void* mega_fn_graph_tc();
const void* mega_fn_server_f64();
const void* mega_fn_server_tc();
const void* mega_fn_task_f64();
const void* mega_fn_task_tc();
const void* mega_fn_graph_oz();
const void* mega_fn_task_oz();
const void* mega_fn_server_oz();

cudaError_t mega_launch_graph_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);
cudaError_t mega_launch_graph_tc(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);
cudaError_t mega_launch_server_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);
cudaError_t mega_launch_server_tc(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);
cudaError_t mega_launch_task_f64(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                                 uint32_t task, uint32_t phase);
cudaError_t mega_launch_task_tc(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                                uint32_t task, uint32_t phase);
cudaError_t mega_launch_graph_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);
cudaError_t mega_launch_task_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g,
                                uint32_t task, uint32_t phase);
cudaError_t mega_launch_server_oz(int ctas, size_t smem, cudaStream_t st, const DevGraph& g);

}  // namespace spx
