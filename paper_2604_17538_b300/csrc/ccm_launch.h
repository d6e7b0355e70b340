// Kernel launches with programmatic dependent launch (PDL): a kernel launched
// this way may be scheduled while the previous kernel of its stream drains;
// it runs no further than its pdl_wait() (griddepcontrol.wait) until that
// kernel has completed and its memory is visible.  Every kernel launched
// through launch_k therefore calls pdl_wait() before it touches memory that
// an earlier kernel of the stream writes or reads.  Without pdl the launch is
// an ordinary one and pdl_wait() returns at once.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <utility>

namespace ccm {

// Kernels this library has launched in the process, counted on the host as
// they are issued (a captured CUDA graph's kernels count once, at capture).
extern std::atomic<long long> g_kernel_launches;
inline void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t stream, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e == cudaSuccess) count_launch();
  return e;
}

}  // namespace ccm
