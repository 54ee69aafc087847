// Programmatic dependent launch: the kernels of the transform, quantizer and
// range passes are launched so that the next kernel of a stream may be
// scheduled while its predecessor drains (its last CTAs run), instead of
// after the predecessor has completed.  Each such kernel calls
// grid_dep_wait() before its first global memory access: that waits for the
// full completion (and memory flush) of the preceding kernel, so every
// read-after-write and write-after-read order of the stream still holds,
// and since every kernel waits, the order is transitive along the stream.
// grid_dep_launch() lets the successor be scheduled once every CTA of this
// grid has started.  Both are no-ops in a kernel launched without the
// attribute (a CUDA graph node, a plain <<<>>> launch).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

namespace mgb {

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Both at the top of a kernel, before any global memory access.
__device__ __forceinline__ void grid_dep_enter() {
  grid_dep_wait();
  grid_dep_launch();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raise (never lower) the dynamic shared memory `kernel` may be launched
// with on the current device.  The limit belongs to the kernel, not to a
// launch: a per-launch set would let a call on another host thread lower it
// between this thread's set and its launch, which would then be refused.  A
// limit that only grows stays valid for every launch that raised it to its
// own need.
inline cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& g = granted[std::make_pair(device, kernel)];
  if (bytes <= g) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) g = bytes;
  return e;
}

template <typename... KArgs>
cudaError_t allow_dynamic_smem(void (*kernel)(KArgs...), size_t bytes) {
  return allow_dynamic_smem(reinterpret_cast<const void*>(kernel), bytes);
}

}  // namespace mgb
