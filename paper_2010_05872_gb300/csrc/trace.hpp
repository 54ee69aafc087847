// Kernel timing trace: while enabled, every kernel launch of the library
// (or, after mgard_trace_select, every launch of one kind) is bracketed by
// CUDA events recorded on its own stream, tagged with the kernel kind, the
// level it worked on and its algorithmic bytes (each input read once, each
// output written once).  mgard_trace_read() aggregates them.  Launches are
// counted whether or not they are bracketed.
#pragma once

#include <cuda_runtime.h>

namespace mgb {

enum KernelKind : int {
  kKLoadVectorDec = 0,
  kKLoadVectorRec,
  kKSolveContig,
  kKSolveStrided,
  kKFinishDec,
  kKFinishRec,
  kKQuantize,
  kKDequantize,
  kKMinmax,
  kKSmallLevels,
  kKPredErr,
  kKIsoArea,
  kKGather,
  kKPack,
  kKUnpack,
  kKLorenzo,
  kKNumKinds
};

const char* kernel_kind_name(int kind);

class TraceScope {
 public:
  TraceScope(int kind, int level, double bytes, cudaStream_t s);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
  // Count `n` more kernel launches in this scope (one is counted already).
  void more_kernels(int n);

 private:
  int slot_ = -1;
  bool on_ = false;
  cudaStream_t s_ = nullptr;
};

}  // namespace mgb
