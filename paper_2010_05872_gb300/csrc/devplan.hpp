// Device-resident plans and the per-device context, shared by the entry
// points of api.cu and the batched form of batch.cu.
#pragma once

#include <array>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "mgard_gb.h"
#include "plan.hpp"

namespace mgb {

// Plan tables resident on one device in the element type of the transform.
struct DevPlan {
  HostPlan h;
  int dtype = MGARD_F32;
  int device = 0;
  void* dmem = nullptr;
  std::vector<LevelK<float>> lvf;   // [L+1], entry l = transition l -> l-1
  std::vector<LevelK<double>> lvd;
  const uint8_t* lev[3] = {nullptr, nullptr, nullptr};
  const uint8_t* lev01 = nullptr;   // per-row level (quantizer)
  std::vector<std::array<const int32_t*, 3>> pos;  // [L+1] level-l node positions per axis
  std::array<const double*, 3> xc{};               // finest coordinates per axis
  std::vector<size_t> offB, offF;   // workspace offsets of the level-l grids / load vectors
  size_t ws_bytes = 0;
  ~DevPlan() {
    if (dmem) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(device);
      cudaFree(dmem);
      cudaSetDevice(cur);
    }
  }
};

// Small per-device scratch for flags and reductions (allocated once).
// flags[1] gathers the bounded waits that gave up (every transform and the
// batched form write it), flags[2] the asynchronous quantizer's problems.
struct DevCtx {
  unsigned int* flags = nullptr;  // [4]
  double* partial = nullptr;      // [2 * kMinmaxBlocks] (adaptive decomposition)
  double* sums = nullptr;         // [2 * kMaxLevels] per-level sums of the adaptive decomposition
  double* h_sums = nullptr;       // pinned host mirror
  std::mutex mu;                  // serialises the adaptive decompositions
};

// Scratch of the calls that wait on a stream (value range, quantization,
// the packed stream's size, the iso-surface area, the status read) and of
// the asynchronous value range, one per (device, stream): such calls on
// different streams share no buffer and no lock, so one stream's wait (say
// behind a large host copy) holds up no other.  Created on the stream's
// first such call and kept for the life of the process.
struct StreamScratch {
  unsigned int* flag = nullptr;     // [1] the call's own flag word
  double* partial = nullptr;        // [2 * kMinmaxBlocks]
  double* result = nullptr;         // [2]
  unsigned int* h_flags = nullptr;  // pinned [4]
  double* h_result = nullptr;       // pinned [2]
  std::mutex mu;                    // serialises the waiting calls on this stream
};

// Look up (or build and upload) the plan of this shape/coords/dtype on the
// current device.  The returned plan lives until mgard_release_plans().
int get_plan(int ndim, const int64_t* dims, const double* const* coords, int dtype, DevPlan** out);

// The per-device flag/reduction context (created on first use).
DevCtx* get_ctx();

// The scratch of stream `s` on the current device (created on first use).
StreamScratch* get_scratch(cudaStream_t s);

template <typename T>
const std::vector<LevelK<T>>& levels(const DevPlan& p);

// Enqueue the decomposition (dec) or recomposition of `data` on `s` with the
// workspace `ws`; `status` receives wait timeouts.  No synchronization.
int run_transform(bool dec, const DevPlan& p, int stop_level, void* data, char* ws,
                  unsigned int* status, cudaStream_t s);

// Bin widths of every level for the absolute bound `tau` (host FP64, Eq.
// LinfTau), with the FP32 helpers of the quantizer's fast paths; tau_out
// (L + 1 values, may be NULL) receives the level tolerances.
int make_table(const DevPlan& p, int stop_level, double tau, LevelTable& tab, double* tau_out);
// The same from given level tolerances t[0..L] (entries from stop_level on
// must be positive and finite).
int make_table_levels(const DevPlan& p, int stop_level, const double* t, LevelTable& tab,
                      double* tau_out);
// The same for any hierarchy of L + 1 levels.
int make_level_table(int L, int stop_level, const double* t, LevelTable& tab, double* tau_out);

}  // namespace mgb
