// Kernel timing trace (see trace.hpp) and its C entry points.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mgard_gb.h"
#include "trace.hpp"

namespace mgb {
namespace {

struct Rec {
  int kind;
  int level;
  double bytes;
  cudaEvent_t a;
  cudaEvent_t b;
};

std::atomic<bool> g_on{false};
std::atomic<int> g_sel_kind{-1};  // bracket only this kind (-1: every kind)
std::atomic<int> g_sel_level{0};
std::atomic<bool> g_sel_any_level{true};
std::atomic<int64_t> g_kernels{0};
std::mutex g_tmu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void recycle_all() {
  for (Rec& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace

const char* kernel_kind_name(int kind) {
  static const char* names[kKNumKinds] = {
      "load_vector_kernel<dec>", "load_vector_kernel<rec>", "solve_contig_kernel",
      "solve_strided_kernel",    "finish_kernel<dec>",      "finish_kernel<rec>",
      "quantize_kernel",         "dequantize_kernel",       "minmax_partial_kernel",
      "small_levels_kernel",     "prediction_errors_kernel", "iso_area_kernel",
      "gather_level_kernel",     "pack_labels_kernel",      "unpack_labels_kernel",
      "lorenzo_kernel"};
  return (kind >= 0 && kind < kKNumKinds) ? names[kind] : "unknown";
}

TraceScope::TraceScope(int kind, int level, double bytes, cudaStream_t s) : s_(s) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  on_ = true;
  g_kernels.fetch_add(1, std::memory_order_relaxed);
  const int sk = g_sel_kind.load(std::memory_order_relaxed);
  if (sk >= 0 && (kind != sk || (!g_sel_any_level.load(std::memory_order_relaxed) &&
                                 level != g_sel_level.load(std::memory_order_relaxed))))
    return;
  std::lock_guard<std::mutex> lk(g_tmu);
  Rec r{kind, level, bytes, take_event(), take_event()};
  if (r.a == nullptr || r.b == nullptr) return;
  cudaEventRecord(r.a, s);
  slot_ = static_cast<int>(g_recs.size());
  g_recs.push_back(r);
}

void TraceScope::more_kernels(int n) {
  if (on_) g_kernels.fetch_add(n, std::memory_order_relaxed);
}

TraceScope::~TraceScope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  if (slot_ < static_cast<int>(g_recs.size())) cudaEventRecord(g_recs[slot_].b, s_);
}

}  // namespace mgb

using namespace mgb;

extern "C" {

int mgard_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (on) {
    for (Rec& r : g_recs) {
      cudaEventSynchronize(r.b);
    }
    recycle_all();
    g_kernels.store(0);
  }
  g_on.store(on != 0);
  return MGARD_OK;
}

int mgard_trace_select(int kind, int level, int any_level) {
  if (kind >= kKNumKinds) return MGARD_ERR_ARG;
  g_sel_level.store(level);
  g_sel_any_level.store(any_level != 0);
  g_sel_kind.store(kind < 0 ? -1 : kind);
  return MGARD_OK;
}

int mgard_trace_read(int max_rows, int* kind, int* level, int64_t* launches, double* total_ms,
                     double* bytes, int* rows_out) {
  if (rows_out == nullptr) return MGARD_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_tmu);
  std::map<std::pair<int, int>, std::tuple<int64_t, double, double>> agg;
  for (Rec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return MGARD_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return MGARD_ERR_CUDA;
    auto& t = agg[{r.kind, r.level}];
    std::get<0>(t) += 1;
    std::get<1>(t) += ms;
    std::get<2>(t) += r.bytes;
  }
  int n = 0;
  for (auto& kv : agg) {
    if (n < max_rows && kind && level && launches && total_ms && bytes) {
      kind[n] = kv.first.first;
      level[n] = kv.first.second;
      launches[n] = std::get<0>(kv.second);
      total_ms[n] = std::get<1>(kv.second);
      bytes[n] = std::get<2>(kv.second);
    }
    ++n;
  }
  *rows_out = n;
  return MGARD_OK;
}

const char* mgard_trace_kernel_name(int kind) { return kernel_kind_name(kind); }

int64_t mgard_trace_kernel_launches(void) { return g_kernels.load(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Arithmetic roof of the element type: the FMA rate of this device, measured
// with independent dependent-FMA chains per thread (8 chains of `steps` FMAs,
// 2 flops each) on a grid of 8 CTAs of 256 threads per SM.
// ---------------------------------------------------------------------------
namespace mgb {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* out, int steps, T a, T b) {
  constexpr int K = 8;
  T x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < steps; ++i) {
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < K; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
int fma_rate(double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MGARD_ERR_CUDA;
  const int blocks = 8 * sms, threads = 256, steps = sizeof(T) == 8 ? 2048 : 16384;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return MGARD_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MGARD_OK;
  float best = 1e30f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MGARD_ERR_CUDA;
  } else {
    for (int r = 0; r < 4 && rc == MGARD_OK; ++r) {  // the first run warms up
      cudaEventRecord(e0, s);
      fma_rate_kernel<T><<<blocks, threads, 0, s>>>(out, steps, T(0.999999), T(1e-7));
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = MGARD_ERR_CUDA;
      else if (r > 0 && ms < best)
        best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == MGARD_OK)
    *flops_per_s = 2.0 * 8.0 * double(steps) * double(blocks) * threads / (double(best) * 1e-3);
  return rc;
}

}  // namespace
}  // namespace mgb

extern "C" int mgard_trace_fma_rate(int dtype, double* flops_per_s, void* stream) {
  if (flops_per_s == nullptr || (dtype != MGARD_F32 && dtype != MGARD_F64)) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return dtype == MGARD_F64 ? mgb::fma_rate<double>(flops_per_s, s)
                            : mgb::fma_rate<float>(flops_per_s, s);
}
