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
