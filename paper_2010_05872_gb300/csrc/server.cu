// Serving runtime: a request loop with continuous batching on one device.
//
// Requests are whole compressions (host field -> host labels: value range,
// decomposition, level-wise quantization, Section 2 and Section 4.1) or
// decompressions (host labels -> host field: dequantization, recomposition).
// A scheduler thread owns up to `slots` CUDA streams.  Pending requests are
// admitted in arrival order as soon as a stream is free and the request's
// device memory (field, labels, workspace) fits in the HBM budget beside the
// requests already admitted; their copies and kernels then overlap on the
// device with the other admitted requests.  Device buffers come from the
// device's stream-ordered memory pool, which keeps freed memory for reuse up
// to the budget, and plans (level hierarchies, operator tables) stay resident
// in the plan cache.  A compression runs in two device phases: range and
// decomposition, then (once the scheduler has read the range and built the
// bin widths on the host, exactly as mgard_compress_host does) quantization
// and the copy of the labels.  The scheduler notices finished phases by
// polling CUDA events and never blocks on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "devplan.hpp"
#include "kernels.cuh"
#include "mgard_gb.h"

namespace mgb {
namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  cudaStream_t s = nullptr;
  unsigned int* flags = nullptr;   // device [4]: quantizer flags, wait-timeout status
  double* partial = nullptr;       // device [2 * kMinmaxBlocks]
  double* result = nullptr;        // device [2]
  unsigned int* h_flags = nullptr; // pinned [4]
  double* h_result = nullptr;      // pinned [2]
  cudaEvent_t ev = nullptr;
  bool busy = false;
};

struct Req {
  int64_t id = 0;
  mgard_request r{};
  Clock::time_point t_arrive;
  DevPlan* plan = nullptr;
  size_t need = 0;     // device bytes reserved
  int slot = -1;
  int phase = 0;       // compress: 1 = range + decompose, 2 = quantize + copy-out
  void* field = nullptr;
  int64_t* labels = nullptr;
  char* ws = nullptr;
  double tau = 0.0;
  int status = MGARD_OK;
};

struct Done {
  int64_t id;
  int status;
  double latency_s;
  double tau;
};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

class Server {
 public:
  int init(size_t budget, int slots) {
    if (cudaGetDevice(&device_) != cudaSuccess) return MGARD_ERR_CUDA;
    budget_ = budget;
    slots_.resize(std::max(1, slots));
    for (Slot& sl : slots_) {
      if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaMalloc(&sl.flags, 4 * sizeof(unsigned)) != cudaSuccess ||
          cudaMalloc(&sl.partial, 2 * kMinmaxBlocks * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&sl.result, 2 * sizeof(double)) != cudaSuccess ||
          cudaMallocHost(&sl.h_flags, 4 * sizeof(unsigned)) != cudaSuccess ||
          cudaMallocHost(&sl.h_result, 2 * sizeof(double)) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
        return MGARD_ERR_CUDA;
      if (cudaMemset(sl.flags, 0, 4 * sizeof(unsigned)) != cudaSuccess) return MGARD_ERR_CUDA;
    }
    // Freed pool memory stays with the pool up to the budget.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device_) == cudaSuccess) {
      uint64_t thr = budget_;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    running_ = true;
    thread_ = std::thread([this] { loop(); });
    return MGARD_OK;
  }

  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      running_ = false;
    }
    if (thread_.joinable()) thread_.join();
    for (Slot& sl : slots_) {
      if (sl.s) cudaStreamSynchronize(sl.s);
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.flags) cudaFree(sl.flags);
      if (sl.partial) cudaFree(sl.partial);
      if (sl.result) cudaFree(sl.result);
      if (sl.h_flags) cudaFreeHost(sl.h_flags);
      if (sl.h_result) cudaFreeHost(sl.h_result);
      if (sl.s) cudaStreamDestroy(sl.s);
    }
  }

  int submit(const mgard_request& r, int64_t* id) {
    if (r.host_in == nullptr || r.host_out == nullptr) return MGARD_ERR_ARG;
    if (r.op != MGARD_OP_COMPRESS && r.op != MGARD_OP_DECOMPRESS) return MGARD_ERR_ARG;
    if (r.op == MGARD_OP_COMPRESS && !(r.rel_bound > 0.0)) return MGARD_ERR_ARG;
    if (r.op == MGARD_OP_DECOMPRESS && !(r.tau > 0.0)) return MGARD_ERR_ARG;
    if (r.dtype != MGARD_F32 && r.dtype != MGARD_F64) return MGARD_ERR_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != device_) cudaSetDevice(device_);
    auto q = std::make_unique<Req>();
    q->r = r;
    int rc = get_plan(r.ndim, r.dims, nullptr, r.dtype, &q->plan);
    if (dev != device_) cudaSetDevice(dev);
    if (rc != MGARD_OK) return rc;
    if (r.stop_level < 0 || r.stop_level > q->plan->h.L) return MGARD_ERR_LEVEL;
    const size_t n = static_cast<size_t>(q->plan->h.count());
    q->need = up256(n * (r.dtype == MGARD_F64 ? 8 : 4)) + up256(n * 8) + up256(q->plan->ws_bytes);
    if (q->need > budget_) return MGARD_ERR_WORKSPACE;
    q->t_arrive = Clock::now();
    std::lock_guard<std::mutex> lk(mu_);
    q->id = next_id_++;
    *id = q->id;
    pending_.push_back(std::move(q));
    return MGARD_OK;
  }

  int poll(int max, int64_t* ids, int* status, double* latency, double* tau, int* count) {
    std::lock_guard<std::mutex> lk(mu_);
    int k = 0;
    while (k < max && !done_.empty()) {
      const Done& d = done_.front();
      if (ids) ids[k] = d.id;
      if (status) status[k] = d.status;
      if (latency) latency[k] = d.latency_s;
      if (tau) tau[k] = d.tau;
      done_.pop_front();
      ++k;
    }
    *count = k;
    return MGARD_OK;
  }

  int drain(double timeout_s) {
    const auto t0 = Clock::now();
    for (;;) {
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (pending_.empty() && inflight_.empty()) return MGARD_OK;
      }
      if (std::chrono::duration<double>(Clock::now() - t0).count() > timeout_s)
        return MGARD_ERR_TIMEOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }

  void counters(int64_t* out) {
    std::lock_guard<std::mutex> lk(mu_);
    out[0] = static_cast<int64_t>(pending_.size());
    out[1] = static_cast<int64_t>(inflight_.size());
    out[2] = static_cast<int64_t>(in_use_);
    out[3] = static_cast<int64_t>(peak_inflight_);
    out[4] = static_cast<int64_t>(peak_in_use_);
  }

 private:
  void finish(Req& q, int status) {
    Slot& sl = slots_[q.slot];
    cudaStream_t s = sl.s;
    if (q.field) cudaFreeAsync(q.field, s);
    if (q.labels) cudaFreeAsync(q.labels, s);
    if (q.ws) cudaFreeAsync(q.ws, s);
    sl.busy = false;
    in_use_ -= q.need;
    const double lat = std::chrono::duration<double>(Clock::now() - q.t_arrive).count();
    done_.push_back(Done{q.id, status, lat, q.tau});
  }

  // Enqueue the first device phase of an admitted request.
  int start(Req& q) {
    Slot& sl = slots_[q.slot];
    cudaStream_t s = sl.s;
    const DevPlan& p = *q.plan;
    const int64_t n = p.h.count();
    const size_t es = p.dtype == MGARD_F64 ? 8 : 4;
    if (cudaMallocAsync(&q.field, up256(n * es), s) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&q.labels), up256(n * 8), s) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&q.ws), up256(std::max<size_t>(p.ws_bytes, 256)),
                        s) != cudaSuccess)
      return MGARD_ERR_CUDA;
    if (cudaMemsetAsync(sl.flags, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return MGARD_ERR_CUDA;
    if (q.r.op == MGARD_OP_COMPRESS) {
      if (cudaMemcpyAsync(q.field, q.r.host_in, n * es, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MGARD_ERR_CUDA;
      const cudaError_t e =
          p.dtype == MGARD_F64
              ? launch_minmax<double>(static_cast<const double*>(q.field), n, sl.partial, sl.flags,
                                      sl.result, s)
              : launch_minmax<float>(static_cast<const float*>(q.field), n, sl.partial, sl.flags,
                                     sl.result, s);
      if (e != cudaSuccess) return MGARD_ERR_CUDA;
      if (cudaMemcpyAsync(sl.h_result, sl.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
        return MGARD_ERR_CUDA;
      int rc = run_transform(true, p, q.r.stop_level, q.field, q.ws, sl.flags + 1, s);
      if (rc != MGARD_OK) return rc;
      if (cudaMemcpyAsync(sl.h_flags, sl.flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
        return MGARD_ERR_CUDA;
      q.phase = 1;
    } else {
      if (cudaMemcpyAsync(q.labels, q.r.host_in, n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MGARD_ERR_CUDA;
      LevelTable tab;
      int rc = make_table(p, q.r.stop_level, q.r.tau, tab, nullptr);
      if (rc != MGARD_OK) return rc;
      q.tau = q.r.tau;
      const auto& d = p.h.dims3;
      const cudaError_t e =
          p.dtype == MGARD_F64
              ? launch_dequantize<double>(q.labels, static_cast<double*>(q.field), p.lev01, p.lev[2],
                                          d[0] * d[1], d[2], q.r.stop_level, tab, s)
              : launch_dequantize<float>(q.labels, static_cast<float*>(q.field), p.lev01, p.lev[2],
                                         d[0] * d[1], d[2], q.r.stop_level, tab, s);
      if (e != cudaSuccess) return MGARD_ERR_CUDA;
      rc = run_transform(false, p, q.r.stop_level, q.field, q.ws, sl.flags + 1, s);
      if (rc != MGARD_OK) return rc;
      if (cudaMemcpyAsync(q.r.host_out, q.field, n * es, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(sl.h_flags, sl.flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess)
        return MGARD_ERR_CUDA;
      q.phase = 2;
    }
    return cudaEventRecord(sl.ev, s) == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
  }

  // The range is known: bin widths on the host, then quantization and the
  // copy of the labels.
  int second_phase(Req& q) {
    Slot& sl = slots_[q.slot];
    cudaStream_t s = sl.s;
    const DevPlan& p = *q.plan;
    if (sl.h_flags[1]) return MGARD_ERR_TIMEOUT;
    if (sl.h_flags[0] & 1u) return MGARD_ERR_NONFINITE;
    const double lo = sl.h_result[0], hi = sl.h_result[1];
    double tau = q.r.rel_bound * (hi - lo);
    if (!(tau > 0.0)) tau = q.r.rel_bound * (std::fabs(lo) > 0.0 ? std::fabs(lo) : 1.0);
    q.tau = tau;
    LevelTable tab;
    int rc = make_table(p, q.r.stop_level, tau, tab, nullptr);
    if (rc != MGARD_OK) return rc;
    if (cudaMemsetAsync(sl.flags, 0, sizeof(unsigned), s) != cudaSuccess) return MGARD_ERR_CUDA;
    const auto& d = p.h.dims3;
    const cudaError_t e =
        p.dtype == MGARD_F64
            ? launch_quantize<double>(static_cast<const double*>(q.field), q.labels, p.lev01,
                                      p.lev[2], d[0] * d[1], d[2], q.r.stop_level, tab, sl.flags, s)
            : launch_quantize<float>(static_cast<const float*>(q.field), q.labels, p.lev01, p.lev[2],
                                     d[0] * d[1], d[2], q.r.stop_level, tab, sl.flags, s);
    if (e != cudaSuccess) return MGARD_ERR_CUDA;
    const int64_t n = p.h.count();
    if (cudaMemcpyAsync(q.r.host_out, q.labels, n * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(sl.h_flags, sl.flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
      return MGARD_ERR_CUDA;
    q.phase = 2;
    return cudaEventRecord(sl.ev, s) == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
  }

  int final_status(const Slot& sl) {
    if (sl.h_flags[1]) return MGARD_ERR_TIMEOUT;
    if (sl.h_flags[0] & 1u) return MGARD_ERR_NONFINITE;
    if (sl.h_flags[0] & 2u) return MGARD_ERR_OVERFLOW;
    return MGARD_OK;
  }

  void loop() {
    cudaSetDevice(device_);
    for (;;) {
      bool worked = false;
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (!running_ && pending_.empty() && inflight_.empty()) break;
        // Progress the admitted requests whose current phase has ended.
        for (size_t i = 0; i < inflight_.size();) {
          Req& q = *inflight_[i];
          Slot& sl = slots_[q.slot];
          const cudaError_t e = cudaEventQuery(sl.ev);
          if (e == cudaErrorNotReady) { ++i; continue; }
          worked = true;
          int rc = e == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
          if (rc == MGARD_OK && q.phase == 1) {
            rc = second_phase(q);
            if (rc == MGARD_OK) { ++i; continue; }
          } else if (rc == MGARD_OK) {
            rc = final_status(sl);
          }
          finish(q, rc);
          inflight_.erase(inflight_.begin() + static_cast<long>(i));
        }
        // Admit in arrival order while a stream is free and memory fits.
        while (!pending_.empty()) {
          Req& q = *pending_.front();
          if (in_use_ + q.need > budget_) break;
          int free_slot = -1;
          for (size_t k = 0; k < slots_.size(); ++k)
            if (!slots_[k].busy) { free_slot = static_cast<int>(k); break; }
          if (free_slot < 0) break;
          std::unique_ptr<Req> own = std::move(pending_.front());
          pending_.pop_front();
          own->slot = free_slot;
          slots_[free_slot].busy = true;
          in_use_ += own->need;
          peak_in_use_ = std::max(peak_in_use_, in_use_);
          worked = true;
          const int rc = start(*own);
          if (rc != MGARD_OK) {
            cudaStreamSynchronize(slots_[free_slot].s);
            finish(*own, rc);
            continue;
          }
          inflight_.push_back(std::move(own));
          peak_inflight_ = std::max(peak_inflight_, inflight_.size());
        }
      }
      if (!worked) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }

  int device_ = 0;
  size_t budget_ = 0;
  std::vector<Slot> slots_;
  std::mutex mu_;
  bool running_ = false;
  std::thread thread_;
  std::deque<std::unique_ptr<Req>> pending_;
  std::vector<std::unique_ptr<Req>> inflight_;
  std::deque<Done> done_;
  size_t in_use_ = 0, peak_in_use_ = 0, peak_inflight_ = 0;
  int64_t next_id_ = 1;
};

}  // namespace
}  // namespace mgb

using mgb::Server;

extern "C" {

int mgard_server_create(size_t hbm_budget, int slots, void** server) {
  if (server == nullptr || hbm_budget == 0 || slots < 1) return MGARD_ERR_ARG;
  auto s = std::make_unique<Server>();
  const int rc = s->init(hbm_budget, slots);
  if (rc != MGARD_OK) return rc;
  *server = s.release();
  return MGARD_OK;
}

int mgard_server_submit(void* server, const mgard_request* req, int64_t* id_out) {
  if (server == nullptr || req == nullptr || id_out == nullptr) return MGARD_ERR_ARG;
  return static_cast<Server*>(server)->submit(*req, id_out);
}

int mgard_server_poll(void* server, int max, int64_t* ids, int* status, double* latency_s,
                      double* tau, int* count_out) {
  if (server == nullptr || count_out == nullptr || max < 0) return MGARD_ERR_ARG;
  return static_cast<Server*>(server)->poll(max, ids, status, latency_s, tau, count_out);
}

int mgard_server_drain(void* server, double timeout_s) {
  if (server == nullptr) return MGARD_ERR_ARG;
  return static_cast<Server*>(server)->drain(timeout_s);
}

int mgard_server_counters(void* server, int64_t* out5) {
  if (server == nullptr || out5 == nullptr) return MGARD_ERR_ARG;
  static_cast<Server*>(server)->counters(out5);
  return MGARD_OK;
}

int mgard_server_destroy(void* server) {
  if (server == nullptr) return MGARD_ERR_ARG;
  delete static_cast<Server*>(server);
  return MGARD_OK;
}

}  // extern "C"
