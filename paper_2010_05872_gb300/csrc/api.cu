// extern "C" entry points declared in include/mgard_gb.h: argument checks,
// the per-device plan cache (host tables uploaded once), the workspace
// layout and the level loops of decomposition / recomposition (Section 2).
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "devplan.hpp"
#include "kernels.cuh"
#include "mgard_gb.h"
#include "plan.hpp"

namespace mgb {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

std::mutex g_mu;
std::map<std::string, std::unique_ptr<DevPlan>> g_plans;
std::map<int, std::unique_ptr<DevCtx>> g_ctx;
std::map<std::pair<int, uintptr_t>, std::unique_ptr<StreamScratch>> g_scratch;

template <typename T>
void fill_levels(DevPlan& p, const std::vector<std::vector<size_t>>& offs, char* base,
                 std::vector<LevelK<T>>& out) {
  out.assign(p.h.L + 1, LevelK<T>{});
  for (int l = 1; l <= p.h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      const AxisTables& t = p.h.ax[l][a];
      const size_t* o = offs[l * 3 + a].data();
      AxisK<T>& k = out[l].ax[a];
      k.iwl = reinterpret_cast<const T*>(base + o[0]);
      k.iwr = reinterpret_cast<const T*>(base + o[1]);
      k.rw = reinterpret_cast<const T*>(base + o[2]);
      k.ta = reinterpret_cast<const T*>(base + o[3]);
      k.tm = reinterpret_cast<const T*>(base + o[4]);
      k.tc = reinterpret_cast<const T*>(base + o[5]);
      k.xd = reinterpret_cast<const T*>(base + o[6]);
      k.xr = reinterpret_cast<const T*>(base + o[7]);
      k.sb = reinterpret_cast<const T*>(base + o[8]);
      k.sg = reinterpret_cast<const T*>(base + o[9]);
      k.sy = reinterpret_cast<const T*>(base + o[10]);
      k.sh = reinterpret_cast<const T*>(base + o[11]);
      k.seg_len = t.seg_len;
      k.n = t.n;
      k.nc = t.nc;
    }
}

template <typename T>
int upload(DevPlan& p) {
  const HostPlan& h = p.h;
  std::vector<std::vector<size_t>> offs((h.L + 1) * 3);
  size_t total = 0;
  auto reserve = [&](size_t bytes) { const size_t o = total; total = align_up(total + bytes, 16); return o; };
  for (int l = 1; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      const AxisTables& t = h.ax[l][a];
      auto& o = offs[l * 3 + a];
      o.push_back(reserve(sizeof(T) * t.iwl.size()));
      o.push_back(reserve(sizeof(T) * t.iwr.size()));
      o.push_back(reserve(sizeof(T) * t.rw.size()));
      o.push_back(reserve(sizeof(T) * t.ta.size()));
      o.push_back(reserve(sizeof(T) * t.tm.size()));
      o.push_back(reserve(sizeof(T) * t.tc.size()));
      o.push_back(reserve(sizeof(T) * t.xd.size()));
      o.push_back(reserve(sizeof(T) * t.xr.size()));
      for (const auto* v : {&t.sb, &t.sg, &t.sy, &t.sh}) o.push_back(reserve(sizeof(T) * v->size()));
    }
  size_t lev_off[3];
  for (int a = 0; a < 3; ++a) lev_off[a] = reserve(h.lev[a].size());
  const size_t lev01_off = reserve(h.lev01.size());
  std::vector<std::array<size_t, 3>> pos_off(h.L + 1);
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) pos_off[l][a] = reserve(sizeof(int32_t) * h.idx[l][a].size());
  size_t x_off[3];
  for (int a = 0; a < 3; ++a) x_off[a] = reserve(sizeof(double) * h.x[a].size());
  std::vector<char> stage(total, 0);
  auto put = [&](size_t off, const std::vector<double>& v) {
    T* dst = reinterpret_cast<T*>(stage.data() + off);
    for (size_t i = 0; i < v.size(); ++i) dst[i] = static_cast<T>(v[i]);
  };
  for (int l = 1; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      const AxisTables& t = h.ax[l][a];
      const auto& o = offs[l * 3 + a];
      put(o[0], t.iwl); put(o[1], t.iwr); put(o[2], t.rw);
      put(o[3], t.ta); put(o[4], t.tm); put(o[5], t.tc);
      put(o[6], t.xd); put(o[7], t.xr);
      put(o[8], t.sb); put(o[9], t.sg); put(o[10], t.sy); put(o[11], t.sh);
    }
  for (int a = 0; a < 3; ++a) std::memcpy(stage.data() + lev_off[a], h.lev[a].data(), h.lev[a].size());
  std::memcpy(stage.data() + lev01_off, h.lev01.data(), h.lev01.size());
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      int32_t* dst = reinterpret_cast<int32_t*>(stage.data() + pos_off[l][a]);
      for (size_t j = 0; j < h.idx[l][a].size(); ++j) dst[j] = static_cast<int32_t>(h.idx[l][a][j]);
    }
  for (int a = 0; a < 3; ++a)
    std::memcpy(stage.data() + x_off[a], h.x[a].data(), sizeof(double) * h.x[a].size());
  if (cudaMalloc(&p.dmem, total) != cudaSuccess) return MGARD_ERR_CUDA;
  if (cudaMemcpy(p.dmem, stage.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) return MGARD_ERR_CUDA;
  char* base = static_cast<char*>(p.dmem);
  if constexpr (sizeof(T) == 4) fill_levels<float>(p, offs, base, p.lvf);
  else fill_levels<double>(p, offs, base, p.lvd);
  for (int a = 0; a < 3; ++a) p.lev[a] = reinterpret_cast<const uint8_t*>(base + lev_off[a]);
  p.lev01 = reinterpret_cast<const uint8_t*>(base + lev01_off);
  p.pos.resize(h.L + 1);
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) p.pos[l][a] = reinterpret_cast<const int32_t*>(base + pos_off[l][a]);
  for (int a = 0; a < 3; ++a) p.xc[a] = reinterpret_cast<const double*>(base + x_off[a]);
  return MGARD_OK;
}

size_t elem_size(int dtype) { return dtype == MGARD_F64 ? 8 : 4; }

void layout_workspace(DevPlan& p) {
  const size_t es = elem_size(p.dtype);
  p.offB.assign(p.h.L + 1, 0);
  p.offF.assign(p.h.L + 1, 0);
  size_t off = 0;
  for (int l = p.h.L - 1; l >= 0; --l) {
    const size_t cnt = static_cast<size_t>(p.h.shape[l][0] * p.h.shape[l][1] * p.h.shape[l][2]);
    p.offB[l] = off; off = align_up(off + cnt * es, kAlign);
    p.offF[l] = off; off = align_up(off + cnt * es, kAlign);
  }
  p.ws_bytes = off;
}

std::string plan_key(int device, int dtype, const HostPlan& h) {
  std::string k;
  auto app = [&](const void* d, size_t n) { k.append(static_cast<const char*>(d), n); };
  app(&device, sizeof device);
  app(&dtype, sizeof dtype);
  app(&h.ndim, sizeof h.ndim);
  app(h.dims3.data(), sizeof(int64_t) * 3);
  app(h.coords_key.data(), sizeof(double) * h.coords_key.size());
  return k;
}

}  // namespace

// Look up (or build and upload) the plan of this shape/coords/dtype on the
// current device.
int get_plan(int ndim, const int64_t* dims, const double* const* coords, int dtype, DevPlan** out) {
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  int rc = check_shape(ndim, dims);
  if (rc != MGARD_OK) return rc;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGARD_ERR_CUDA;
  // Cheap key first: coordinates are validated by the full build.
  HostPlan probe;
  probe.ndim = ndim;
  const int pad = 3 - ndim;
  for (int d = 0; d < ndim; ++d) probe.dims3[pad + d] = dims[d];
  for (int d = 0; d < ndim; ++d) {
    const double* c = coords ? coords[d] : nullptr;
    if (c) probe.coords_key.insert(probe.coords_key.end(), c, c + dims[d]);
    probe.coords_key.push_back(c ? 1.0 : 0.0);
  }
  const std::string key = plan_key(device, dtype, probe);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) { *out = it->second.get(); return MGARD_OK; }
  auto p = std::make_unique<DevPlan>();
  rc = build_host_plan(ndim, dims, coords, p->h);
  if (rc != MGARD_OK) return rc;
  p->dtype = dtype;
  p->device = device;
  rc = (dtype == MGARD_F64) ? upload<double>(*p) : upload<float>(*p);
  if (rc != MGARD_OK) return rc;
  layout_workspace(*p);
  *out = p.get();
  g_plans.emplace(key, std::move(p));
  return MGARD_OK;
}

DevCtx* get_ctx() {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ctx.find(device);
  if (it != g_ctx.end()) return it->second.get();
  auto c = std::make_unique<DevCtx>();
  if (cudaMalloc(&c->flags, 4 * sizeof(unsigned)) != cudaSuccess) return nullptr;
  if (cudaMemset(c->flags, 0, 4 * sizeof(unsigned)) != cudaSuccess) return nullptr;
  if (cudaMalloc(&c->partial, 2 * kMinmaxBlocks * sizeof(double)) != cudaSuccess) return nullptr;
  if (cudaMalloc(&c->sums, 2 * kMaxLevels * sizeof(double)) != cudaSuccess) return nullptr;
  if (cudaMallocHost(&c->h_sums, 2 * kMaxLevels * sizeof(double)) != cudaSuccess) return nullptr;
  DevCtx* raw = c.get();
  g_ctx.emplace(device, std::move(c));
  return raw;
}

StreamScratch* get_scratch(cudaStream_t s) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return nullptr;
  const auto key = std::make_pair(device, reinterpret_cast<uintptr_t>(s));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_scratch.find(key);
  if (it != g_scratch.end()) return it->second.get();
  auto sc = std::make_unique<StreamScratch>();
  void* dmem = nullptr;
  const size_t bytes = 256 + sizeof(double) * (2 * kMinmaxBlocks + 2);
  if (cudaMalloc(&dmem, bytes) != cudaSuccess) return nullptr;
  if (cudaMemset(dmem, 0, bytes) != cudaSuccess ||
      cudaMallocHost(&sc->h_flags, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaFree(dmem);
    return nullptr;
  }
  if (cudaMallocHost(&sc->h_result, 2 * sizeof(double)) != cudaSuccess) {
    cudaFreeHost(sc->h_flags);
    cudaFree(dmem);
    return nullptr;
  }
  sc->flag = static_cast<unsigned int*>(dmem);
  sc->result = reinterpret_cast<double*>(static_cast<char*>(dmem) + 256);
  sc->partial = sc->result + 2;
  StreamScratch* raw = sc.get();
  g_scratch.emplace(key, std::move(sc));
  return raw;
}

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA; }
#define MGB_TRY(expr) do { const cudaError_t e_ = (expr); if (e_ != cudaSuccess) return MGARD_ERR_CUDA; } while (0)

int check_transform_args(const DevPlan& p, int stop_level, const void* data, const void* ws,
                         size_t ws_bytes) {
  if (stop_level < 0 || stop_level > p.h.L) return MGARD_ERR_LEVEL;
  if (data == nullptr || reinterpret_cast<uintptr_t>(data) % elem_size(p.dtype) != 0) return MGARD_ERR_ARG;
  if (p.h.L > stop_level) {
    if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % kAlign != 0) return MGARD_ERR_WORKSPACE;
    if (ws_bytes < p.ws_bytes) return MGARD_ERR_WORKSPACE;
  }
  return MGARD_OK;
}

template <typename T>
const std::vector<LevelK<T>>& levels(const DevPlan& p);
template <>
const std::vector<LevelK<float>>& levels<float>(const DevPlan& p) { return p.lvf; }
template <>
const std::vector<LevelK<double>>& levels<double>(const DevPlan& p) { return p.lvd; }

namespace {

// Decomposition, levels L .. l~+1: load vector (reads the level-l grid only),
// solves with the correction applied to the gathered coarse values; then,
// coarsest first, the finishing pass writes each level's coefficients and the
// final coarser values into the level-l grid.
// The highest level ls (stop < ls <= L) whose grid and every grid below it
// fit the one-CTA form of the coarsest levels, or stop if none does.
template <typename T>
int small_top(const DevPlan& p, int stop) {
  const auto& lv = levels<T>(p);
  int ls = stop;
  for (int l = stop + 1; l <= p.h.L && l - stop <= kSmallMaxLevels; ++l) {
    const auto& d = p.h.shape[l];
    if (d[0] * d[1] * d[2] > kSmallMaxNodes) break;
    if (small_levels_smem<T>(&lv[stop + 1], l - stop) > kSmallMaxSmem) break;
    ls = l;
  }
  return ls;
}

template <typename T>
int run_decompose(const DevPlan& p, int stop, T* data, char* ws, unsigned int* status,
                  cudaStream_t s) {
  const int L = p.h.L;
  const auto& lv = levels<T>(p);
  std::vector<T*> B(L + 1), F(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) {
    B[l] = reinterpret_cast<T*>(ws + p.offB[l]);
    F[l] = reinterpret_cast<T*>(ws + p.offF[l]);
  }
  const int ls = small_top<T>(p, stop);
  for (int l = L; l > ls; --l) {
    MGB_TRY(launch_load_vector<T>(lv[l], true, B[l], B[l - 1], F[l - 1], l, status, s));
    MGB_TRY(launch_solves<T>(lv[l], F[l - 1], B[l - 1], kApplyDecompose, l, status, s));
  }
  if (ls > stop) MGB_TRY(launch_small_levels<T>(&lv[stop + 1], ls - stop, true, B[ls], ls, s));
  for (int l = ls + 1; l <= L; ++l)
    MGB_TRY(launch_finish<T>(lv[l], B[l - 1], F[l - 1], T(-1), B[l], l, status, s));
  return MGARD_OK;
}

// Recomposition: gather every level's coarse part and load vector top-down,
// then bottom-up solve, subtract the correction and interpolate.
template <typename T>
int run_recompose(const DevPlan& p, int stop, T* data, char* ws, unsigned int* status,
                  cudaStream_t s) {
  const int L = p.h.L;
  const auto& lv = levels<T>(p);
  std::vector<T*> B(L + 1), F(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) {
    B[l] = reinterpret_cast<T*>(ws + p.offB[l]);
    F[l] = reinterpret_cast<T*>(ws + p.offF[l]);
  }
  const int ls = small_top<T>(p, stop);
  for (int l = L; l > ls; --l)
    MGB_TRY(launch_load_vector<T>(lv[l], false, B[l], B[l - 1], F[l - 1], l, status, s));
  if (ls > stop) MGB_TRY(launch_small_levels<T>(&lv[stop + 1], ls - stop, false, B[ls], ls, s));
  for (int l = ls + 1; l <= L; ++l) {
    MGB_TRY(launch_solves<T>(lv[l], F[l - 1], B[l - 1], kApplyRecompose, l, status, s));
    MGB_TRY(launch_finish<T>(lv[l], B[l - 1], B[l - 1], T(1), B[l], l, status, s));
  }
  return MGARD_OK;
}

// Levels of more nodes than this are decided one at a time (decomposing one
// in vain would cost more than the wait); the smaller ones are decomposed
// ahead of their decisions.
constexpr int64_t kAdaptiveAheadNodes = 20000000;

// Adaptive decomposition (the stopping-level search of Algorithm 1): from
// the finest level down, the sampled prediction-error sums of the level-l
// grid decide between stopping at l and decomposing it; then the finish
// passes of the decomposed levels.  One host synchronization per sampled level.
template <typename T>
int run_adaptive(const DevPlan& p, double tau, T* data, char* ws, DevCtx* c, cudaStream_t s,
                 int* stop_out, double* sums) {
  const int L = p.h.L;
  const auto& lv = levels<T>(p);
  std::vector<T*> B(L + 1), F(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) {
    B[l] = reinterpret_cast<T*>(ws + p.offB[l]);
    F[l] = reinterpret_cast<T*>(ws + p.offF[l]);
  }
  unsigned int* status = c->flags + 1;
  double t[kMaxLevels];
  auto nodes = [&](int l) { return p.h.shape[l][0] * p.h.shape[l][1] * p.h.shape[l][2]; };
  auto decompose_level = [&](int l) -> int {
    MGB_TRY(launch_load_vector<T>(lv[l], true, B[l], B[l - 1], F[l - 1], l, status, s));
    MGB_TRY(launch_solves<T>(lv[l], F[l - 1], B[l - 1], kApplyDecompose, l, status, s));
    return MGARD_OK;
  };
  auto record = [&](int l) {
    if (sums) {
      sums[2 * l] = c->h_sums[2 * l];
      sums[2 * l + 1] = c->h_sums[2 * l + 1];
    }
    return c->h_sums[2 * l] < c->h_sums[2 * l + 1];  // Lorenzo wins: stop here
  };
  int stop = -1;
  int l = L;
  // Large levels one at a time: sample, wait for the sums, decide.
  for (; l >= 1 && nodes(l) > kAdaptiveAheadNodes; --l) {
    level_tolerances(p.h, l, tau, t);  // t[l]: tau_0 were l the stopping level
    MGB_TRY(launch_prediction_errors<T>(lv[l], B[l], t[l], c->partial, c->sums + 2 * l, l, s));
    MGB_TRY(cudaMemcpyAsync(c->h_sums + 2 * l, c->sums + 2 * l, 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    MGB_TRY(cudaStreamSynchronize(s));
    if (record(l)) {
      stop = l;
      break;
    }
    const int rc = decompose_level(l);
    if (rc != MGARD_OK) return rc;
  }
  if (stop < 0) {
    // The smaller levels all at once: each is sampled and decomposed without
    // a wait (the load vector and solves of a level write only coarser
    // arrays, so work below the stopping level changes nothing that is
    // kept); one read of their sums then gives the stopping level, the first
    // from the finest whose Lorenzo sum is below its interpolation sum.
    const int top = l;
    for (int m = top; m >= 1; --m) {
      level_tolerances(p.h, m, tau, t);
      MGB_TRY(launch_prediction_errors<T>(lv[m], B[m], t[m], c->partial, c->sums + 2 * m, m, s));
      const int rc = decompose_level(m);
      if (rc != MGARD_OK) return rc;
    }
    if (top >= 1) {
      MGB_TRY(cudaMemcpyAsync(c->h_sums + 2, c->sums + 2, 2 * top * sizeof(double),
                              cudaMemcpyDeviceToHost, s));
      MGB_TRY(cudaStreamSynchronize(s));
    }
    stop = 0;
    for (int m = top; m >= 1; --m)
      if (record(m)) {
        stop = m;
        break;
      }
  }
  for (int l = stop + 1; l <= L; ++l)
    MGB_TRY(launch_finish<T>(lv[l], B[l - 1], F[l - 1], T(-1), B[l], l, status, s));
  *stop_out = stop;
  return MGARD_OK;
}

int transform(bool dec, int ndim, const int64_t* dims, const double* const* coords, int dtype,
              int stop_level, void* data, void* workspace, size_t ws_bytes, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (stop_level == p->h.L) return MGARD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  unsigned int* status = c->flags + 1;
  if (dtype == MGARD_F64)
    return dec ? run_decompose<double>(*p, stop_level, static_cast<double*>(data), ws, status, s)
               : run_recompose<double>(*p, stop_level, static_cast<double*>(data), ws, status, s);
  return dec ? run_decompose<float>(*p, stop_level, static_cast<float*>(data), ws, status, s)
             : run_recompose<float>(*p, stop_level, static_cast<float*>(data), ws, status, s);
}

int transform_host(bool dec, int ndim, const int64_t* dims, const double* const* coords, int dtype,
                   int stop_level, const void* host_in, void* host_out, void* dev_data,
                   void* workspace, size_t ws_bytes, void* stream) {
  if (host_in == nullptr || host_out == nullptr) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, dev_data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = static_cast<size_t>(p->h.count()) * elem_size(dtype);
  MGB_TRY(cudaMemcpyAsync(dev_data, host_in, bytes, cudaMemcpyHostToDevice, s));
  rc = transform(dec, ndim, dims, coords, dtype, stop_level, dev_data, workspace, ws_bytes, stream);
  if (rc != MGARD_OK) return rc;
  MGB_TRY(cudaMemcpyAsync(host_out, dev_data, bytes, cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  return MGARD_OK;
}

}  // namespace

int run_transform(bool dec, const DevPlan& p, int stop_level, void* data, char* ws,
                  unsigned int* status, cudaStream_t s) {
  if (p.dtype == MGARD_F64)
    return dec ? run_decompose<double>(p, stop_level, static_cast<double*>(data), ws, status, s)
               : run_recompose<double>(p, stop_level, static_cast<double*>(data), ws, status, s);
  return dec ? run_decompose<float>(p, stop_level, static_cast<float*>(data), ws, status, s)
             : run_recompose<float>(p, stop_level, static_cast<float*>(data), ws, status, s);
}

int make_table(const DevPlan& p, int stop_level, double tau, LevelTable& tab, double* tau_out) {
  if (!(tau > 0.0) || !std::isfinite(tau)) return MGARD_ERR_ARG;
  if (stop_level < 0 || stop_level > p.h.L) return MGARD_ERR_LEVEL;
  double t[kMaxLevels];
  level_tolerances(p.h, stop_level, tau, t);
  return make_table_levels(p, stop_level, t, tab, tau_out);
}

int make_table_levels(const DevPlan& p, int stop_level, const double* t, LevelTable& tab,
                      double* tau_out) {
  return make_level_table(p.h.L, stop_level, t, tab, tau_out);
}

int make_level_table(int L, int stop_level, const double* t, LevelTable& tab, double* tau_out) {
  if (stop_level < 0 || stop_level > L) return MGARD_ERR_LEVEL;
  for (int l = stop_level; l <= L; ++l)
    if (!(t[l] > 0.0) || !std::isfinite(t[l])) return MGARD_ERR_ARG;
  for (int l = 0; l < 48; ++l) {
    tab.q[l] = 1.0;
    tab.rq[l] = std::nanf("");
    tab.qf[l] = 1.0f;
    tab.dqf[l] = 0.0f;
  }
  for (int l = 0; l <= L; ++l) {
    // Levels below the stopping level are quantized with tau_{l~}.
    tab.q[l] = 2.0 * t[std::max(l, stop_level)];
    // The FP32 reciprocal drives the exact fast path of the quantizer; it is
    // only usable when it is a normal float.
    const double r = 1.0 / tab.q[l];
    const float rf = static_cast<float>(r);
    tab.rq[l] = (std::isfinite(rf) && rf >= 1.17549435e-38f) ? rf : std::nanf("");
    // FP32 split of q for the dequantizer's FP32 route (q - fl32(q) is exact
    // in FP64); a q outside the normal FP32 range disables that route.
    const float qf = static_cast<float>(tab.q[l]);
    const bool qok = std::isfinite(qf) && qf >= 1.17549435e-38f;
    tab.qf[l] = qok ? qf : std::nanf("");
    tab.dqf[l] = qok ? static_cast<float>(tab.q[l] - static_cast<double>(qf)) : 0.0f;
  }
  if (tau_out)
    for (int l = 0; l <= L; ++l) tau_out[l] = t[std::max(l, stop_level)];
  return MGARD_OK;
}

}  // namespace mgb

using namespace mgb;

extern "C" {

int mgard_num_levels(int ndim, const int64_t* dims, int* L_out) {
  if (L_out == nullptr) return MGARD_ERR_ARG;
  return count_levels(ndim, dims, L_out);
}

int mgard_workspace_size(int ndim, const int64_t* dims, int dtype, size_t* bytes) {
  if (bytes == nullptr) return MGARD_ERR_ARG;
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  int L = 0;
  int rc = count_levels(ndim, dims, &L);
  if (rc != MGARD_OK) return rc;
  int64_t cur[3] = {1, 1, 1};
  const int pad = 3 - ndim;
  for (int d = 0; d < ndim; ++d) cur[pad + d] = dims[d];
  size_t off = 0;
  const size_t es = elem_size(dtype);
  for (int l = L - 1; l >= 0; --l) {
    for (int a = pad; a < 3; ++a) cur[a] = cur[a] / 2 + 1;
    const size_t cnt = static_cast<size_t>(cur[0] * cur[1] * cur[2]);
    off = align_up(off + cnt * es, kAlign);
    off = align_up(off + cnt * es, kAlign);
  }
  *bytes = off;
  return MGARD_OK;
}

int mgard_level_tolerances(int ndim, const int64_t* dims, const double* const* coords,
                           int stop_level, double tau_linf, double* tau_out) {
  if (tau_out == nullptr) return MGARD_ERR_ARG;
  if (!(tau_linf > 0.0) || !std::isfinite(tau_linf)) return MGARD_ERR_ARG;
  HostPlan h;
  int rc = build_host_plan(ndim, dims, coords, h);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > h.L) return MGARD_ERR_LEVEL;
  level_tolerances(h, stop_level, tau_linf, tau_out);
  return MGARD_OK;
}

int mgard_level_tolerances_mode(int ndim, const int64_t* dims, const double* const* coords,
                                int stop_level, double tau, int mode, double* tau_out) {
  if (tau_out == nullptr || mode < 0 || mode > 2) return MGARD_ERR_ARG;
  if (!(tau > 0.0) || !std::isfinite(tau)) return MGARD_ERR_ARG;
  HostPlan h;
  int rc = build_host_plan(ndim, dims, coords, h);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > h.L) return MGARD_ERR_LEVEL;
  level_tolerances_mode(h, stop_level, tau, mode, tau_out);
  return MGARD_OK;
}

int mgard_decompose(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                    int stop_level, void* data, void* workspace, size_t ws_bytes, void* stream) {
  return transform(true, ndim, dims, coords, dtype, stop_level, data, workspace, ws_bytes, stream);
}

int mgard_recompose(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                    int stop_level, void* data, void* workspace, size_t ws_bytes, void* stream) {
  return transform(false, ndim, dims, coords, dtype, stop_level, data, workspace, ws_bytes, stream);
}

int mgard_decompose_adaptive(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                             double tau_linf, void* data, void* workspace, size_t ws_bytes,
                             int* stop_out, double* sums_out, void* stream) {
  if (stop_out == nullptr) return MGARD_ERR_ARG;
  if (!(tau_linf > 0.0) || !std::isfinite(tau_linf)) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (p->h.ndim != 3) return MGARD_ERR_SHAPE;
  rc = check_transform_args(*p, 0, data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (sums_out)
    for (int i = 0; i < 2 * (p->h.L + 1); ++i) sums_out[i] = std::nan("");
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  return dtype == MGARD_F64
             ? run_adaptive<double>(*p, tau_linf, static_cast<double*>(data), ws, c, s, stop_out,
                                    sums_out)
             : run_adaptive<float>(*p, tau_linf, static_cast<float*>(data), ws, c, s, stop_out,
                                   sums_out);
}

int mgard_level_grid(int ndim, const int64_t* dims, const double* const* coords, int level,
                     int64_t* shape_out, double* coords_out) {
  if (shape_out == nullptr) return MGARD_ERR_ARG;
  int L = 0;
  const int rc = count_levels(ndim, dims, &L);
  if (rc != MGARD_OK) return rc;
  if (level < 0 || level > L) return MGARD_ERR_LEVEL;
  size_t o = 0;
  for (int d = 0; d < ndim; ++d) {
    // Level-l positions from the finest: keep cpos(k, n) for k <= n / 2.
    std::vector<int64_t> ix(static_cast<size_t>(dims[d]));
    for (int64_t j = 0; j < dims[d]; ++j) ix[j] = j;
    for (int l = L; l > level; --l) {
      const int64_t n = static_cast<int64_t>(ix.size());
      std::vector<int64_t> c;
      for (int64_t k = 0; k < n / 2 + 1; ++k) c.push_back(ix[std::min(2 * k, n - 1)]);
      ix.swap(c);
    }
    shape_out[d] = static_cast<int64_t>(ix.size());
    if (coords_out) {
      const double* c = coords != nullptr ? coords[d] : nullptr;
      for (int64_t j : ix) coords_out[o++] = c ? c[j] : static_cast<double>(j);
    }
  }
  return MGARD_OK;
}

int mgard_recompose_partial(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                            int stop_level, int level, const void* data, void* out, void* workspace,
                            size_t ws_bytes, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > p->h.L || level < stop_level || level > p->h.L)
    return MGARD_ERR_LEVEL;
  const size_t es = elem_size(dtype);
  if (data == nullptr || out == nullptr || reinterpret_cast<uintptr_t>(data) % es ||
      reinterpret_cast<uintptr_t>(out) % es)
    return MGARD_ERR_ARG;
  // The level-k grid is a hierarchy of its own (the coarser levels of this
  // one), with the coordinates of its nodes.
  const int pad = 3 - ndim;
  int64_t dk[3];
  std::vector<std::vector<double>> ck(ndim);
  std::vector<const double*> cptr(ndim);
  for (int d = 0; d < ndim; ++d) {
    const auto& ix = p->h.idx[level][pad + d];
    dk[d] = static_cast<int64_t>(ix.size());
    for (int64_t j : ix) ck[d].push_back(p->h.x[pad + d][j]);
    cptr[d] = ck[d].data();
  }
  DevPlan* pk = nullptr;
  rc = get_plan(ndim, dk, cptr.data(), dtype, &pk);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*pk, stop_level, out, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t* pos[3] = {p->pos[level][0], p->pos[level][1], p->pos[level][2]};
  const int64_t* shape3 = p->h.shape[level].data();
  if (dtype == MGARD_F64)
    MGB_TRY(launch_gather_level<double>(static_cast<const double*>(data), p->h.dims3.data(), pos,
                                        shape3, static_cast<double*>(out), s));
  else
    MGB_TRY(launch_gather_level<float>(static_cast<const float*>(data), p->h.dims3.data(), pos,
                                       shape3, static_cast<float*>(out), s));
  if (stop_level == level) return MGARD_OK;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  return run_transform(false, *pk, stop_level, out, static_cast<char*>(workspace), c->flags + 1, s);
}

int mgard_iso_area(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                   const void* data, double iso, double* area_out, void* stream) {
  if (area_out == nullptr || !std::isfinite(iso)) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (p->h.ndim != 3) return MGARD_ERR_SHAPE;
  if (data == nullptr || reinterpret_cast<uintptr_t>(data) % elem_size(dtype)) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);
  if (sc == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sc->mu);
  const double* x[3] = {p->xc[0], p->xc[1], p->xc[2]};
  if (dtype == MGARD_F64)
    MGB_TRY(launch_iso_area<double>(static_cast<const double*>(data), p->h.dims3.data(), x, iso,
                                    sc->partial, sc->result, s));
  else
    MGB_TRY(launch_iso_area<float>(static_cast<const float*>(data), p->h.dims3.data(), x, iso,
                                   sc->partial, sc->result, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_result, sc->result, sizeof(double), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  *area_out = sc->h_result[0];
  return MGARD_OK;
}

int mgard_pack_bound(int64_t count, size_t* bytes) {
  if (count < 0 || bytes == nullptr) return MGARD_ERR_ARG;
  *bytes = pack_header_bytes(count) + 8 * static_cast<size_t>(count);
  return MGARD_OK;
}

namespace {

// Host-side check of a packed stream of `count` labels held in host memory:
// the count, the widths and the total size.
int check_stream(const uint8_t* h, size_t bytes, int64_t count) {
  const size_t hdr = pack_header_bytes(count);
  if (bytes < hdr) return MGARD_ERR_ARG;
  uint64_t n = 0;
  std::memcpy(&n, h, 8);
  if (n != static_cast<uint64_t>(count)) return MGARD_ERR_ARG;
  const int64_t nchunks = (count + kPackChunk - 1) / kPackChunk;
  uint64_t words = 0;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int w = h[8 + c];
    if (w > 64) return MGARD_ERR_ARG;
    const uint64_t nc = static_cast<uint64_t>(std::min<int64_t>(kPackChunk, count - c * kPackChunk));
    words += (nc * w + 63) / 64;
  }
  return hdr + 8 * words <= bytes ? MGARD_OK : MGARD_ERR_ARG;
}

// Pack on the device; *bytes_out receives the stream size (waits).
int pack_device(int64_t count, const int64_t* labels, void* out, size_t capacity,
                size_t* bytes_out, StreamScratch* sc, cudaStream_t s) {
  size_t bound = 0;
  mgard_pack_bound(count, &bound);
  if (capacity < bound) return MGARD_ERR_WORKSPACE;
  const int64_t nchunks = (count + kPackChunk - 1) / kPackChunk;
  uint64_t* scratch = nullptr;
  MGB_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(uint64_t) * (nchunks + 1), s));
  cudaError_t e = launch_pack_labels(labels, count, static_cast<uint8_t*>(out), scratch + 1, scratch, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sc->h_result, scratch, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MGARD_ERR_CUDA;
  uint64_t words = 0;
  std::memcpy(&words, sc->h_result, sizeof words);
  *bytes_out = pack_header_bytes(count) + 8 * static_cast<size_t>(words);
  return MGARD_OK;
}

int unpack_device(const void* in, int64_t count, int64_t* labels, cudaStream_t s) {
  const int64_t nchunks = (count + kPackChunk - 1) / kPackChunk;
  if (nchunks == 0) return MGARD_OK;
  uint64_t* scratch = nullptr;
  MGB_TRY(cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(uint64_t) * (nchunks + 1), s));
  const cudaError_t e =
      launch_unpack_labels(static_cast<const uint8_t*>(in), count, scratch + 1, scratch, labels, s);
  cudaFreeAsync(scratch, s);
  return e == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
}

}  // namespace

namespace {

// Lorenzo transform of the coarse block N_stop of `labels` (finest layout).
int lorenzo_device(bool encode, const DevPlan& p, int stop_level, int64_t* labels, cudaStream_t s) {
  const auto& sh = p.h.shape[stop_level];
  const int64_t total = sh[0] * sh[1] * sh[2];
  uint64_t* tmp = nullptr;
  MGB_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(uint64_t) * total, s));
  const int32_t* pos[3] = {p.pos[stop_level][0], p.pos[stop_level][1], p.pos[stop_level][2]};
  const cudaError_t e = launch_lorenzo(encode, labels, p.h.dims3.data(), pos, sh.data(), tmp, s);
  cudaFreeAsync(tmp, s);
  return e == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
}

int lorenzo_entry(bool encode, int ndim, const int64_t* dims, const double* const* coords,
                  int dtype, int stop_level, int64_t* labels, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > p->h.L) return MGARD_ERR_LEVEL;
  if (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8) return MGARD_ERR_ARG;
  return lorenzo_device(encode, *p, stop_level, labels, static_cast<cudaStream_t>(stream));
}

}  // namespace

int mgard_lorenzo_encode(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, int64_t* labels, void* stream) {
  return lorenzo_entry(true, ndim, dims, coords, dtype, stop_level, labels, stream);
}

int mgard_lorenzo_decode(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, int64_t* labels, void* stream) {
  return lorenzo_entry(false, ndim, dims, coords, dtype, stop_level, labels, stream);
}

int mgard_pack_labels(int64_t count, const int64_t* labels, void* out, size_t capacity,
                      size_t* bytes_out, void* stream) {
  if (count < 0 || bytes_out == nullptr || out == nullptr || reinterpret_cast<uintptr_t>(out) % 8)
    return MGARD_ERR_ARG;
  if (count > 0 && (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8)) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);
  if (sc == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sc->mu);
  return pack_device(count, labels, out, capacity, bytes_out, sc, s);
}

int mgard_unpack_labels(const void* in, size_t bytes, int64_t count, int64_t* labels, void* stream) {
  if (count < 0 || in == nullptr || reinterpret_cast<uintptr_t>(in) % 8) return MGARD_ERR_ARG;
  if (count > 0 && (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8)) return MGARD_ERR_ARG;
  const size_t hdr = pack_header_bytes(count);
  if (bytes < hdr) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<uint8_t> h(hdr);
  MGB_TRY(cudaMemcpyAsync(h.data(), in, hdr, cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  // The payload size follows from the header alone.
  std::vector<uint8_t> probe(h);
  const int rc = check_stream(probe.data(), bytes, count);
  if (rc != MGARD_OK) return rc;
  return unpack_device(in, count, labels, s);
}

int mgard_compress_host_packed(int ndim, const int64_t* dims, const double* const* coords,
                               int dtype, int stop_level, double rel_bound, const void* host_field,
                               void* host_stream, size_t host_capacity, size_t* stream_bytes,
                               double* tau_out, void* dev_data, int64_t* dev_labels,
                               void* dev_stream, size_t dev_capacity, void* workspace,
                               size_t ws_bytes, void* stream) {
  if (host_field == nullptr || host_stream == nullptr || stream_bytes == nullptr ||
      tau_out == nullptr || dev_stream == nullptr || reinterpret_cast<uintptr_t>(dev_stream) % 8)
    return MGARD_ERR_ARG;
  if (!(rel_bound > 0.0) || !std::isfinite(rel_bound)) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, dev_data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (dev_labels == nullptr || reinterpret_cast<uintptr_t>(dev_labels) % 8) return MGARD_ERR_ARG;
  const int64_t count = p->h.count();
  size_t bound = 0;
  mgard_pack_bound(count, &bound);
  if (dev_capacity < bound) return MGARD_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = static_cast<size_t>(count) * elem_size(dtype);
  MGB_TRY(cudaMemcpyAsync(dev_data, host_field, bytes, cudaMemcpyHostToDevice, s));
  double mm[2];
  rc = mgard_value_range(count, dtype, dev_data, mm, stream);
  if (rc != MGARD_OK) return rc;
  double tau = rel_bound * (mm[1] - mm[0]);
  if (!(tau > 0.0)) tau = rel_bound * (std::fabs(mm[0]) > 0.0 ? std::fabs(mm[0]) : 1.0);
  rc = transform(true, ndim, dims, coords, dtype, stop_level, dev_data, workspace, ws_bytes, stream);
  if (rc != MGARD_OK) return rc;
  rc = mgard_quantize(ndim, dims, coords, dtype, stop_level, tau, dev_data, dev_labels, nullptr,
                      stream);
  if (rc != MGARD_OK) return rc;
  rc = lorenzo_device(true, *p, stop_level, dev_labels, s);
  if (rc != MGARD_OK) return rc;
  size_t sb = 0;
  {
    StreamScratch* sc = get_scratch(s);
    if (sc == nullptr) return MGARD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(sc->mu);
    rc = pack_device(count, dev_labels, dev_stream, dev_capacity, &sb, sc, s);
  }
  if (rc != MGARD_OK) return rc;
  if (sb > host_capacity) return MGARD_ERR_WORKSPACE;
  MGB_TRY(cudaMemcpyAsync(host_stream, dev_stream, sb, cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  *stream_bytes = sb;
  *tau_out = tau;
  return MGARD_OK;
}

int mgard_decompress_host_packed(int ndim, const int64_t* dims, const double* const* coords,
                                 int dtype, int stop_level, double tau_linf,
                                 const void* host_stream, size_t stream_bytes, void* host_field,
                                 void* dev_data, int64_t* dev_labels, void* dev_stream,
                                 size_t dev_capacity, void* workspace, size_t ws_bytes,
                                 void* stream) {
  if (host_field == nullptr || host_stream == nullptr || dev_stream == nullptr ||
      reinterpret_cast<uintptr_t>(dev_stream) % 8 || stream_bytes > dev_capacity)
    return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, dev_data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (dev_labels == nullptr || reinterpret_cast<uintptr_t>(dev_labels) % 8) return MGARD_ERR_ARG;
  const int64_t count = p->h.count();
  rc = check_stream(static_cast<const uint8_t*>(host_stream), stream_bytes, count);
  if (rc != MGARD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MGB_TRY(cudaMemcpyAsync(dev_stream, host_stream, stream_bytes, cudaMemcpyHostToDevice, s));
  rc = unpack_device(dev_stream, count, dev_labels, s);
  if (rc != MGARD_OK) return rc;
  rc = lorenzo_device(false, *p, stop_level, dev_labels, s);
  if (rc != MGARD_OK) return rc;
  rc = mgard_dequantize(ndim, dims, coords, dtype, stop_level, tau_linf, dev_labels, dev_data, stream);
  if (rc != MGARD_OK) return rc;
  rc = transform(false, ndim, dims, coords, dtype, stop_level, dev_data, workspace, ws_bytes, stream);
  if (rc != MGARD_OK) return rc;
  MGB_TRY(cudaMemcpyAsync(host_field, dev_data, static_cast<size_t>(count) * elem_size(dtype),
                          cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  return MGARD_OK;
}

int mgard_decompose_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, const void* host_in, void* host_out, void* dev_data,
                         void* workspace, size_t ws_bytes, void* stream) {
  return transform_host(true, ndim, dims, coords, dtype, stop_level, host_in, host_out, dev_data,
                        workspace, ws_bytes, stream);
}

int mgard_recompose_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, const void* host_in, void* host_out, void* dev_data,
                         void* workspace, size_t ws_bytes, void* stream) {
  return transform_host(false, ndim, dims, coords, dtype, stop_level, host_in, host_out, dev_data,
                        workspace, ws_bytes, stream);
}

namespace {

int quantize_table(const DevPlan& p, int dtype, int stop_level, const LevelTable& tab,
                   const void* coeffs, int64_t* labels, void* stream) {
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);
  if (sc == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sc->mu);
  MGB_TRY(cudaMemsetAsync(sc->flag, 0, sizeof(unsigned), s));
  const auto& d = p.h.dims3;
  if (dtype == MGARD_F64)
    MGB_TRY(launch_quantize<double>(static_cast<const double*>(coeffs), labels, p.lev01, p.lev[2],
                                    d[0] * d[1], d[2], stop_level, tab, sc->flag, s));
  else
    MGB_TRY(launch_quantize<float>(static_cast<const float*>(coeffs), labels, p.lev01, p.lev[2],
                                   d[0] * d[1], d[2], stop_level, tab, sc->flag, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_flags, sc->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_flags + 1, c->flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  if (sc->h_flags[1]) {
    MGB_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(unsigned), s));
    return MGARD_ERR_TIMEOUT;
  }
  const unsigned f = sc->h_flags[0];
  if (f & 1u) return MGARD_ERR_NONFINITE;
  if (f & 2u) return MGARD_ERR_OVERFLOW;
  return MGARD_OK;
}

int dequantize_table(const DevPlan& p, int dtype, int stop_level, const LevelTable& tab,
                     const int64_t* labels, void* coeffs, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto& d = p.h.dims3;
  if (dtype == MGARD_F64)
    return cuda_rc(launch_dequantize<double>(labels, static_cast<double*>(coeffs), p.lev01,
                                             p.lev[2], d[0] * d[1], d[2], stop_level, tab, s));
  return cuda_rc(launch_dequantize<float>(labels, static_cast<float*>(coeffs), p.lev01, p.lev[2],
                                          d[0] * d[1], d[2], stop_level, tab, s));
}

int check_q_args(int dtype, const void* coeffs, const int64_t* labels) {
  if (coeffs == nullptr || labels == nullptr) return MGARD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(coeffs) % elem_size(dtype) || reinterpret_cast<uintptr_t>(labels) % 8)
    return MGARD_ERR_ARG;
  return MGARD_OK;
}

}  // namespace

int mgard_quantize(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                   int stop_level, double tau_linf, const void* coeffs, int64_t* labels,
                   double* tau_levels_out, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  LevelTable tab;
  rc = make_table(*p, stop_level, tau_linf, tab, tau_levels_out);
  if (rc != MGARD_OK) return rc;
  return quantize_table(*p, dtype, stop_level, tab, coeffs, labels, stream);
}

int mgard_quantize_async(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, double tau_linf, const void* coeffs, int64_t* labels,
                         double* tau_levels_out, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  LevelTable tab;
  rc = make_table(*p, stop_level, tau_linf, tab, tau_levels_out);
  if (rc != MGARD_OK) return rc;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int* flags = c->flags + 2;  // gathered until mgard_quantize_status
  const auto& d = p->h.dims3;
  if (dtype == MGARD_F64)
    MGB_TRY(launch_quantize<double>(static_cast<const double*>(coeffs), labels, p->lev01,
                                    p->lev[2], d[0] * d[1], d[2], stop_level, tab, flags, s));
  else
    MGB_TRY(launch_quantize<float>(static_cast<const float*>(coeffs), labels, p->lev01, p->lev[2],
                                   d[0] * d[1], d[2], stop_level, tab, flags, s));
  return MGARD_OK;
}

int mgard_quantize_status(void* stream) {
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);
  if (sc == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sc->mu);
  MGB_TRY(cudaMemcpyAsync(sc->h_flags, c->flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  const unsigned f = sc->h_flags[2], t = sc->h_flags[1];
  if (f) MGB_TRY(cudaMemsetAsync(c->flags + 2, 0, sizeof(unsigned), s));
  if (t) {
    MGB_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(unsigned), s));
    return MGARD_ERR_TIMEOUT;
  }
  if (f & 1u) return MGARD_ERR_NONFINITE;
  if (f & 4u) return MGARD_ERR_ARG;
  if (f & 2u) return MGARD_ERR_OVERFLOW;
  return MGARD_OK;
}

int mgard_quantize_levels(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                          int stop_level, const double* tau_levels, const void* coeffs,
                          int64_t* labels, void* stream) {
  if (tau_levels == nullptr) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  LevelTable tab;
  rc = make_table_levels(*p, stop_level, tau_levels, tab, nullptr);
  if (rc != MGARD_OK) return rc;
  return quantize_table(*p, dtype, stop_level, tab, coeffs, labels, stream);
}

int mgard_dequantize_levels(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                            int stop_level, const double* tau_levels, const int64_t* labels,
                            void* coeffs, void* stream) {
  if (tau_levels == nullptr) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  LevelTable tab;
  rc = make_table_levels(*p, stop_level, tau_levels, tab, nullptr);
  if (rc != MGARD_OK) return rc;
  return dequantize_table(*p, dtype, stop_level, tab, labels, coeffs, stream);
}

int mgard_dequantize(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                     int stop_level, double tau_linf, const int64_t* labels, void* coeffs,
                     void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (coeffs == nullptr || labels == nullptr) return MGARD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(coeffs) % elem_size(dtype) || reinterpret_cast<uintptr_t>(labels) % 8)
    return MGARD_ERR_ARG;
  LevelTable tab;
  rc = make_table(*p, stop_level, tau_linf, tab, nullptr);
  if (rc != MGARD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto& d = p->h.dims3;
  if (dtype == MGARD_F64)
    return cuda_rc(launch_dequantize<double>(labels, static_cast<double*>(coeffs), p->lev01,
                                             p->lev[2], d[0] * d[1], d[2], stop_level, tab, s));
  return cuda_rc(launch_dequantize<float>(labels, static_cast<float*>(coeffs), p->lev01, p->lev[2],
                                          d[0] * d[1], d[2], stop_level, tab, s));
}

int mgard_value_range(int64_t count, int dtype, const void* data, double* minmax_out, void* stream) {
  if (count < 1 || data == nullptr || minmax_out == nullptr) return MGARD_ERR_ARG;
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(data) % elem_size(dtype)) return MGARD_ERR_ARG;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);
  if (sc == nullptr) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sc->mu);
  MGB_TRY(cudaMemsetAsync(sc->flag, 0, sizeof(unsigned), s));
  if (dtype == MGARD_F64)
    MGB_TRY(launch_minmax<double>(static_cast<const double*>(data), count, sc->partial, sc->flag, sc->result, s));
  else
    MGB_TRY(launch_minmax<float>(static_cast<const float*>(data), count, sc->partial, sc->flag, sc->result, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_result, sc->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_flags, sc->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaMemcpyAsync(sc->h_flags + 1, c->flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  if (sc->h_flags[1]) {
    MGB_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(unsigned), s));
    return MGARD_ERR_TIMEOUT;
  }
  if (sc->h_flags[0] & 1u) return MGARD_ERR_NONFINITE;
  minmax_out[0] = sc->h_result[0];
  minmax_out[1] = sc->h_result[1];
  return MGARD_OK;
}

int mgard_value_range_async(int64_t count, int dtype, const void* data, double* range,
                            void* stream) {
  if (count < 1 || data == nullptr || range == nullptr) return MGARD_ERR_ARG;
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(data) % elem_size(dtype)) return MGARD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(range) % sizeof(double)) return MGARD_ERR_ARG;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StreamScratch* sc = get_scratch(s);  // its partial sums: ordered by the stream
  if (sc == nullptr) return MGARD_ERR_CUDA;
  unsigned int* flags = c->flags + 2;  // gathered until mgard_quantize_status
  if (dtype == MGARD_F64)
    MGB_TRY(launch_minmax<double>(static_cast<const double*>(data), count, sc->partial, flags, range, s));
  else
    MGB_TRY(launch_minmax<float>(static_cast<const float*>(data), count, sc->partial, flags, range, s));
  return MGARD_OK;
}

namespace {
// The device-range form of the level tolerances for a plan and stopping level.
int rel_tol(const DevPlan& p, int stop_level, double rel_bound, const double* range,
            unsigned int* flags, RelTol& rt) {
  if (stop_level < 0 || stop_level > p.h.L) return MGARD_ERR_LEVEL;
  if (!(rel_bound > 0.0) || !std::isfinite(rel_bound)) return MGARD_ERR_ARG;
  if (range == nullptr || reinterpret_cast<uintptr_t>(range) % sizeof(double)) return MGARD_ERR_ARG;
  rt = RelTol{};
  rt.range = range;
  rt.rel = rel_bound;
  rt.L = p.h.L;
  rt.stop = stop_level;
  rt.flags = flags;
  level_tolerance_terms(p.h, stop_level, &rt.C, &rt.kappa, &rt.kpow);
  return MGARD_OK;
}
}  // namespace

int mgard_quantize_rel_async(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                             int stop_level, double rel_bound, const double* range,
                             const void* coeffs, int64_t* labels, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  RelTol rt;
  rc = rel_tol(*p, stop_level, rel_bound, range, c->flags + 2, rt);
  if (rc != MGARD_OK) return rc;
  const LevelTable tab{};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto& d = p->h.dims3;
  if (dtype == MGARD_F64)
    MGB_TRY(launch_quantize<double>(static_cast<const double*>(coeffs), labels, p->lev01,
                                    p->lev[2], d[0] * d[1], d[2], stop_level, tab, c->flags + 2, s,
                                    &rt));
  else
    MGB_TRY(launch_quantize<float>(static_cast<const float*>(coeffs), labels, p->lev01, p->lev[2],
                                   d[0] * d[1], d[2], stop_level, tab, c->flags + 2, s, &rt));
  return MGARD_OK;
}

int mgard_dequantize_rel(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, double rel_bound, const double* range,
                         const int64_t* labels, void* coeffs, void* stream) {
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_q_args(dtype, coeffs, labels);
  if (rc != MGARD_OK) return rc;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  RelTol rt;
  rc = rel_tol(*p, stop_level, rel_bound, range, c->flags + 2, rt);
  if (rc != MGARD_OK) return rc;
  const LevelTable tab{};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto& d = p->h.dims3;
  if (dtype == MGARD_F64)
    return cuda_rc(launch_dequantize<double>(labels, static_cast<double*>(coeffs), p->lev01,
                                             p->lev[2], d[0] * d[1], d[2], stop_level, tab, s,
                                             &rt));
  return cuda_rc(launch_dequantize<float>(labels, static_cast<float*>(coeffs), p->lev01, p->lev[2],
                                          d[0] * d[1], d[2], stop_level, tab, s, &rt));
}

int mgard_compress_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                        int stop_level, double rel_bound, const void* host_field,
                        int64_t* host_labels, double* tau_out, void* dev_data, int64_t* dev_labels,
                        void* workspace, size_t ws_bytes, void* stream) {
  if (host_field == nullptr || host_labels == nullptr || tau_out == nullptr) return MGARD_ERR_ARG;
  if (!(rel_bound > 0.0) || !std::isfinite(rel_bound)) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, dev_data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (dev_labels == nullptr || reinterpret_cast<uintptr_t>(dev_labels) % 8) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t count = p->h.count();
  const size_t bytes = static_cast<size_t>(count) * elem_size(dtype);
  MGB_TRY(cudaMemcpyAsync(dev_data, host_field, bytes, cudaMemcpyHostToDevice, s));
  double mm[2];
  rc = mgard_value_range(count, dtype, dev_data, mm, stream);
  if (rc != MGARD_OK) return rc;
  double tau = rel_bound * (mm[1] - mm[0]);
  if (!(tau > 0.0)) tau = rel_bound * (std::fabs(mm[0]) > 0.0 ? std::fabs(mm[0]) : 1.0);
  rc = transform(true, ndim, dims, coords, dtype, stop_level, dev_data, workspace, ws_bytes, stream);
  if (rc != MGARD_OK) return rc;
  rc = mgard_quantize(ndim, dims, coords, dtype, stop_level, tau, dev_data, dev_labels, nullptr,
                      stream);
  if (rc != MGARD_OK) return rc;
  MGB_TRY(cudaMemcpyAsync(host_labels, dev_labels, static_cast<size_t>(count) * 8,
                          cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  *tau_out = tau;
  return MGARD_OK;
}

int mgard_decompress_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                          int stop_level, double tau_linf, const int64_t* host_labels,
                          void* host_field, void* dev_data, int64_t* dev_labels, void* workspace,
                          size_t ws_bytes, void* stream) {
  if (host_field == nullptr || host_labels == nullptr) return MGARD_ERR_ARG;
  DevPlan* p = nullptr;
  int rc = get_plan(ndim, dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  rc = check_transform_args(*p, stop_level, dev_data, workspace, ws_bytes);
  if (rc != MGARD_OK) return rc;
  if (dev_labels == nullptr || reinterpret_cast<uintptr_t>(dev_labels) % 8) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t count = p->h.count();
  MGB_TRY(cudaMemcpyAsync(dev_labels, host_labels, static_cast<size_t>(count) * 8,
                          cudaMemcpyHostToDevice, s));
  rc = mgard_dequantize(ndim, dims, coords, dtype, stop_level, tau_linf, dev_labels, dev_data, stream);
  if (rc != MGARD_OK) return rc;
  rc = transform(false, ndim, dims, coords, dtype, stop_level, dev_data, workspace, ws_bytes, stream);
  if (rc != MGARD_OK) return rc;
  MGB_TRY(cudaMemcpyAsync(host_field, dev_data, static_cast<size_t>(count) * elem_size(dtype),
                          cudaMemcpyDeviceToHost, s));
  MGB_TRY(cudaStreamSynchronize(s));
  return MGARD_OK;
}

int mgard_release_plans(void) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGARD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (it->second->device == device) it = g_plans.erase(it);
    else ++it;
  }
  release_plans4(device);
  return MGARD_OK;
}

const char* mgard_error_string(int code) {
  switch (code) {
    case MGARD_OK: return "ok";
    case MGARD_ERR_ARG: return "invalid argument (null or misaligned pointer, bad dtype, tau <= 0)";
    case MGARD_ERR_SHAPE:
      return "invalid shape (ndim, or an axis length or node count outside the call's limits)";
    case MGARD_ERR_COORDS: return "coordinates must be finite and strictly increasing";
    case MGARD_ERR_LEVEL: return "stop level outside [0, L]";
    case MGARD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case MGARD_ERR_OVERFLOW: return "a quantization label would exceed 2^62 in magnitude";
    case MGARD_ERR_NONFINITE: return "input contains NaN or Inf";
    case MGARD_ERR_CUDA: return "CUDA runtime error";
    case MGARD_ERR_TIMEOUT: return "bounded device-side wait timed out";
    default: return "unknown error code";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free decomposition.  The paper has no counterpart: this is an
// interface for callers that must not allocate device memory while they
// compress, e.g. an in-situ simulation that has reserved nearly all of HBM
// for its own state (a cudaMalloc could fail there, and it may also wait for
// work in flight on other streams).  The workspace and the plan tables live
// in one file-scope __device__ array of kNoAllocBytes; no cudaMalloc,
// cudaFree, pinned-host allocation or allocating library is called.
// ---------------------------------------------------------------------------
namespace mgb {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB per device
// Layout: [0, 256) status word (wait timeouts; set to zero at each call),
// then the plan tables, then the level workspace.  Nothing else needs to
// start at zero: the workspace is fully written before it is read.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocState {
  char* base = nullptr;   // device address of g_noalloc_scratch on this device
  std::string key;        // plan whose tables are resident, empty if none
  DevPlan plan;           // table pointers into the scratch (dmem stays null)
  size_t ws_off = 0;      // workspace offset in the scratch
};
std::mutex g_noalloc_mu;
std::map<int, std::unique_ptr<NoAllocState>> g_noalloc;

// Stage the plan tables of `p.h` into host memory with the offsets that
// fill_levels expects, then copy them to `dst` (device) on `s`.
template <typename T>
int noalloc_tables(DevPlan& p, char* dst, size_t cap, size_t* used, cudaStream_t s) {
  const HostPlan& h = p.h;
  std::vector<std::vector<size_t>> offs((h.L + 1) * 3);
  size_t total = 0;
  auto reserve = [&](size_t bytes) { const size_t o = total; total = align_up(total + bytes, 16); return o; };
  for (int l = 1; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      const AxisTables& t = h.ax[l][a];
      auto& o = offs[l * 3 + a];
      for (const auto* v : {&t.iwl, &t.iwr, &t.rw, &t.ta, &t.tm, &t.tc, &t.xd, &t.xr, &t.sb, &t.sg,
                            &t.sy, &t.sh})
        o.push_back(reserve(sizeof(T) * v->size()));
    }
  size_t lev_off[3];
  for (int a = 0; a < 3; ++a) lev_off[a] = reserve(h.lev[a].size());
  const size_t lev01_off = reserve(h.lev01.size());
  std::vector<std::array<size_t, 3>> pos_off(h.L + 1);
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) pos_off[l][a] = reserve(sizeof(int32_t) * h.idx[l][a].size());
  size_t x_off[3];
  for (int a = 0; a < 3; ++a) x_off[a] = reserve(sizeof(double) * h.x[a].size());
  total = align_up(total, kAlign);
  if (total > cap) return MGARD_ERR_WORKSPACE;
  std::vector<char> stage(total, 0);
  auto put = [&](size_t off, const std::vector<double>& v) {
    T* d = reinterpret_cast<T*>(stage.data() + off);
    for (size_t i = 0; i < v.size(); ++i) d[i] = static_cast<T>(v[i]);
  };
  for (int l = 1; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      const AxisTables& t = h.ax[l][a];
      const auto& o = offs[l * 3 + a];
      int i = 0;
      for (const auto* v : {&t.iwl, &t.iwr, &t.rw, &t.ta, &t.tm, &t.tc, &t.xd, &t.xr, &t.sb, &t.sg,
                            &t.sy, &t.sh})
        put(o[i++], *v);
    }
  for (int a = 0; a < 3; ++a) std::memcpy(stage.data() + lev_off[a], h.lev[a].data(), h.lev[a].size());
  std::memcpy(stage.data() + lev01_off, h.lev01.data(), h.lev01.size());
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) {
      int32_t* dst = reinterpret_cast<int32_t*>(stage.data() + pos_off[l][a]);
      for (size_t j = 0; j < h.idx[l][a].size(); ++j) dst[j] = static_cast<int32_t>(h.idx[l][a][j]);
    }
  for (int a = 0; a < 3; ++a)
    std::memcpy(stage.data() + x_off[a], h.x[a].data(), sizeof(double) * h.x[a].size());
  // Pageable source: the copy has consumed `stage` when the call returns.
  if (cudaMemcpyAsync(dst, stage.data(), total, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MGARD_ERR_CUDA;
  if constexpr (sizeof(T) == 4) fill_levels<float>(p, offs, dst, p.lvf);
  else fill_levels<double>(p, offs, dst, p.lvd);
  for (int a = 0; a < 3; ++a) p.lev[a] = reinterpret_cast<const uint8_t*>(dst + lev_off[a]);
  p.lev01 = reinterpret_cast<const uint8_t*>(dst + lev01_off);
  // Node positions and coordinates complete the plan as upload() does.
  p.pos.assign(h.L + 1, {});
  for (int l = 0; l <= h.L; ++l)
    for (int a = 0; a < 3; ++a) p.pos[l][a] = reinterpret_cast<const int32_t*>(dst + pos_off[l][a]);
  for (int a = 0; a < 3; ++a) p.xc[a] = reinterpret_cast<const double*>(dst + x_off[a]);
  *used = total;
  return MGARD_OK;
}

}  // namespace
}  // namespace mgb

extern "C" int mgard_decompose_noalloc(int ndim, const int64_t* dims, const double* const* coords,
                                       int dtype, int stop_level, void* data, int* timed_out,
                                       void* stream) {
  using namespace mgb;
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  int rc = check_shape(ndim, dims);
  if (rc != MGARD_OK) return rc;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostPlan probe;
  probe.ndim = ndim;
  const int pad = 3 - ndim;
  for (int d = 0; d < ndim; ++d) probe.dims3[pad + d] = dims[d];
  for (int d = 0; d < ndim; ++d) {
    const double* c = coords ? coords[d] : nullptr;
    if (c) probe.coords_key.insert(probe.coords_key.end(), c, c + dims[d]);
    probe.coords_key.push_back(c ? 1.0 : 0.0);
  }
  const std::string key = plan_key(device, dtype, probe);

  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto& slot = g_noalloc[device];
  if (!slot) {
    // Set-up once per device: the device address of the scratch array.
    auto st = std::make_unique<NoAllocState>();
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr)
      return MGARD_ERR_CUDA;
    st->base = static_cast<char*>(addr);
    slot = std::move(st);
  }
  NoAllocState& st = *slot;
  if (st.key != key) {
    // A new plan: build the host tables, check that tables and workspace fit,
    // then copy the tables in.
    HostPlan h;
    rc = build_host_plan(ndim, dims, coords, h);
    if (rc != MGARD_OK) return rc;
    st.key.clear();
    st.plan.h = std::move(h);
    st.plan.dtype = dtype;
    st.plan.device = device;
    layout_workspace(st.plan);
    const size_t avail = kNoAllocBytes - kAlign;
    if (st.plan.ws_bytes > avail) return MGARD_ERR_WORKSPACE;
    size_t used = 0;
    char* tables = st.base + kAlign;
    // The tables are copied only when tables and workspace both fit.
    rc = (dtype == MGARD_F64)
             ? noalloc_tables<double>(st.plan, tables, avail - st.plan.ws_bytes, &used, s)
             : noalloc_tables<float>(st.plan, tables, avail - st.plan.ws_bytes, &used, s);
    if (rc != MGARD_OK) return rc;
    st.ws_off = kAlign + used;
    st.key = key;
  }
  char* ws = st.base + st.ws_off;
  rc = check_transform_args(st.plan, stop_level, data, ws, kNoAllocBytes - st.ws_off);
  if (rc != MGARD_OK) return rc;
  if (timed_out) *timed_out = 0;
  if (stop_level == st.plan.h.L) return MGARD_OK;
  unsigned int* status = reinterpret_cast<unsigned int*>(st.base);
  if (cudaMemsetAsync(status, 0, sizeof(unsigned int), s) != cudaSuccess) return MGARD_ERR_CUDA;
  rc = (dtype == MGARD_F64)
           ? run_decompose<double>(st.plan, stop_level, static_cast<double*>(data), ws, status, s)
           : run_decompose<float>(st.plan, stop_level, static_cast<float*>(data), ws, status, s);
  if (rc != MGARD_OK || timed_out == nullptr) return rc;
  unsigned int word = 0;
  if (cudaMemcpyAsync(&word, status, sizeof word, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MGARD_ERR_CUDA;
  *timed_out = word != 0;
  return word != 0 ? MGARD_ERR_TIMEOUT : MGARD_OK;
}
