// Batched form: the decomposition or recomposition of many 3D FP32 fields of
// uneven shape in ONE persistent kernel launch, replayed as a CUDA graph.
//
// Work model.  Every field's transform is a chain of stages, exactly the
// kernels of the per-field path (Section 2 level loop): per level, the load
// vector, the axis-2, axis-1 and axis-0 solves (the last applying the
// correction), and the finish passes coarsest first.  A stage is split into
// tiles, the CTA work units of those kernels.  The host lists all tiles of
// all fields, stage by stage across the fields (longest fields first), and
// the persistent CTAs take them in that order through an atomic counter.
// Before a tile runs, its CTA waits until every tile of the field's previous
// stage is done (a per-stage counter, acquire load, bounded wait); when a
// tile ends its CTA releases it (fence, then increment).  A tile is only
// taken after every tile listed before it was taken by a running CTA, so the
// waits always end.  A wait that passes 2 s records a timeout in the
// per-device status word (reported as MGARD_ERR_TIMEOUT by the next
// quantize or value-range call) and ends the CTA.
//
// Tile shapes (coarse planes per load-vector tile, plane pairs per finish
// tile, lines per contiguous-solve tile, line groups per segmented-solve
// tile) are parameters of the plan, chosen by the autotuner of
// mgard_batch_autotune.  Segmented solves of short lines put several
// 32-line groups side by side in one CTA; the finish tiles use a 4-stage
// ring.  Per tile kind, the kernel counts tiles, cycles spent before a tile
// starts and cycles running tiles (mgard_batch_stats).
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "devplan.hpp"
#include "finish_tile.cuh"
#include "kernels.cuh"
#include "lv_tile.cuh"
#include "mgard_gb.h"
#include "pdl.cuh"
#include "solve_tile.cuh"
#include "tma.cuh"

namespace mgb {
namespace {

enum BatchKind : int {
  kBLoadVecDec = 0,
  kBLoadVecRec,
  kBSolveContigTma,
  kBSolveContig,
  kBSolveSeg,
  kBFinish,
  kBKinds
};

// One stage of one field (device side).
struct BatchStage {
  int kind;
  int ntiles;
  int mode;          // apply mode of a solve
  int rows;          // lines per contiguous-solve tile
  int groups;        // 32-line groups per segmented-solve tile (a multiple of gpp)
  int gpp;           // groups solved side by side per pass
  int64_t nlines;    // lines of a solve
  int64_t S;         // stride of a segmented solve
  int64_t block_stride;
  uint64_t fine_count;
  float sign;        // finish: -1 decomposition, +1 recomposition
  int axis;          // solved axis
  MarchGeom mg;
  FinishGeom fg;
  float* fine;
  float* coarse;
  float* F;
  float* B;
  const float* nodal_src;
  const float* interp_src;
  LevelK<float> lv;
};

constexpr int kBatchThreads = 288;
constexpr int kLvNS = 4, kLvT1 = 4;  // the batched tiles keep their own shape
constexpr int kLvGMax = 8;           // row groups of a load-vector tile (narrow fields)
constexpr int kFinNS = 4, kFinT1 = 4;  // as the load-vector tiles, a shape of their own
constexpr int kFinGMax = 8;          // row groups of a finish tile (narrow fields)

__global__ void __launch_bounds__(kBatchThreads, 2)
batch_kernel(const BatchStage* __restrict__ stages, const int4* __restrict__ items, int nitems,
             unsigned int* __restrict__ head, unsigned int* __restrict__ done,
             unsigned int* __restrict__ status, unsigned long long* __restrict__ stats,
             unsigned long long wait_limit_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_abort;
  __shared__ __align__(16) BatchStage st;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      s_item = static_cast<int>(atomicAdd(head, 1u));
      s_abort = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 item = items[it];  // x: stage, y: tile, z: stage it waits for, w: its tiles
    const long long c_wait = clock64();
    if (tid == 0 && item.z >= 0) {
      const uint64_t t0 = global_ns();
      while (ld_acquire_gpu(done + item.z) < static_cast<unsigned>(item.w)) {
        __nanosleep(256);
        if (global_ns() - t0 > wait_limit_ns) {
          *reinterpret_cast<volatile unsigned*>(status) = 2u;
          s_abort = 1;
          break;
        }
      }
      fence_proxy_async_global();  // the tile's bulk copies read what it acquired
    }
    {
      const int* src = reinterpret_cast<const int*>(stages + item.x);
      int* dst = reinterpret_cast<int*>(&st);
      for (int i = tid; i < static_cast<int>(sizeof(BatchStage) / sizeof(int)); i += blockDim.x)
        dst[i] = src[i];
    }
    __syncthreads();
    if (s_abort) break;
    const long long c_run = clock64();
    switch (st.kind) {
      case kBLoadVecDec:
        load_vector_march_tile<float, true, kLvNS, kLvT1, true, true, 1, kLvGMax>(st.lv, st.fine, st.coarse, st.F,
                                                                st.mg, st.fine_count, status,
                                                                item.y, smem_raw);
        break;
      case kBLoadVecRec:
        load_vector_march_tile<float, false, kLvNS, kLvT1, true, true, 1, kLvGMax>(st.lv, st.fine, st.coarse, st.F,
                                                                 st.mg, st.fine_count, status,
                                                                 item.y, smem_raw);
        break;
      case kBSolveContigTma:
        solve_contig_tma_tile<float, true>(st.lv.ax[2], st.F, st.B, st.nlines, st.rows, st.mode, status,
                                     item.y, smem_raw);
        break;
      case kBSolveContig:
        solve_contig_tile<float>(st.lv.ax[2], st.F, st.B, st.nlines, st.rows, st.mode, item.y,
                                 smem_raw);
        break;
      case kBSolveSeg: {
        // st.gpp groups of 32 lines side by side per pass, st.groups per tile.
        const int passes = st.groups / st.gpp;
        for (int q = 0; q < passes; ++q) {
          const int64_t t = static_cast<int64_t>(item.y) * passes + q;
          if (t * st.gpp * 32 >= st.nlines) break;
          if (q > 0) __syncthreads();  // the previous pass's reads of shared memory are done
          solve_seg_tile<float, true>(st.lv.ax[st.axis], st.F, st.B, st.nlines, st.S, st.block_stride,
                                st.mode, static_cast<int>(t), smem_raw, st.gpp);
        }
        break;
      }
      default:
        finish_march_tile<float, kFinNS, kFinT1, true, kFinGMax>(st.lv, st.nodal_src, st.interp_src, st.sign,
                                                 st.fine, st.fg, status, item.y, smem_raw);
        break;
    }
    __syncthreads();
    if (tid == 0) {
      // Per kind: tiles, cycles waiting (dependency + descriptor), cycles running.
      const long long c_end = clock64();
      atomicAdd(stats + 3 * st.kind, 1ull);
      atomicAdd(stats + 3 * st.kind + 1, static_cast<unsigned long long>(c_run - c_wait));
      atomicAdd(stats + 3 * st.kind + 2, static_cast<unsigned long long>(c_end - c_run));
      __threadfence();
      atomicAdd(done + item.x, 1u);
      if (*reinterpret_cast<volatile unsigned*>(status) != 0u) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) break;
  }
}

// ------------------------------------------------------------- host side

struct Tuning {
  int lv_t0 = 16;      // coarse planes per load-vector tile
  int fin_t0 = 8;      // plane pairs per finish tile
  int rows = 128;      // lines per contiguous-solve tile
  int groups = 4;      // 32-line groups per segmented-solve tile
};

struct BatchPlan {
  int device = 0;
  int nstages = 0, nitems = 0;
  size_t smem = 0;
  int grid = 0;
  void* dmem = nullptr;                 // stages, items, counters
  BatchStage* d_stages = nullptr;
  int4* d_items = nullptr;
  unsigned int* d_counters = nullptr;   // [0] head, [1 + s] done of stage s
  unsigned long long* d_stats = nullptr;  // [3 * kinds] tiles, wait cycles, run cycles
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dmem) cudaFree(dmem);
  }
};

std::mutex g_bmu;
BatchPlan* g_last = nullptr;  // the plan launched last (for mgard_batch_stats)
std::map<std::string, std::unique_ptr<BatchPlan>> g_bplans;
std::map<std::string, Tuning> g_tuned;  // by shape list

constexpr size_t kWsAlign = 256;
inline size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

std::string shapes_key(int n, const int64_t* dims3) {
  return std::string(reinterpret_cast<const char*>(dims3), sizeof(int64_t) * 3 * n);
}

// Per-field plans (the shared plan cache) and workspace offsets.
int field_plans(int n, const int64_t* dims3, std::vector<DevPlan*>& plans,
                std::vector<size_t>& ws_off, size_t* total) {
  plans.assign(n, nullptr);
  ws_off.assign(n, 0);
  size_t off = 0;
  for (int f = 0; f < n; ++f) {
    const int rc = get_plan(3, dims3 + 3 * f, nullptr, MGARD_F32, &plans[f]);
    if (rc != MGARD_OK) return rc;
    ws_off[f] = off;
    off = up(off + plans[f]->ws_bytes, kWsAlign);
  }
  *total = off;
  return MGARD_OK;
}

size_t lv_smem(const MarchGeom& g) { return sizeof(float) * static_cast<size_t>(kLvNS) * g.BUF; }
size_t fin_smem(const FinishGeom& g, bool sep) {
  return sizeof(float) * (2 * kFinNS * static_cast<size_t>(g.FBUF) +
                          (sep ? 2 : 1) * (kFinNS + 1) * static_cast<size_t>(g.CBUF));
}

// Stages of one field for decomposition (dir 0) or recomposition (dir 1).
int field_stages(const DevPlan& p, float* data, char* ws, int dir, const Tuning& tu,
                 std::vector<BatchStage>& out, size_t* smem) {
  const int L = p.h.L;
  std::vector<float*> B(L + 1), F(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) {
    B[l] = reinterpret_cast<float*>(ws + p.offB[l]);
    F[l] = reinterpret_cast<float*>(ws + p.offF[l]);
  }
  auto base = [&](int kind, int l) {
    BatchStage s;
    std::memset(&s, 0, sizeof s);
    s.kind = kind;
    s.lv = p.lvf[l];
    return s;
  };
  auto lv_stage = [&](int l, bool dec) -> int {
    BatchStage s = base(dec ? kBLoadVecDec : kBLoadVecRec, l);
    // As many row groups as the block holds for this width (one column per
    // thread), no more than the coarse rows need.
    const int gthreads = 32 * ((s.lv.ax[2].nc + 31) / 32);
    const int groups = std::max(1, std::min({kLvGMax, kBatchThreads / gthreads,
                                             (s.lv.ax[1].nc + kLvT1 - 1) / kLvT1}));
    if (!plan_geometry(s.lv, s.mg, 1, kLvT1, kLvNS, groups) || s.mg.threads > kBatchThreads)
      return MGARD_ERR_SHAPE;
    const int c0 = s.lv.ax[0].nc;
    s.mg.t0 = std::max(1, std::min(tu.lv_t0, c0));
    s.mg.nb0 = (c0 + s.mg.t0 - 1) / s.mg.t0;
    s.ntiles = s.mg.nb0 * s.mg.nb1 * s.mg.nb2;
    s.fine = B[l];
    s.coarse = B[l - 1];
    s.F = F[l - 1];
    s.fine_count = uint64_t(s.lv.ax[0].n) * s.lv.ax[1].n * s.lv.ax[2].n;
    *smem = std::max(*smem, lv_smem(s.mg));
    out.push_back(s);
    return MGARD_OK;
  };
  auto solve_stages = [&](int l, int mode) -> int {
    const LevelK<float>& lv = p.lvf[l];
    const int64_t c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
    {  // axis 2, contiguous lines
      const size_t per_row = sizeof(float) * static_cast<size_t>(c2 | 1);
      BatchStage s = base((c2 & 1) ? kBSolveContigTma : kBSolveContig, l);
      s.nlines = c0 * c1;
      s.rows = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(
          std::min<int64_t>(tu.rows, 128), (96 * 1024) / static_cast<int64_t>(per_row))));
      s.ntiles = static_cast<int>((s.nlines + s.rows - 1) / s.rows);
      s.mode = kApplyNone;
      s.axis = 2;
      s.F = F[l - 1];
      s.B = B[l - 1];
      const size_t tpad = (3 * sizeof(float) * static_cast<size_t>(c2) + 15) / 16 * 16;
      *smem = std::max(*smem, (c2 & 1) ? tpad + per_row * s.rows + 32 : per_row * s.rows);
      out.push_back(s);
    }
    for (int a = 1; a >= 0; --a) {  // axes 1 and 0, strided lines
      const AxisK<float>& ax = lv.ax[a];
      const int nseg = (ax.nc + ax.seg_len - 1) / ax.seg_len;
      if (32 * nseg > kBatchThreads) return MGARD_ERR_SHAPE;
      BatchStage s = base(kBSolveSeg, l);
      s.axis = a;
      s.S = (a == 0) ? c1 * c2 : c2;
      s.nlines = (a == 0) ? s.S : c0 * s.S;
      s.block_stride = ax.nc * s.S;
      s.gpp = std::max(1, kBatchThreads / 32 / nseg);
      s.groups = std::max(s.gpp, (std::max(1, tu.groups) + s.gpp - 1) / s.gpp * s.gpp);
      s.ntiles = static_cast<int>((s.nlines + 32 * s.groups - 1) / (32 * s.groups));
      s.mode = (a == 0) ? mode : kApplyNone;
      s.F = F[l - 1];
      s.B = B[l - 1];
      *smem = std::max(*smem, sizeof(float) * (5 * static_cast<size_t>(ax.nc) +
                                               32 * static_cast<size_t>(nseg) * s.gpp));
      out.push_back(s);
    }
    return MGARD_OK;
  };
  auto finish_stage = [&](int l, bool dec) -> int {
    BatchStage s = base(kBFinish, l);
    // As many row groups as the block holds for this width (one fine column
    // per thread), no more than the coarse rows need.
    const int gthreads = 32 * ((s.lv.ax[2].n + 31) / 32);
    const int groups = std::max(1, std::min({kFinGMax, kBatchThreads / gthreads,
                                             (s.lv.ax[1].nc + kFinT1 - 1) / kFinT1}));
    if (!finish_geometry(s.lv, s.fg, groups) || s.fg.threads > kBatchThreads) return MGARD_ERR_SHAPE;
    const int npairs = (s.lv.ax[0].n + 1) / 2;
    s.fg.t0 = std::max(1, std::min(tu.fin_t0, npairs));
    s.fg.nb0 = (npairs + s.fg.t0 - 1) / s.fg.t0;
    s.ntiles = s.fg.nb0 * s.fg.nb1 * s.fg.nb2;
    s.nodal_src = B[l - 1];
    s.interp_src = dec ? F[l - 1] : B[l - 1];
    s.sign = dec ? -1.0f : 1.0f;
    s.fine = B[l];
    *smem = std::max(*smem, fin_smem(s.fg, dec));
    out.push_back(s);
    return MGARD_OK;
  };
  int rc = MGARD_OK;
  if (dir == 0) {
    for (int l = L; l >= 1 && rc == MGARD_OK; --l) {
      rc = lv_stage(l, true);
      if (rc == MGARD_OK) rc = solve_stages(l, kApplyDecompose);
    }
    for (int l = 1; l <= L && rc == MGARD_OK; ++l) rc = finish_stage(l, true);
  } else {
    for (int l = L; l >= 1 && rc == MGARD_OK; --l) rc = lv_stage(l, false);
    for (int l = 1; l <= L && rc == MGARD_OK; ++l) {
      rc = solve_stages(l, kApplyRecompose);
      if (rc == MGARD_OK) rc = finish_stage(l, false);
    }
  }
  return rc;
}

int build_batch(int n, const int64_t* dims3, void* const* data, char* ws, size_t ws_bytes,
                int dir, const Tuning& tu, unsigned int* status, BatchPlan& bp) {
  std::vector<DevPlan*> plans;
  std::vector<size_t> ws_off;
  size_t total = 0;
  int rc = field_plans(n, dims3, plans, ws_off, &total);
  if (rc != MGARD_OK) return rc;
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % kWsAlign != 0 || ws_bytes < total)
    return MGARD_ERR_WORKSPACE;
  std::vector<std::vector<BatchStage>> per(n);
  size_t smem = 0;
  for (int f = 0; f < n; ++f) {
    if (data[f] == nullptr || reinterpret_cast<uintptr_t>(data[f]) % sizeof(float) != 0)
      return MGARD_ERR_ARG;
    rc = field_stages(*plans[f], static_cast<float*>(data[f]), ws + ws_off[f], dir, tu, per[f],
                      &smem);
    if (rc != MGARD_OK) return rc;
  }
  if (smem > 200 * 1024) return MGARD_ERR_SHAPE;
  // Longest fields first; stages listed round by round across the fields.
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int f) {
    return dims3[3 * f] * dims3[3 * f + 1] * dims3[3 * f + 2];
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<BatchStage> stages;
  std::vector<int> first(n, 0);
  for (int f = 0; f < n; ++f) {
    first[f] = static_cast<int>(stages.size());
    stages.insert(stages.end(), per[f].begin(), per[f].end());
  }
  size_t maxst = 0;
  for (int f = 0; f < n; ++f) maxst = std::max(maxst, per[f].size());
  std::vector<int4> items;
  for (size_t k = 0; k < maxst; ++k)
    for (int f : order) {
      if (k >= per[f].size()) continue;
      const int sg = first[f] + static_cast<int>(k);
      const int dep = (k == 0) ? -1 : sg - 1;
      const int dep_tiles = (k == 0) ? 0 : stages[sg - 1].ntiles;
      for (int t = 0; t < stages[sg].ntiles; ++t) items.push_back(make_int4(sg, t, dep, dep_tiles));
    }
  bp.nstages = static_cast<int>(stages.size());
  bp.nitems = static_cast<int>(items.size());
  bp.smem = smem;
  const size_t b_st = up(sizeof(BatchStage) * stages.size(), 256);
  const size_t b_it = up(sizeof(int4) * items.size(), 256);
  const size_t b_ct = up(sizeof(unsigned) * (1 + stages.size()), 256);
  const size_t b_sx = up(sizeof(unsigned long long) * 3 * kBKinds, 256);
  if (cudaMalloc(&bp.dmem, b_st + b_it + b_ct + b_sx) != cudaSuccess) return MGARD_ERR_CUDA;
  char* d = static_cast<char*>(bp.dmem);
  bp.d_stages = reinterpret_cast<BatchStage*>(d);
  bp.d_items = reinterpret_cast<int4*>(d + b_st);
  bp.d_counters = reinterpret_cast<unsigned*>(d + b_st + b_it);
  bp.d_stats = reinterpret_cast<unsigned long long*>(d + b_st + b_it + b_ct);
  if (cudaMemcpy(bp.d_stages, stages.data(), sizeof(BatchStage) * stages.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(bp.d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return MGARD_ERR_CUDA;
  if (allow_dynamic_smem(batch_kernel, smem) != cudaSuccess)
    return MGARD_ERR_CUDA;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBatchThreads, smem);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bp.device);
  bp.grid = std::max(1, per_sm) * sms;
  // The graph: zero the counters, then the persistent launch.
  if (cudaGraphCreate(&bp.graph, 0) != cudaSuccess) return MGARD_ERR_CUDA;
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof mp);
  mp.dst = bp.d_counters;
  mp.elementSize = sizeof(unsigned);
  mp.width = 1 + stages.size();
  mp.height = 1;
  mp.value = 0;
  cudaGraphNode_t n_set = nullptr, n_run = nullptr, n_sx = nullptr;
  if (cudaGraphAddMemsetNode(&n_set, bp.graph, nullptr, 0, &mp) != cudaSuccess) return MGARD_ERR_CUDA;
  mp.dst = bp.d_stats;
  mp.width = 2 * 3 * kBKinds;  // 64-bit words as pairs of 32-bit zeros
  if (cudaGraphAddMemsetNode(&n_sx, bp.graph, &n_set, 1, &mp) != cudaSuccess) return MGARD_ERR_CUDA;
  const BatchStage* a_st = bp.d_stages;
  const int4* a_it = bp.d_items;
  int a_n = bp.nitems;
  unsigned* a_head = bp.d_counters;
  unsigned* a_done = bp.d_counters + 1;
  unsigned* a_status = status;
  unsigned long long* a_stats = bp.d_stats;
  unsigned long long a_wait = kWaitLimitNs;
  void* args[] = {&a_st, &a_it, &a_n, &a_head, &a_done, &a_status, &a_stats, &a_wait};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof kp);
  kp.func = reinterpret_cast<void*>(batch_kernel);
  kp.gridDim = dim3(bp.grid);
  kp.blockDim = dim3(kBatchThreads);
  kp.sharedMemBytes = static_cast<unsigned>(smem);
  kp.kernelParams = args;
  if (cudaGraphAddKernelNode(&n_run, bp.graph, &n_sx, 1, &kp) != cudaSuccess) return MGARD_ERR_CUDA;
  if (cudaGraphInstantiate(&bp.exec, bp.graph, 0) != cudaSuccess) return MGARD_ERR_CUDA;
  return MGARD_OK;
}

int batch_size(int n, const int64_t* dims3) {
  if (n <= 0 || dims3 == nullptr) return MGARD_ERR_ARG;
  for (int f = 0; f < n; ++f) {
    const int rc = check_shape(3, dims3 + 3 * f);
    if (rc != MGARD_OK) return rc;
  }
  return MGARD_OK;
}

int batch_run(int dir, int n, const int64_t* dims3, void* const* data, void* workspace,
              size_t ws_bytes, const Tuning* force, void* stream) {
  int rc = batch_size(n, dims3);
  if (rc != MGARD_OK) return rc;
  if (data == nullptr) return MGARD_ERR_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGARD_ERR_CUDA;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  const std::string shapes = shapes_key(n, dims3);
  std::lock_guard<std::mutex> lk(g_bmu);
  Tuning tu;
  if (force) tu = *force;
  else if (g_tuned.count(shapes)) tu = g_tuned[shapes];
  std::string key = shapes;
  key.append(reinterpret_cast<const char*>(data), sizeof(void*) * n);
  key.append(reinterpret_cast<const char*>(&workspace), sizeof workspace);
  key.append(reinterpret_cast<const char*>(&ws_bytes), sizeof ws_bytes);
  key.append(reinterpret_cast<const char*>(&dir), sizeof dir);
  key.append(reinterpret_cast<const char*>(&device), sizeof device);
  key.append(reinterpret_cast<const char*>(&tu), sizeof tu);
  auto it = g_bplans.find(key);
  if (it == g_bplans.end()) {
    auto bp = std::make_unique<BatchPlan>();
    bp->device = device;
    rc = build_batch(n, dims3, data, static_cast<char*>(workspace), ws_bytes, dir, tu,
                     c->flags + 1, *bp);
    if (rc != MGARD_OK) return rc;
    it = g_bplans.emplace(key, std::move(bp)).first;
  }
  g_last = it->second.get();
  return cudaGraphLaunch(it->second->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MGARD_OK
             : MGARD_ERR_CUDA;
}

}  // namespace
}  // namespace mgb

using namespace mgb;

extern "C" {

int mgard_batch_workspace_size(int nfields, const int64_t* dims3, size_t* bytes) {
  int rc = batch_size(nfields, dims3);
  if (rc != MGARD_OK) return rc;
  if (bytes == nullptr) return MGARD_ERR_ARG;
  std::vector<DevPlan*> plans;
  std::vector<size_t> off;
  size_t total = 0;
  rc = field_plans(nfields, dims3, plans, off, &total);
  if (rc != MGARD_OK) return rc;
  *bytes = std::max<size_t>(total, kWsAlign);
  return MGARD_OK;
}

int mgard_batch_decompose(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                          size_t ws_bytes, void* stream) {
  return batch_run(0, nfields, dims3, data, workspace, ws_bytes, nullptr, stream);
}

int mgard_batch_recompose(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                          size_t ws_bytes, void* stream) {
  return batch_run(1, nfields, dims3, data, workspace, ws_bytes, nullptr, stream);
}

int mgard_batch_autotune(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                         size_t ws_bytes, void* stream, int* choice_out) {
  int rc = batch_size(nfields, dims3);
  if (rc != MGARD_OK) return rc;
  if (data == nullptr) return MGARD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Keep the fields: every candidate runs decompose + recompose on them.
  std::vector<size_t> bytes(nfields);
  size_t total = 0;
  for (int f = 0; f < nfields; ++f) {
    bytes[f] = sizeof(float) * dims3[3 * f] * dims3[3 * f + 1] * dims3[3 * f + 2];
    total += up(bytes[f], kWsAlign);
  }
  void* save = nullptr;
  if (cudaMalloc(&save, total) != cudaSuccess) return MGARD_ERR_CUDA;
  std::vector<char*> saved(nfields);
  {
    size_t o = 0;
    for (int f = 0; f < nfields; ++f) {
      saved[f] = static_cast<char*>(save) + o;
      o += up(bytes[f], kWsAlign);
      cudaMemcpyAsync(saved[f], data[f], bytes[f], cudaMemcpyDeviceToDevice, s);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Tuning best;
  float best_ms = 1e30f;
  rc = MGARD_OK;
  for (int lv_t0 : {8, 16, 32})
    for (int fin_t0 : {4, 8, 16})
      for (int rows : {64, 128})
        for (int groups : {1, 4, 8}) {
        Tuning tu;
        tu.lv_t0 = lv_t0;
        tu.fin_t0 = fin_t0;
        tu.rows = rows;
        tu.groups = groups;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == MGARD_OK; ++rep) {  // the first run builds the plan
          cudaEventRecord(e0, s);
          rc = batch_run(0, nfields, dims3, data, workspace, ws_bytes, &tu, stream);
          if (rc == MGARD_OK) rc = batch_run(1, nfields, dims3, data, workspace, ws_bytes, &tu, stream);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = MGARD_ERR_CUDA;
          cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rc != MGARD_OK) break;
        if (ms < best_ms) { best_ms = ms; best = tu; }
      }
  for (int f = 0; f < nfields; ++f)
    cudaMemcpyAsync(data[f], saved[f], bytes[f], cudaMemcpyDeviceToDevice, s);
  cudaStreamSynchronize(s);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MGARD_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_bmu);
    g_tuned[shapes_key(nfields, dims3)] = best;
    // Plans of the other candidates are no longer needed.
    for (auto it = g_bplans.begin(); it != g_bplans.end();) {
      Tuning t;
      std::memcpy(&t, it->first.data() + it->first.size() - sizeof(Tuning), sizeof t);
      if (std::memcmp(&t, &best, sizeof t) != 0) it = g_bplans.erase(it);
      else ++it;
    }
  }
  if (choice_out) {
    choice_out[0] = best.lv_t0;
    choice_out[1] = best.fin_t0;
    choice_out[2] = best.rows;
    choice_out[3] = best.groups;
  }
  return MGARD_OK;
}

int mgard_batch_wait_selftest(int64_t limit_ns, void* stream) {
  if (limit_ns <= 0 || limit_ns > 1000000000LL) return MGARD_ERR_ARG;
  DevCtx* c = get_ctx();
  if (c == nullptr) return MGARD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // One stage (never run: the only item aborts in its wait), one item that
  // waits for one finished tile of its own stage, counters and stats at 0.
  const size_t b_st = up(sizeof(BatchStage), 256);
  const size_t b_it = up(sizeof(int4), 256);
  const size_t b_ct = up(2 * sizeof(unsigned), 256);
  const size_t b_sx = up(sizeof(unsigned long long) * 3 * kBKinds, 256);
  void* dmem = nullptr;
  if (cudaMalloc(&dmem, b_st + b_it + b_ct + b_sx) != cudaSuccess) return MGARD_ERR_CUDA;
  char* d = static_cast<char*>(dmem);
  const int4 item = make_int4(0, 0, 0, 1);
  int rc = MGARD_OK;
  if (cudaMemsetAsync(d, 0, b_st + b_it + b_ct + b_sx, s) != cudaSuccess ||
      cudaMemcpyAsync(d + b_st, &item, sizeof item, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    rc = MGARD_ERR_CUDA;
  } else {
    batch_kernel<<<1, kBatchThreads, 0, s>>>(
        reinterpret_cast<const BatchStage*>(d), reinterpret_cast<const int4*>(d + b_st), 1,
        reinterpret_cast<unsigned*>(d + b_st + b_it),
        reinterpret_cast<unsigned*>(d + b_st + b_it) + 1, c->flags + 1,
        reinterpret_cast<unsigned long long*>(d + b_st + b_it + b_ct),
        static_cast<unsigned long long>(limit_ns));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      rc = MGARD_ERR_CUDA;
  }
  cudaFree(dmem);
  return rc;
}

int mgard_batch_release(void) {
  std::lock_guard<std::mutex> lk(g_bmu);
  g_bplans.clear();
  g_last = nullptr;
  return MGARD_OK;
}

int mgard_batch_stats(uint64_t* out, int n) {
  std::lock_guard<std::mutex> lk(g_bmu);
  if (out == nullptr || n < 3 * kBKinds) return MGARD_ERR_ARG;
  if (g_last == nullptr) return MGARD_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return MGARD_ERR_CUDA;
  return cudaMemcpy(out, g_last->d_stats, sizeof(uint64_t) * 3 * kBKinds, cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? MGARD_OK
             : MGARD_ERR_CUDA;
}

}  // extern "C"
