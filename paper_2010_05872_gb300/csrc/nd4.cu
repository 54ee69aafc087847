// Four-dimensional grids (QMCPACK's shape class, Section 6): the same
// multilevel decomposition, recomposition and level-wise quantization on a
// 4D tensor-product grid, built from one-axis passes over the array seen as
// (outer, n, inner) for each axis in turn.  This is the plain form of the
// method (every operator applied axis by axis, the way it factors), not the
// fused 1-3D kernels.
//
// Decomposition of level l (v the level-l grid, n its shape, c the coarse
// shape):
//   v_c   = v at the coarse nodes (gather),
//   Pi    = multilinear interpolant of v_c, expanded one axis at a time,
//   w     = v - Pi (zero at the coarse nodes: the coefficients, Section 2),
//   F     = (R_0 x R_1 x R_2 x R_3) w, one restriction pass per axis (R the
//           rows of P^T M_f, Section 5.2),
//   z     = M_c^{-1} F, a Thomas solve along every axis (Section 5.4),
//   Q_{l-1}u = v_c + z, and v keeps w at its coefficient nodes.
// The coarse values go back into the nodal positions, coarsest first.
// Recomposition inverts it: w from the coefficient nodes, z = M_c^{-1} R w,
// c' = Q_{l-1}u - z, v = Pi(c') + w.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mgard_gb.h"
#include "pdl.cuh"
#include "plan.hpp"

namespace mgb {
namespace {

__device__ __forceinline__ int cpos4(int k, int n) { return min(2 * k, n - 1); }
__device__ __forceinline__ bool coef4(int j, int n) { return (j & 1) && j != n - 1; }

constexpr int kT = 256;

unsigned grid_of(int64_t n) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + kT - 1) / kT)));
}

struct Shape4 {
  int n[4];
  __host__ __device__ int64_t count() const { return int64_t(n[0]) * n[1] * n[2] * n[3]; }
};

__device__ __forceinline__ void unflat(int64_t t, const Shape4& s, int i[4]) {
  i[3] = static_cast<int>(t % s.n[3]);
  t /= s.n[3];
  i[2] = static_cast<int>(t % s.n[2]);
  t /= s.n[2];
  i[1] = static_cast<int>(t % s.n[1]);
  i[0] = static_cast<int>(t / s.n[1]);
}
__device__ __forceinline__ int64_t flat(const int i[4], const Shape4& s) {
  return ((int64_t(i[0]) * s.n[1] + i[1]) * s.n[2] + i[2]) * s.n[3] + i[3];
}

// Coarse grid c <- fine grid f at the coarse nodes (or the reverse).
template <typename T, bool GATHER>
__global__ void __launch_bounds__(kT)
nodal4_kernel(T* __restrict__ f, Shape4 fs, T* __restrict__ c, Shape4 cs) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < cs.count();
       t += int64_t(gridDim.x) * blockDim.x) {
    int k[4], j[4];
    unflat(t, cs, k);
    for (int a = 0; a < 4; ++a) j[a] = cpos4(k[a], fs.n[a]);
    if (GATHER) c[t] = f[flat(j, fs)];
    else f[flat(j, fs)] = c[t];
  }
}

// One axis of the multilinear interpolant: out (the axis fine, n) from in
// (the axis coarse, nc = n / 2 + 1), other axes equal.
template <typename T>
__global__ void __launch_bounds__(kT)
expand_axis_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t outer, int n, int nc,
                   int64_t inner, const T* __restrict__ iwl, const T* __restrict__ iwr) {
  grid_dep_enter();
  const int64_t total = outer * n * inner;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % inner;
    const int j = static_cast<int>((t / inner) % n);
    const int64_t o = t / (inner * n);
    const T* row = in + o * nc * inner + i;
    if (coef4(j, n)) {
      out[t] = iwl[j] * row[int64_t((j - 1) >> 1) * inner] + iwr[j] * row[int64_t((j + 1) >> 1) * inner];
    } else {
      const int k = j == n - 1 ? nc - 1 : (j >> 1);
      out[t] = row[int64_t(k) * inner];
    }
  }
}

// One axis of the restriction: out[.., k, ..] = sum_d rw[5k + d] in[.., cpos(k) + d - 2, ..].
template <typename T>
__global__ void __launch_bounds__(kT)
restrict_axis_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t outer, int n, int nc,
                     int64_t inner, const T* __restrict__ rw) {
  grid_dep_enter();
  const int64_t total = outer * nc * inner;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % inner;
    const int k = static_cast<int>((t / inner) % nc);
    const int64_t o = t / (inner * nc);
    const T* row = in + o * n * inner + i;
    const int c = cpos4(k, n);
    T acc = T(0);
    for (int d = 0; d < 5; ++d) {
      const int j = c + d - 2;
      if (j >= 0 && j < n) acc += rw[5 * k + d] * row[int64_t(j) * inner];
    }
    out[t] = acc;
  }
}

// Thomas solve of M_c along one axis, a thread per line.
template <typename T>
__global__ void __launch_bounds__(kT)
thomas_axis_kernel(T* __restrict__ F, int64_t outer, int nc, int64_t inner, const T* __restrict__ ta,
                   const T* __restrict__ tm, const T* __restrict__ tc) {
  grid_dep_enter();
  const int64_t lines = outer * inner;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < lines;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t % inner, o = t / inner;
    T* l = F + o * nc * inner + i;
    T y = T(0);
    for (int k = 0; k < nc; ++k) {
      y = (l[int64_t(k) * inner] - ta[k] * y) * tm[k];
      l[int64_t(k) * inner] = y;
    }
    T x = T(0);
    for (int k = nc - 1; k >= 0; --k) {
      x = l[int64_t(k) * inner] - tc[k] * x;
      l[int64_t(k) * inner] = x;
    }
  }
}

// out = a + s * b elementwise.
template <typename T>
__global__ void __launch_bounds__(kT)
axpy4_kernel(T* __restrict__ out, const T* __restrict__ a, const T* __restrict__ b, T s, int64_t n) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x)
    out[t] = a[t] + s * b[t];
}

// MODE 0: w = v at the coefficient nodes, 0 at the coarse nodes.
// MODE 1: v = w at the coefficient nodes (v's coarse nodes untouched).
template <typename T, int MODE>
__global__ void __launch_bounds__(kT)
coef4_kernel(T* __restrict__ v, T* __restrict__ w, Shape4 s) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < s.count();
       t += int64_t(gridDim.x) * blockDim.x) {
    int j[4];
    unflat(t, s, j);
    const bool c = coef4(j[0], s.n[0]) || coef4(j[1], s.n[1]) || coef4(j[2], s.n[2]) ||
                   coef4(j[3], s.n[3]);
    if (MODE == 0) w[t] = c ? v[t] : T(0);
    else if (c) v[t] = w[t];
  }
}

// Level-wise quantization / dequantization of a 4D array: the level of a
// node is the largest of its axes' levels, raised to the stopping level;
// label = round(x / q_l) ties away from zero in FP64, value = label q_l.
template <typename T>
__global__ void __launch_bounds__(kT)
quantize4_kernel(const T* __restrict__ x, int64_t* __restrict__ labels, Shape4 s,
                 const uint8_t* __restrict__ l0, const uint8_t* __restrict__ l1,
                 const uint8_t* __restrict__ l2, const uint8_t* __restrict__ l3, int stop,
                 const double* __restrict__ q, unsigned int* __restrict__ flags) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < s.count();
       t += int64_t(gridDim.x) * blockDim.x) {
    int j[4];
    unflat(t, s, j);
    const int lev = max(max(max(int(l0[j[0]]), int(l1[j[1]])), max(int(l2[j[2]]), int(l3[j[3]]))), stop);
    const double v = static_cast<double>(x[t]);
    if (!isfinite(v)) {
      atomicOr(flags, 1u);
      labels[t] = 0;
      continue;
    }
    const double y = v / q[lev];
    if (!(fabs(y) < 4611686018427387904.0)) {  // 2^62
      atomicOr(flags, 2u);
      labels[t] = 0;
      continue;
    }
    const double tr = trunc(y);
    labels[t] = static_cast<int64_t>(tr) + (fabs(y - tr) >= 0.5 ? (y < 0 ? -1 : 1) : 0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kT)
dequantize4_kernel(const int64_t* __restrict__ labels, T* __restrict__ x, Shape4 s,
                   const uint8_t* __restrict__ l0, const uint8_t* __restrict__ l1,
                   const uint8_t* __restrict__ l2, const uint8_t* __restrict__ l3, int stop,
                   const double* __restrict__ q) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < s.count();
       t += int64_t(gridDim.x) * blockDim.x) {
    int j[4];
    unflat(t, s, j);
    const int lev = max(max(max(int(l0[j[0]]), int(l1[j[1]])), max(int(l2[j[2]]), int(l3[j[3]]))), stop);
    x[t] = static_cast<T>(static_cast<double>(labels[t]) * q[lev]);
  }
}

// ------------------------------------------------------------------ plan

struct Ax4 {
  int n = 1, nc = 1;
  size_t off[6];  // iwl, iwr, rw, ta, tm, tc (byte offsets in the table block)
};

struct Plan4 {
  int dtype = MGARD_F32, device = 0, L = 0;
  std::vector<Shape4> shape;            // [L+1]
  std::vector<std::array<Ax4, 4>> ax;   // [L+1], entry l = transition l -> l-1
  std::vector<double> knorm;            // [L+1]
  std::vector<double> hd;               // [L+1] largest hat-integral products (unused here)
  std::array<std::vector<uint8_t>, 4> lev;
  size_t lev_off[4] = {0, 0, 0, 0};
  size_t q_off = 0;                     // kMaxLevels doubles of bin widths (per call)
  void* dmem = nullptr;
  std::vector<size_t> offB;             // compact level grids l < L
  size_t off_buf[4] = {0, 0, 0, 0};     // four scratch arrays of #N_L elements
  size_t ws_bytes = 0;
  ~Plan4() {
    if (dmem) cudaFree(dmem);
  }
  template <typename T>
  const T* tab(int l, int a, int which) const {
    return reinterpret_cast<const T*>(static_cast<const char*>(dmem) + ax[l][a].off[which]);
  }
};

std::mutex g_mu4;
std::map<std::string, std::unique_ptr<Plan4>> g_plans4;

inline size_t up16(size_t v) { return (v + 15) / 16 * 16; }
inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

int count_levels4(const int64_t* dims, int* L) {
  if (dims == nullptr) return MGARD_ERR_ARG;
  int64_t cur[4];
  for (int a = 0; a < 4; ++a) {
    if (dims[a] < 3 || dims[a] > (int64_t(1) << 20)) return MGARD_ERR_SHAPE;
    cur[a] = dims[a];
  }
  if (cur[0] * cur[1] * cur[2] * cur[3] > (int64_t(1) << 40)) return MGARD_ERR_SHAPE;
  int l = 0;
  while (std::min(std::min(cur[0], cur[1]), std::min(cur[2], cur[3])) > 3) {
    for (int a = 0; a < 4; ++a) cur[a] = cur[a] / 2 + 1;
    ++l;
  }
  *L = l;
  return MGARD_OK;
}

// Host tables (FP64), the C_Linf bound per level and the node levels; the
// device block (uploaded unless only the bound is wanted) holds the tables in
// the element type.
template <typename T>
int build_plan4(const int64_t* dims, const double* const* coords, Plan4& p, bool upload) {
  int rc = count_levels4(dims, &p.L);
  if (rc != MGARD_OK) return rc;
  if (p.L + 1 > kMaxLevels) return MGARD_ERR_SHAPE;
  const int L = p.L;
  std::array<std::vector<double>, 4> x;
  std::vector<std::array<std::vector<int64_t>, 4>> idx(L + 1);
  for (int a = 0; a < 4; ++a) {
    const double* c = coords ? coords[a] : nullptr;
    x[a].resize(dims[a]);
    for (int64_t j = 0; j < dims[a]; ++j) {
      x[a][j] = c ? c[j] : double(j);
      if (!std::isfinite(x[a][j]) || (j > 0 && !(x[a][j] > x[a][j - 1]))) return MGARD_ERR_COORDS;
    }
    idx[L][a].resize(dims[a]);
    for (int64_t j = 0; j < dims[a]; ++j) idx[L][a][j] = j;
    for (int l = L; l >= 1; --l) {
      const auto& f = idx[l][a];
      const int64_t n = static_cast<int64_t>(f.size());
      idx[l - 1][a].clear();
      for (int64_t k = 0; k < n / 2 + 1; ++k) idx[l - 1][a].push_back(f[std::min(2 * k, n - 1)]);
    }
  }
  p.shape.resize(L + 1);
  for (int l = 0; l <= L; ++l)
    for (int a = 0; a < 4; ++a) p.shape[l].n[a] = static_cast<int>(idx[l][a].size());
  p.ax.resize(L + 1);
  p.knorm.assign(L + 1, 0.0);
  std::vector<std::array<AxisTables, 4>> host(L + 1);
  size_t total = 0;
  auto reserve = [&](size_t bytes) { const size_t o = total; total = up16(total + bytes); return o; };
  for (int l = 1; l <= L; ++l) {
    for (int a = 0; a < 4; ++a) {
      std::vector<double> xl(idx[l][a].size());
      for (size_t j = 0; j < xl.size(); ++j) xl[j] = x[a][idx[l][a][j]];
      build_axis_tables(xl, host[l][a]);
      const AxisTables& t = host[l][a];
      Ax4& g = p.ax[l][a];
      g.n = t.n;
      g.nc = t.nc;
      g.off[0] = reserve(sizeof(T) * t.iwl.size());
      g.off[1] = reserve(sizeof(T) * t.iwr.size());
      g.off[2] = reserve(sizeof(T) * t.rw.size());
      g.off[3] = reserve(sizeof(T) * t.ta.size());
      g.off[4] = reserve(sizeof(T) * t.tm.size());
      g.off[5] = reserve(sizeof(T) * t.tc.size());
    }
    // C_Linf bound: the telescoping sum over the four axes (as in 1-3D).
    double norm = 0.0;
    for (int d = 0; d < 4; ++d) {
      double term = host[l][d].dmax;
      for (int e = 0; e < d; ++e) term *= host[l][e].smax;
      for (int e = d + 1; e < 4; ++e) term *= host[l][e].rmax;
      norm += term;
    }
    p.knorm[l] = norm;
  }
  for (int a = 0; a < 4; ++a) {
    p.lev[a].assign(dims[a], static_cast<uint8_t>(L));
    for (int l = L - 1; l >= 0; --l)
      for (int64_t j : idx[l][a]) p.lev[a][j] = static_cast<uint8_t>(l);
    p.lev_off[a] = reserve(p.lev[a].size());
  }
  p.q_off = reserve(sizeof(double) * kMaxLevels);
  if (!upload) return MGARD_OK;
  std::vector<char> stage(total, 0);
  auto put = [&](size_t off, const std::vector<double>& v) {
    T* dst = reinterpret_cast<T*>(stage.data() + off);
    for (size_t i = 0; i < v.size(); ++i) dst[i] = static_cast<T>(v[i]);
  };
  for (int l = 1; l <= L; ++l)
    for (int a = 0; a < 4; ++a) {
      const AxisTables& t = host[l][a];
      const Ax4& g = p.ax[l][a];
      put(g.off[0], t.iwl); put(g.off[1], t.iwr); put(g.off[2], t.rw);
      put(g.off[3], t.ta); put(g.off[4], t.tm); put(g.off[5], t.tc);
    }
  for (int a = 0; a < 4; ++a) std::memcpy(stage.data() + p.lev_off[a], p.lev[a].data(), p.lev[a].size());
  if (cudaMalloc(&p.dmem, total) != cudaSuccess) return MGARD_ERR_CUDA;
  if (cudaMemcpy(p.dmem, stage.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) return MGARD_ERR_CUDA;
  // Workspace: compact grids of the levels below L, then four scratch arrays.
  const size_t es = sizeof(T);
  size_t off = 0;
  p.offB.assign(L + 1, 0);
  for (int l = L - 1; l >= 0; --l) {
    p.offB[l] = off;
    off = up256(off + es * static_cast<size_t>(p.shape[l].count()));
  }
  for (int b = 0; b < 4; ++b) {
    p.off_buf[b] = off;
    off = up256(off + es * static_cast<size_t>(p.shape[L].count()));
  }
  p.ws_bytes = off;
  return MGARD_OK;
}

int get_plan4(const int64_t* dims, const double* const* coords, int dtype, Plan4** out) {
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  int L = 0;
  int rc = count_levels4(dims, &L);
  if (rc != MGARD_OK) return rc;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MGARD_ERR_CUDA;
  std::string key(reinterpret_cast<const char*>(&device), sizeof device);
  key.append(reinterpret_cast<const char*>(&dtype), sizeof dtype);
  key.append(reinterpret_cast<const char*>(dims), 4 * sizeof(int64_t));
  for (int a = 0; a < 4; ++a) {
    const double* c = coords ? coords[a] : nullptr;
    const char flag = c ? 1 : 0;
    key.push_back(flag);
    if (c) key.append(reinterpret_cast<const char*>(c), sizeof(double) * dims[a]);
  }
  std::lock_guard<std::mutex> lk(g_mu4);
  auto it = g_plans4.find(key);
  if (it != g_plans4.end()) {
    *out = it->second.get();
    return MGARD_OK;
  }
  auto p = std::make_unique<Plan4>();
  p->dtype = dtype;
  p->device = device;
  rc = dtype == MGARD_F64 ? build_plan4<double>(dims, coords, *p, true)
                          : build_plan4<float>(dims, coords, *p, true);
  if (rc != MGARD_OK) return rc;
  *out = p.get();
  g_plans4.emplace(key, std::move(p));
  return MGARD_OK;
}

double linf_constant4(const Plan4& p, int stop) {
  double C = 1.0;
  for (int l = stop + 1; l <= p.L; ++l) C = std::max(C, 1.0 + p.knorm[l]);
  return C;
}

void level_tolerances4(const Plan4& p, int stop, double tau, double* out) {
  const double C = linf_constant4(p, stop);
  const double kappa = 4.0;  // sqrt(2^4)
  double kpow = 1.0;
  for (int i = 0; i < p.L + 1 - stop; ++i) kpow *= kappa;
  const double t0 = (1.0 - kappa) * tau / ((1.0 - kpow) * C);
  for (int l = 0; l <= stop; ++l) out[l] = t0;
  for (int l = stop + 1; l <= p.L; ++l) out[l] = kappa * out[l - 1];
}

// ------------------------------------------------------------- transform

struct View {
  int64_t outer, inner;
};
View axis_view(const Shape4& s, int a) {
  View v{1, 1};
  for (int b = 0; b < a; ++b) v.outer *= s.n[b];
  for (int b = a + 1; b < 4; ++b) v.inner *= s.n[b];
  return v;
}

// Pi(c) (c of shape cs) into out (shape fs), through the scratch x / y.
template <typename T>
void expand4(const Plan4& p, int l, const T* c, T* out, T* x, T* y, cudaStream_t s) {
  Shape4 cur = p.shape[l - 1];
  const T* src = c;
  T* bufs[2] = {x, y};
  for (int a = 0; a < 4; ++a) {
    Shape4 next = cur;
    next.n[a] = p.shape[l].n[a];
    T* dst = a == 3 ? out : bufs[a & 1];
    const View v = axis_view(next, a);
    launch_pdl(expand_axis_kernel<T>, dim3(grid_of(next.count())), dim3(kT), 0, s, src, dst, v.outer,
               next.n[a], cur.n[a], v.inner, p.tab<T>(l, a, 0), p.tab<T>(l, a, 1));
    src = dst;
    cur = next;
  }
}

// R w (w of the level-l shape) into out (the coarse shape), then M_c^{-1}
// along every axis, through the scratch x / y.
template <typename T>
void correction4(const Plan4& p, int l, const T* w, T* out, T* x, T* y, cudaStream_t s) {
  Shape4 cur = p.shape[l];
  const T* src = w;
  T* bufs[2] = {x, y};
  for (int a = 0; a < 4; ++a) {
    Shape4 next = cur;
    next.n[a] = p.shape[l - 1].n[a];
    T* dst = a == 3 ? out : bufs[a & 1];
    const View v = axis_view(cur, a);
    launch_pdl(restrict_axis_kernel<T>, dim3(grid_of(next.count())), dim3(kT), 0, s, src, dst,
               v.outer, cur.n[a], next.n[a], v.inner, p.tab<T>(l, a, 2));
    src = dst;
    cur = next;
  }
  for (int a = 3; a >= 0; --a) {
    const View v = axis_view(cur, a);
    launch_pdl(thomas_axis_kernel<T>, dim3(grid_of(v.outer * v.inner)), dim3(kT), 0, s, out,
               v.outer, cur.n[a], v.inner, p.tab<T>(l, a, 3), p.tab<T>(l, a, 4), p.tab<T>(l, a, 5));
  }
}

template <typename T>
int run4(bool dec, const Plan4& p, int stop, T* data, char* ws, cudaStream_t s) {
  const int L = p.L;
  std::vector<T*> B(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) B[l] = reinterpret_cast<T*>(ws + p.offB[l]);
  T* E = reinterpret_cast<T*>(ws + p.off_buf[0]);
  T* W = reinterpret_cast<T*>(ws + p.off_buf[1]);
  T* X = reinterpret_cast<T*>(ws + p.off_buf[2]);
  T* Y = reinterpret_cast<T*>(ws + p.off_buf[3]);
  if (dec) {
    for (int l = L; l > stop; --l) {
      const Shape4 fs = p.shape[l], cs = p.shape[l - 1];
      launch_pdl(nodal4_kernel<T, true>, dim3(grid_of(cs.count())), dim3(kT), 0, s, B[l], fs, B[l - 1], cs);
      expand4<T>(p, l, B[l - 1], E, X, Y, s);
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(fs.count())), dim3(kT), 0, s, W,
                 static_cast<const T*>(B[l]), static_cast<const T*>(E), T(-1), fs.count());
      correction4<T>(p, l, W, E, X, Y, s);  // z into E (coarse shape)
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(cs.count())), dim3(kT), 0, s, B[l - 1],
                 static_cast<const T*>(B[l - 1]), static_cast<const T*>(E), T(1), cs.count());
      launch_pdl(coef4_kernel<T, 1>, dim3(grid_of(fs.count())), dim3(kT), 0, s, B[l], W, fs);
    }
    for (int l = stop + 1; l <= L; ++l)
      launch_pdl(nodal4_kernel<T, false>, dim3(grid_of(p.shape[l - 1].count())), dim3(kT), 0, s,
                 B[l], p.shape[l], B[l - 1], p.shape[l - 1]);
  } else {
    for (int l = L; l > stop; --l)
      launch_pdl(nodal4_kernel<T, true>, dim3(grid_of(p.shape[l - 1].count())), dim3(kT), 0, s,
                 B[l], p.shape[l], B[l - 1], p.shape[l - 1]);
    for (int l = stop + 1; l <= L; ++l) {
      const Shape4 fs = p.shape[l], cs = p.shape[l - 1];
      launch_pdl(coef4_kernel<T, 0>, dim3(grid_of(fs.count())), dim3(kT), 0, s, B[l], W, fs);
      correction4<T>(p, l, W, E, X, Y, s);  // z
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(cs.count())), dim3(kT), 0, s, B[l - 1],
                 static_cast<const T*>(B[l - 1]), static_cast<const T*>(E), T(-1), cs.count());
      expand4<T>(p, l, B[l - 1], E, X, Y, s);
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(fs.count())), dim3(kT), 0, s, B[l],
                 static_cast<const T*>(E), static_cast<const T*>(W), T(1), fs.count());
    }
  }
  return cudaGetLastError() == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
}

int transform4(bool dec, const int64_t* dims, const double* const* coords, int dtype, int stop,
               void* data, void* workspace, size_t ws_bytes, void* stream) {
  Plan4* p = nullptr;
  int rc = get_plan4(dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (stop < 0 || stop > p->L) return MGARD_ERR_LEVEL;
  const size_t es = dtype == MGARD_F64 ? 8 : 4;
  if (data == nullptr || reinterpret_cast<uintptr_t>(data) % es) return MGARD_ERR_ARG;
  if (stop == p->L) return MGARD_OK;
  if (workspace == nullptr || reinterpret_cast<uintptr_t>(workspace) % 256 || ws_bytes < p->ws_bytes)
    return MGARD_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return dtype == MGARD_F64 ? run4<double>(dec, *p, stop, static_cast<double*>(data), static_cast<char*>(workspace), s)
                            : run4<float>(dec, *p, stop, static_cast<float*>(data), static_cast<char*>(workspace), s);
}

int quant4(bool quantize, const int64_t* dims, const double* const* coords, int dtype, int stop,
           double tau, void* coeffs, int64_t* labels, double* tau_out, void* stream) {
  if (!(tau > 0.0) || !std::isfinite(tau)) return MGARD_ERR_ARG;
  Plan4* p = nullptr;
  int rc = get_plan4(dims, coords, dtype, &p);
  if (rc != MGARD_OK) return rc;
  if (stop < 0 || stop > p->L) return MGARD_ERR_LEVEL;
  const size_t es = dtype == MGARD_F64 ? 8 : 4;
  if (coeffs == nullptr || labels == nullptr || reinterpret_cast<uintptr_t>(coeffs) % es ||
      reinterpret_cast<uintptr_t>(labels) % 8)
    return MGARD_ERR_ARG;
  double t[kMaxLevels], q[kMaxLevels];
  level_tolerances4(*p, stop, tau, t);
  for (int l = 0; l < kMaxLevels; ++l) q[l] = l <= p->L ? 2.0 * t[l] : 1.0;
  if (tau_out)
    for (int l = 0; l <= p->L; ++l) tau_out[l] = t[l];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_mu4);  // the bin-width slot of the plan
  char* base = static_cast<char*>(p->dmem);
  double* dq = reinterpret_cast<double*>(base + p->q_off);
  if (cudaMemcpyAsync(dq, q, sizeof q, cudaMemcpyHostToDevice, s) != cudaSuccess) return MGARD_ERR_CUDA;
  const uint8_t* lv[4];
  for (int a = 0; a < 4; ++a) lv[a] = reinterpret_cast<const uint8_t*>(base + p->lev_off[a]);
  const Shape4 sh = p->shape[p->L];
  if (!quantize) {
    if (dtype == MGARD_F64)
      launch_pdl(dequantize4_kernel<double>, dim3(grid_of(sh.count())), dim3(kT), 0, s,
                 static_cast<const int64_t*>(labels), static_cast<double*>(coeffs), sh, lv[0], lv[1],
                 lv[2], lv[3], stop, static_cast<const double*>(dq));
    else
      launch_pdl(dequantize4_kernel<float>, dim3(grid_of(sh.count())), dim3(kT), 0, s,
                 static_cast<const int64_t*>(labels), static_cast<float*>(coeffs), sh, lv[0], lv[1],
                 lv[2], lv[3], stop, static_cast<const double*>(dq));
    // The bin widths must outlive the launch: wait before the slot is reused.
    return cudaStreamSynchronize(s) == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
  }
  unsigned int* flags = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&flags), sizeof(unsigned), s) != cudaSuccess)
    return MGARD_ERR_CUDA;
  cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
  if (dtype == MGARD_F64)
    launch_pdl(quantize4_kernel<double>, dim3(grid_of(sh.count())), dim3(kT), 0, s,
               static_cast<const double*>(coeffs), labels, sh, lv[0], lv[1], lv[2], lv[3], stop,
               static_cast<const double*>(dq), flags);
  else
    launch_pdl(quantize4_kernel<float>, dim3(grid_of(sh.count())), dim3(kT), 0, s,
               static_cast<const float*>(coeffs), labels, sh, lv[0], lv[1], lv[2], lv[3], stop,
               static_cast<const double*>(dq), flags);
  unsigned h = 0;
  cudaMemcpyAsync(&h, flags, sizeof h, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(flags, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MGARD_ERR_CUDA;
  if (h & 1u) return MGARD_ERR_NONFINITE;
  if (h & 2u) return MGARD_ERR_OVERFLOW;
  return MGARD_OK;
}

}  // namespace

void release_plans4(int device) {
  std::lock_guard<std::mutex> lk(g_mu4);
  for (auto it = g_plans4.begin(); it != g_plans4.end();) {
    if (it->second->device == device) it = g_plans4.erase(it);
    else ++it;
  }
}

}  // namespace mgb

using namespace mgb;

extern "C" {

int mgard_num_levels_4d(const int64_t* dims, int* L_out) {
  if (L_out == nullptr) return MGARD_ERR_ARG;
  return count_levels4(dims, L_out);
}

int mgard_workspace_size_4d(const int64_t* dims, int dtype, size_t* bytes) {
  if (bytes == nullptr) return MGARD_ERR_ARG;
  if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_ERR_ARG;
  int L = 0;
  const int rc = count_levels4(dims, &L);
  if (rc != MGARD_OK) return rc;
  const size_t es = dtype == MGARD_F64 ? 8 : 4;
  int64_t cur[4] = {dims[0], dims[1], dims[2], dims[3]};
  const size_t nL = static_cast<size_t>(cur[0] * cur[1] * cur[2] * cur[3]);
  size_t off = 0;
  for (int l = L - 1; l >= 0; --l) {
    for (int a = 0; a < 4; ++a) cur[a] = cur[a] / 2 + 1;
    off = up256(off + es * static_cast<size_t>(cur[0] * cur[1] * cur[2] * cur[3]));
  }
  for (int b = 0; b < 4; ++b) off = up256(off + es * nL);
  *bytes = off;
  return MGARD_OK;
}

int mgard_level_tolerances_4d(const int64_t* dims, const double* const* coords, int stop_level,
                              double tau_linf, double* tau_out) {
  if (tau_out == nullptr || !(tau_linf > 0.0) || !std::isfinite(tau_linf)) return MGARD_ERR_ARG;
  Plan4 p;  // host tables only: no device needed
  const int rc = build_plan4<double>(dims, coords, p, false);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > p.L) return MGARD_ERR_LEVEL;
  level_tolerances4(p, stop_level, tau_linf, tau_out);
  return MGARD_OK;
}

int mgard_decompose_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                       void* data, void* workspace, size_t ws_bytes, void* stream) {
  return transform4(true, dims, coords, dtype, stop_level, data, workspace, ws_bytes, stream);
}

int mgard_recompose_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                       void* data, void* workspace, size_t ws_bytes, void* stream) {
  return transform4(false, dims, coords, dtype, stop_level, data, workspace, ws_bytes, stream);
}

int mgard_quantize_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                      double tau_linf, const void* coeffs, int64_t* labels, double* tau_levels_out,
                      void* stream) {
  return quant4(true, dims, coords, dtype, stop_level, tau_linf, const_cast<void*>(coeffs), labels,
                tau_levels_out, stream);
}

int mgard_dequantize_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                        double tau_linf, const int64_t* labels, void* coeffs, void* stream) {
  return quant4(false, dims, coords, dtype, stop_level, tau_linf, coeffs,
                const_cast<int64_t*>(labels), nullptr, stream);
}

}  // extern "C"
