// Four-dimensional grids (QMCPACK's shape class, Section 6): the same
// multilevel decomposition, recomposition and level-wise quantization on a
// 4D tensor-product grid.  The operators are applied the way they factor,
// axis by axis, in separate passes (not the fused 1-3D kernels).
//
// Decomposition of level l (v the level-l grid, c the compact coarse grid):
//   one pass: c = v at the coarse nodes, and at every other node
//             v <- w = v - Pi(v at the coarse nodes) (the coefficients,
//             Section 2; Pi the multilinear interpolant),
//   F = (R_0 x R_1 x R_2 x R_3) w, one restriction pass per axis (R the
//       rows of P^T M_f, Section 5.2; the first pass reads v with its
//       coarse nodes taken as 0),
//   z = M_c^{-1} F, a Thomas solve along every axis (Section 5.4),
//   Q_{l-1}u = c + z.
// The coarse values go back into the nodal positions, coarsest first.
// Recomposition inverts it: the level grids are gathered from u_mc, then
// per level z = M_c^{-1} R w (w the coefficients at their nodes),
// c' = Q_{l-1}u - z and, in one pass, v = Pi(c') + w.
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

#include "devplan.hpp"
#include "mgard_gb.h"
#include "pdl.cuh"
#include "plan.hpp"

namespace mgb {
namespace {

__host__ __device__ __forceinline__ int cpos4(int k, int n) { return min(2 * k, n - 1); }
__host__ __device__ __forceinline__ bool coef4(int j, int n) { return (j & 1) && j != n - 1; }

constexpr int kT = 256;
constexpr int64_t kMaxNodes4 = (int64_t(1) << 31) - 1;  // 32-bit index arithmetic

unsigned grid_of(int64_t n) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + kT - 1) / kT)));
}

// Division by a run-time invariant divisor as a multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Theorem 4.2 with N = 32): for d >= 1,
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// floor(n / d) = (mulhi(m, n) + n) >> l for every 0 <= n < 2^32; the sum
// does not wrap because mulhi(m, n) <= n and n < 2^31 here.
struct FDiv {
  uint32_t m = 1, l = 0;
  FDiv() = default;
  explicit FDiv(uint32_t d) {
    while ((uint64_t(1) << l) < d) ++l;
    m = static_cast<uint32_t>(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(m, n) + n) >> l; }
};

struct Shape4 {
  int n[4];
  FDiv f[4];
  __host__ __device__ int64_t count() const { return int64_t(n[0]) * n[1] * n[2] * n[3]; }
};

Shape4 make_shape4(const int* n) {
  Shape4 s;
  for (int a = 0; a < 4; ++a) {
    s.n[a] = n[a];
    s.f[a] = FDiv(static_cast<uint32_t>(n[a]));
  }
  return s;
}

__device__ __forceinline__ void unflat(uint32_t t, const Shape4& s, int i[4]) {
  uint32_t q = s.f[3].div(t);
  i[3] = static_cast<int>(t - q * s.n[3]);
  t = q;
  q = s.f[2].div(t);
  i[2] = static_cast<int>(t - q * s.n[2]);
  t = q;
  q = s.f[1].div(t);
  i[1] = static_cast<int>(t - q * s.n[1]);
  i[0] = static_cast<int>(q);
}
__device__ __forceinline__ uint32_t flat(const int i[4], const Shape4& s) {
  return ((uint32_t(i[0]) * s.n[1] + i[1]) * s.n[2] + i[2]) * s.n[3] + i[3];
}

#define GRID_LOOP(t, total)                                                        \
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < (total); t += gridDim.x * blockDim.x)

// Coarse grid c <- fine grid f at the coarse nodes (or the reverse).
template <typename T, bool GATHER>
__global__ void __launch_bounds__(kT)
nodal4_kernel(T* __restrict__ f, Shape4 fs, T* __restrict__ c, Shape4 cs) {
  grid_dep_enter();
  const uint32_t total = static_cast<uint32_t>(cs.count());
  GRID_LOOP(t, total) {
    int k[4], j[4];
    unflat(t, cs, k);
    for (int a = 0; a < 4; ++a) j[a] = cpos4(k[a], fs.n[a]);
    if (GATHER) c[t] = f[flat(j, fs)];
    else f[flat(j, fs)] = c[t];
  }
}

// The per-axis interpolation tables of one level transition.
template <typename T>
struct Interp4 {
  const T* iwl[4];
  const T* iwr[4];
};

// Taps of the multilinear interpolant at fine index j of one axis: the node
// itself (coarse on this axis) or its two coarse neighbours.  `fine` gives
// positions in the fine axis, otherwise in the compact coarse axis.
template <typename T>
__device__ __forceinline__ int taps4(int j, int n, int nc, bool fine, const T* iwl, const T* iwr,
                                     int pos[2], T w[2]) {
  if (coef4(j, n)) {
    pos[0] = fine ? j - 1 : (j - 1) >> 1;
    pos[1] = fine ? j + 1 : (j + 1) >> 1;
    w[0] = iwl[j];
    w[1] = iwr[j];
    return 2;
  }
  pos[0] = fine ? j : (j == n - 1 ? nc - 1 : j >> 1);
  pos[1] = pos[0];
  w[0] = T(1);
  w[1] = T(0);
  return 1;
}

// Decomposition of one level in one pass: at every node that is not in the
// coarse grid, v <- v - Pi(v at the coarse nodes) (the coefficient; the
// interpolant's taps all lie on coarse nodes, which no thread writes); every
// coarse node's value goes to the compact coarse array c.
// Recomposition's last step, in place: v <- Pi(c) + v at the coefficient
// nodes, v <- c at the coarse nodes (c the compact corrected coarse array).
//
// A warp takes one plane (j0, j1) of the level grid and a chunk of kChunk4
// nodes of axis 3 (lane l at j3 = kChunk4 q - 1 + l; lanes 1..30 write,
// lanes 0 and 31 only supply taps) and walks axis 2.  At a node coarse on
// axes 2 and 3 a lane sums the interpolant over axes 0-1 (R, from up to 4
// coarse planes); along axis 2 the coefficient rows interpolate the R of the
// coarse rows on either side (kept in registers), and along axis 3 the
// coefficient lanes combine their neighbours' values through warp shuffles.
// So every coarse value is loaded once per plane, and the taps and weights
// of axes 0-1 are formed once per walk.
constexpr int kChunk4 = 30;

template <typename T, bool DEC>
__global__ void __launch_bounds__(kT)
interp4_kernel(T* __restrict__ v, T* __restrict__ c, Shape4 fs, Shape4 cs, Interp4<T> ip,
               int nchunks, FDiv f_chunks) {
  grid_dep_enter();
  const int lane = threadIdx.x & 31;
  const int n2 = fs.n[2], n3 = fs.n[3], nc2 = cs.n[2], nc3 = cs.n[3];
  const uint32_t items = uint32_t(fs.n[0]) * fs.n[1] * uint32_t(nchunks);
  const uint32_t nwarps = gridDim.x * (kT / 32);
  const Shape4& src = DEC ? fs : cs;
  const T* base = DEC ? v : c;
  const uint32_t splane = uint32_t(src.n[2]) * src.n[3];
  for (uint32_t it = blockIdx.x * (kT / 32) + (threadIdx.x >> 5); it < items; it += nwarps) {
    const uint32_t pl = f_chunks.div(it);
    const int q = static_cast<int>(it - pl * nchunks);
    const uint32_t j0u = fs.f[1].div(pl);
    const int j1 = static_cast<int>(pl - j0u * fs.n[1]);
    const int j0 = static_cast<int>(j0u);
    int p0[2], p1[2];
    T w0[2], w1[2];
    const int c0 = taps4<T>(j0, fs.n[0], cs.n[0], DEC, ip.iwl[0], ip.iwr[0], p0, w0);
    const int c1 = taps4<T>(j1, fs.n[1], cs.n[1], DEC, ip.iwl[1], ip.iwr[1], p1, w1);
    const bool coarse01 = c0 == 1 && c1 == 1;
    uint32_t po[2][2];
    T w01[2][2];
#pragma unroll
    for (int a0 = 0; a0 < 2; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 2; ++a1) {
        po[a0][a1] = (uint32_t(p0[a0]) * src.n[1] + p1[a1]) * splane;
        w01[a0][a1] = w0[a0] * w1[a1];
      }
    uint32_t cplane = 0;  // the plane's offset in c when it is coarse on axes 0-1
    if (DEC && coarse01) {
      const int k0 = j0 == fs.n[0] - 1 ? cs.n[0] - 1 : (j0 >> 1);
      const int k1 = j1 == fs.n[1] - 1 ? cs.n[1] - 1 : (j1 >> 1);
      cplane = (uint32_t(k0) * cs.n[1] + k1) * uint32_t(nc2) * uint32_t(nc3);
    }
    const int j3 = kChunk4 * q - 1 + lane;
    const bool in3 = j3 >= 0 && j3 < n3;
    const bool coarse3 = in3 && !coef4(j3, n3);
    const bool out3 = in3 && lane != 0 && lane != 31;
    const int k3 = j3 == n3 - 1 ? nc3 - 1 : (j3 >> 1);
    const int at3 = DEC ? j3 : k3;
    const T w3l = out3 && !coarse3 ? ip.iwl[3][j3] : T(0);
    const T w3r = out3 && !coarse3 ? ip.iwr[3][j3] : T(0);
    T* vplane = v + pl * uint32_t(n2) * uint32_t(n3);

    // R at a row j2 that is coarse on axis 2.
    auto coarse_row = [&](int j2) -> T {
      const int at2 = DEC ? j2 : (j2 == n2 - 1 ? nc2 - 1 : (j2 >> 1));
      const uint32_t off = uint32_t(at2) * src.n[3] + at3;
      T R = T(0);
      if (coarse3) {
#pragma unroll
        for (int a0 = 0; a0 < 2; ++a0) {
          if (a0 >= c0) break;
#pragma unroll
          for (int a1 = 0; a1 < 2; ++a1) {
            if (a1 >= c1) break;
            R += w01[a0][a1] * base[po[a0][a1] + off];
          }
        }
      }
      return R;
    };
    // Row j2 given the interpolant over axes 0-2 at the lane's node (coarse
    // on axis 3) or at its neighbours (coefficient on axis 3); vj is the
    // row's current value at the lane's node.
    auto emit = [&](int j2, T R, bool coarse2, T vj) {
      const T Rl = __shfl_up_sync(0xffffffffu, R, 1);
      const T Rr = __shfl_down_sync(0xffffffffu, R, 1);
      if (!out3) return;
      T* p = vplane + uint32_t(j2) * n3 + j3;
      if (coarse3 && coarse2 && coarse01) {
        if (DEC) c[cplane + (uint32_t(j2 == n2 - 1 ? nc2 - 1 : (j2 >> 1)) * nc3) + k3] = R;
        else *p = R;
        return;
      }
      const T pi = coarse3 ? R : w3l * Rl + w3r * Rr;
      *p = DEC ? vj - pi : vj + pi;
    };
    // A step covers a coefficient row of axis 2 and the coarse row after it,
    // or a single coarse row.  The loads of the next step are issued before
    // the current step's stores (two steps in flight per warp).
    auto fetch = [&](int js, T& Rn, T& va, T& vb, bool& pair) {
      pair = coef4(js, n2);
      Rn = coarse_row(pair ? js + 1 : js);
      va = out3 ? vplane[uint32_t(js) * n3 + j3] : T(0);
      vb = out3 && pair ? vplane[uint32_t(js + 1) * n3 + j3] : T(0);
    };
    T Rn, va, vb, Rprev = T(0);
    bool pair;
    fetch(0, Rn, va, vb, pair);
    for (int js = 0;;) {
      const int jn = js + (pair ? 2 : 1);
      T Rn2 = T(0), va2 = T(0), vb2 = T(0);
      bool pair2 = false;
      if (jn < n2) fetch(jn, Rn2, va2, vb2, pair2);
      if (pair) {
        emit(js, ip.iwl[2][js] * Rprev + ip.iwr[2][js] * Rn, false, va);
        emit(js + 1, Rn, true, vb);
      } else {
        emit(js, Rn, true, va);
      }
      Rprev = Rn;
      if (jn >= n2) break;
      js = jn;
      Rn = Rn2;
      va = va2;
      vb = vb2;
      pair = pair2;
    }
  }
}

// One axis of the restriction, out[.., k, ..] = sum_d rw[5k + d] in[.., cpos(k) + d - 2, ..]
// over the array seen as (outer, n, inner) -> (outer, nc, inner), a thread per
// output (used along the contiguous axis, inner = 1, where neighbouring
// threads read neighbouring inputs).
template <typename T>
__global__ void __launch_bounds__(kT)
restrict_axis_kernel(const T* __restrict__ in, T* __restrict__ out, uint32_t outer, int n, int nc,
                     uint32_t inner, FDiv f_inner, FDiv f_nc, const T* __restrict__ rw) {
  grid_dep_enter();
  const uint32_t total = outer * uint32_t(nc) * inner;
  GRID_LOOP(t, total) {
    const uint32_t q = f_inner.div(t);
    const uint32_t i = t - q * inner;
    const uint32_t o = f_nc.div(q);
    const int k = static_cast<int>(q - o * nc);
    const T* row = in + o * uint32_t(n) * inner + i;
    const int c = cpos4(k, n);
    T acc = T(0);
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      const int j = c + d - 2;
      if (j >= 0 && j < n) acc += rw[5 * k + d] * row[uint32_t(j) * inner];
    }
    out[t] = acc;
  }
}

// The restriction along an axis whose lines are strided (inner > 1): a
// thread per line (o, i) walks k = 0..nc-1 with the five taps c-2..c+2
// (c = cpos(k)) in registers, loading each input once.  MASK as above.
template <typename T, bool MASK>
__global__ void __launch_bounds__(kT)
restrict_lines_kernel(const T* __restrict__ in, T* __restrict__ out, uint32_t outer, int n, int nc,
                      uint32_t inner, FDiv f_inner, const T* __restrict__ rw, Shape4 fs) {
  grid_dep_enter();
  const uint32_t lines = outer * inner;
  GRID_LOOP(t, lines) {
    const uint32_t o = f_inner.div(t);
    const uint32_t i = t - o * inner;
    const T* src = in + o * uint32_t(n) * inner + i;
    T* dst = out + o * uint32_t(nc) * inner + i;
    bool inner_coarse = false;
    if (MASK) {
      const uint32_t q3 = fs.f[3].div(i);
      const int j3 = static_cast<int>(i - q3 * fs.n[3]);
      const uint32_t j1 = fs.f[2].div(q3);
      const int j2 = static_cast<int>(q3 - j1 * fs.n[2]);
      inner_coarse = !coef4(int(j1), fs.n[1]) && !coef4(j2, fs.n[2]) && !coef4(j3, fs.n[3]);
    }
    auto ld = [&](int j) -> T {
      if (j >= n || (MASK && inner_coarse && !coef4(j, n))) return T(0);
      return src[uint32_t(j) * inner];
    };
    T x0 = T(0), x1 = T(0), x2 = ld(0), x3 = ld(1), x4 = ld(2);
    dst[0] = rw[0] * x0 + rw[1] * x1 + rw[2] * x2 + rw[3] * x3 + rw[4] * x4;
    // Steps of two fine nodes while cpos(k) = 2k; with n even the last
    // coarse node is the last fine node, one step further.
    const int k2 = (n & 1) ? nc : nc - 1;
#pragma unroll 4
    for (int k = 1; k < k2; ++k) {
      x0 = x2; x1 = x3; x2 = x4;
      x3 = ld(2 * k + 1);
      x4 = ld(2 * k + 2);
      const T* r5 = rw + 5 * k;
      dst[uint32_t(k) * inner] = r5[0] * x0 + r5[1] * x1 + r5[2] * x2 + r5[3] * x3 + r5[4] * x4;
    }
    if (k2 < nc) {
      x0 = x1; x1 = x2; x2 = x3; x3 = x4;
      const T* r5 = rw + 5 * k2;
      dst[uint32_t(k2) * inner] = r5[0] * x0 + r5[1] * x1 + r5[2] * x2 + r5[3] * x3;
    }
  }
}

// Thomas solve of M_c along one axis, a thread per line; the loads of a
// block of kTB rows are issued together ahead of the recurrence.
constexpr int kTB = 8;

template <typename T>
__global__ void __launch_bounds__(kT)
thomas_axis_kernel(T* __restrict__ F, uint32_t outer, int nc, uint32_t inner, FDiv f_inner,
                   const T* __restrict__ ta, const T* __restrict__ tm, const T* __restrict__ tc) {
  grid_dep_enter();
  const uint32_t lines = outer * inner;
  GRID_LOOP(t, lines) {
    const uint32_t o = f_inner.div(t);
    const uint32_t i = t - o * inner;
    T* l = F + o * uint32_t(nc) * inner + i;
    T y = T(0);
    for (int k0 = 0; k0 < nc; k0 += kTB) {
      T f[kTB];
#pragma unroll
      for (int u = 0; u < kTB; ++u)
        if (k0 + u < nc) f[u] = l[uint32_t(k0 + u) * inner];
#pragma unroll
      for (int u = 0; u < kTB; ++u)
        if (k0 + u < nc) {
          y = (f[u] - ta[k0 + u] * y) * tm[k0 + u];
          l[uint32_t(k0 + u) * inner] = y;
        }
    }
    T x = T(0);
    for (int k1 = nc - 1; k1 >= 0; k1 -= kTB) {
      T f[kTB];
#pragma unroll
      for (int u = 0; u < kTB; ++u)
        if (k1 - u >= 0) f[u] = l[uint32_t(k1 - u) * inner];
#pragma unroll
      for (int u = 0; u < kTB; ++u)
        if (k1 - u >= 0) {
          x = f[u] - tc[k1 - u] * x;
          l[uint32_t(k1 - u) * inner] = x;
        }
    }
  }
}

// Thomas solve along the contiguous axis (inner = 1): a CTA stages
// kThomasLines consecutive lines (one contiguous span of the array) in
// shared memory with coalesced copies, a thread solves one line there (row
// pitch ld = nc rounded up to odd, against bank conflicts), and the span is
// copied back.
constexpr int kThomasLines = 128;

template <typename T>
__global__ void __launch_bounds__(kThomasLines)
thomas_contig_kernel(T* __restrict__ F, uint32_t lines, int nc, int ld, FDiv f_nc,
                     const T* __restrict__ ta, const T* __restrict__ tm, const T* __restrict__ tc) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem4[];
  T* sm = reinterpret_cast<T*>(smem4);
  for (uint32_t l0 = blockIdx.x * kThomasLines; l0 < lines; l0 += gridDim.x * kThomasLines) {
    const uint32_t nl = min(uint32_t(kThomasLines), lines - l0);
    const uint32_t cnt = nl * uint32_t(nc);
    T* g = F + l0 * uint32_t(nc);
    for (uint32_t e = threadIdx.x; e < cnt; e += kThomasLines) {
      const uint32_t li = f_nc.div(e);
      sm[li * ld + (e - li * nc)] = g[e];
    }
    __syncthreads();
    if (threadIdx.x < nl) {
      T* l = sm + threadIdx.x * ld;
      T y = T(0);
      for (int k = 0; k < nc; ++k) {
        y = (l[k] - ta[k] * y) * tm[k];
        l[k] = y;
      }
      T x = T(0);
      for (int k = nc - 1; k >= 0; --k) {
        x = l[k] - tc[k] * x;
        l[k] = x;
      }
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < cnt; e += kThomasLines) {
      const uint32_t li = f_nc.div(e);
      g[e] = sm[li * ld + (e - li * nc)];
    }
    __syncthreads();
  }
}

// out = a + s * b elementwise.
template <typename T>
__global__ void __launch_bounds__(kT)
axpy4_kernel(T* __restrict__ out, const T* __restrict__ a, const T* __restrict__ b, T s, uint32_t n) {
  grid_dep_enter();
  GRID_LOOP(t, n) out[t] = a[t] + s * b[t];
}

#undef GRID_LOOP

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
  std::array<std::vector<uint8_t>, 4> lev;  // per finest index of an axis: least level holding it
  size_t lev012_off = 0;  // per row (j0, j1, j2): the largest of its three axes' levels
  size_t lev3_off = 0;    // per index of axis 3
  void* dmem = nullptr;
  std::vector<size_t> offB;             // compact level grids l < L
  size_t off_buf[3] = {0, 0, 0};        // scratch: two of #N_L elements, one of #N_{L-1}
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
  if (cur[0] * cur[1] * cur[2] * cur[3] > kMaxNodes4) return MGARD_ERR_SHAPE;
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
  for (int l = 0; l <= L; ++l) {
    int n[4];
    for (int a = 0; a < 4; ++a) n[a] = static_cast<int>(idx[l][a].size());
    p.shape[l] = make_shape4(n);
  }
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
  }
  if (!upload) return MGARD_OK;
  // The quantizer sees the array as rows (j0, j1, j2) of n3 elements.
  std::vector<uint8_t> lev012(static_cast<size_t>(dims[0] * dims[1] * dims[2]));
  for (int64_t j0 = 0, r = 0; j0 < dims[0]; ++j0)
    for (int64_t j1 = 0; j1 < dims[1]; ++j1)
      for (int64_t j2 = 0; j2 < dims[2]; ++j2, ++r)
        lev012[r] = std::max(std::max(p.lev[0][j0], p.lev[1][j1]), p.lev[2][j2]);
  p.lev012_off = reserve(lev012.size());
  p.lev3_off = reserve(p.lev[3].size());
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
  std::memcpy(stage.data() + p.lev012_off, lev012.data(), lev012.size());
  std::memcpy(stage.data() + p.lev3_off, p.lev[3].data(), p.lev[3].size());
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
  for (int b = 0; b < 3; ++b) {
    p.off_buf[b] = off;
    off = up256(off + es * static_cast<size_t>(p.shape[b < 2 ? L : std::max(L - 1, 0)].count()));
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
  uint32_t outer, inner;
};
View axis_view(const Shape4& s, int a) {
  View v{1, 1};
  for (int b = 0; b < a; ++b) v.outer *= static_cast<uint32_t>(s.n[b]);
  for (int b = a + 1; b < 4; ++b) v.inner *= static_cast<uint32_t>(s.n[b]);
  return v;
}

// The shape s with axis a set to n.
Shape4 with_axis(const Shape4& s, int a, int n) {
  int m[4] = {s.n[0], s.n[1], s.n[2], s.n[3]};
  m[a] = n;
  return make_shape4(m);
}

template <typename T>
Interp4<T> interp_tables(const Plan4& p, int l) {
  Interp4<T> ip;
  for (int a = 0; a < 4; ++a) {
    ip.iwl[a] = p.tab<T>(l, a, 0);
    ip.iwr[a] = p.tab<T>(l, a, 1);
  }
  return ip;
}

// A warp per (plane, chunk of axis 3) work item.
template <typename T, bool DEC>
void launch_interp4(const Plan4& p, int l, T* v, T* c, cudaStream_t s) {
  const Shape4 fs = p.shape[l], cs = p.shape[l - 1];
  const int nchunks = (fs.n[3] + kChunk4 - 1) / kChunk4;  // chunk q writes j3 = 30q .. 30q + 29
  const int64_t items = int64_t(fs.n[0]) * fs.n[1] * nchunks;
  const unsigned g = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>(152 * 16, (items + kT / 32 - 1) / (kT / 32))));
  launch_pdl(interp4_kernel<T, DEC>, dim3(g), dim3(kT), 0, s, v, c, fs, cs, interp_tables<T>(p, l),
             nchunks, FDiv(static_cast<uint32_t>(nchunks)));
}

// z = M_c^{-1} R w into out (the coarse shape), w read from the level-l
// array v at its coefficient nodes (0 at the coarse nodes): a restriction
// pass per axis through the scratch x / y, then a Thomas pass per axis.
template <typename T>
void correction4(const Plan4& p, int l, const T* v, T* out, T* x, T* y, cudaStream_t s) {
  const Shape4 fs = p.shape[l];
  Shape4 cur = fs;
  const T* src = v;
  T* bufs[2] = {x, y};
  for (int a = 0; a < 4; ++a) {
    const Shape4 next = with_axis(cur, a, p.shape[l - 1].n[a]);
    T* dst = a == 3 ? out : bufs[a & 1];
    const View w = axis_view(cur, a);
    const FDiv fi(w.inner);
    const T* rw = p.tab<T>(l, a, 2);
    if (w.inner == 1)
      launch_pdl(restrict_axis_kernel<T>, dim3(grid_of(next.count())), dim3(kT), 0, s, src, dst,
                 w.outer, cur.n[a], next.n[a], w.inner, fi, FDiv(static_cast<uint32_t>(next.n[a])), rw);
    else if (a == 0)
      launch_pdl(restrict_lines_kernel<T, true>, dim3(grid_of(int64_t(w.outer) * w.inner)), dim3(kT), 0,
                 s, src, dst, w.outer, cur.n[a], next.n[a], w.inner, fi, rw, fs);
    else
      launch_pdl(restrict_lines_kernel<T, false>, dim3(grid_of(int64_t(w.outer) * w.inner)), dim3(kT), 0,
                 s, src, dst, w.outer, cur.n[a], next.n[a], w.inner, fi, rw, fs);
    src = dst;
    cur = next;
  }
  for (int a = 3; a >= 0; --a) {
    const View w = axis_view(cur, a);
    const int nc = cur.n[a];
    const int ld = nc | 1;
    const size_t smem = sizeof(T) * kThomasLines * ld;
    const T *ta = p.tab<T>(l, a, 3), *tm = p.tab<T>(l, a, 4), *tc = p.tab<T>(l, a, 5);
    if (w.inner == 1 && smem <= 48 * 1024) {
      const int64_t lines = w.outer;
      const unsigned g = static_cast<unsigned>(
          std::max<int64_t>(1, std::min<int64_t>(152 * 8, (lines + kThomasLines - 1) / kThomasLines)));
      launch_pdl(thomas_contig_kernel<T>, dim3(g), dim3(kThomasLines), smem, s, out, w.outer, nc, ld,
                 FDiv(static_cast<uint32_t>(nc)), ta, tm, tc);
    } else {
      launch_pdl(thomas_axis_kernel<T>, dim3(grid_of(int64_t(w.outer) * w.inner)), dim3(kT), 0, s,
                 out, w.outer, nc, w.inner, FDiv(w.inner), ta, tm, tc);
    }
  }
}

template <typename T>
int run4(bool dec, const Plan4& p, int stop, T* data, char* ws, cudaStream_t s) {
  const int L = p.L;
  std::vector<T*> B(L + 1);
  B[L] = data;
  for (int l = 0; l < L; ++l) B[l] = reinterpret_cast<T*>(ws + p.offB[l]);
  T* X = reinterpret_cast<T*>(ws + p.off_buf[0]);
  T* Y = reinterpret_cast<T*>(ws + p.off_buf[1]);
  T* Z = reinterpret_cast<T*>(ws + p.off_buf[2]);
  if (dec) {
    for (int l = L; l > stop; --l) {
      const Shape4 fs = p.shape[l], cs = p.shape[l - 1];
      // Coefficients in place, the coarse values into B[l-1].
      launch_interp4<T, true>(p, l, B[l], B[l - 1], s);
      correction4<T>(p, l, B[l], Z, X, Y, s);
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(cs.count())), dim3(kT), 0, s, B[l - 1],
                 static_cast<const T*>(B[l - 1]), static_cast<const T*>(Z), T(1), static_cast<uint32_t>(cs.count()));
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
      correction4<T>(p, l, B[l], Z, X, Y, s);
      launch_pdl(axpy4_kernel<T>, dim3(grid_of(cs.count())), dim3(kT), 0, s, B[l - 1],
                 static_cast<const T*>(B[l - 1]), static_cast<const T*>(Z), T(-1), static_cast<uint32_t>(cs.count()));
      launch_interp4<T, false>(p, l, B[l], B[l - 1], s);
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
  double t[kMaxLevels];
  level_tolerances4(*p, stop, tau, t);
  LevelTable tab;
  rc = make_level_table(p->L, stop, t, tab, tau_out);
  if (rc != MGARD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* base = static_cast<const char*>(p->dmem);
  const uint8_t* lev012 = reinterpret_cast<const uint8_t*>(base + p->lev012_off);
  const uint8_t* lev3 = reinterpret_cast<const uint8_t*>(base + p->lev3_off);
  const int64_t rows = dims[0] * dims[1] * dims[2], n3 = dims[3];
  // The quantizer kernels of the 1-3D path on the (rows, n3) view: the same
  // exact fast paths and FP64 fallbacks.
  if (!quantize) {
    const cudaError_t e =
        dtype == MGARD_F64
            ? launch_dequantize<double>(labels, static_cast<double*>(coeffs), lev012, lev3, rows, n3,
                                        stop, tab, s)
            : launch_dequantize<float>(labels, static_cast<float*>(coeffs), lev012, lev3, rows, n3,
                                       stop, tab, s);
    return e == cudaSuccess ? MGARD_OK : MGARD_ERR_CUDA;
  }
  unsigned int* flags = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&flags), sizeof(unsigned), s) != cudaSuccess)
    return MGARD_ERR_CUDA;
  cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
  const cudaError_t e =
      dtype == MGARD_F64
          ? launch_quantize<double>(static_cast<const double*>(coeffs), labels, lev012, lev3, rows, n3,
                                    stop, tab, flags, s)
          : launch_quantize<float>(static_cast<const float*>(coeffs), labels, lev012, lev3, rows, n3,
                                   stop, tab, flags, s);
  unsigned h = 0;
  cudaMemcpyAsync(&h, flags, sizeof h, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(flags, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || e != cudaSuccess) return MGARD_ERR_CUDA;
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
  size_t off = 0, nL1 = nL;
  for (int l = L - 1; l >= 0; --l) {
    for (int a = 0; a < 4; ++a) cur[a] = cur[a] / 2 + 1;
    const size_t cnt = static_cast<size_t>(cur[0] * cur[1] * cur[2] * cur[3]);
    if (l == L - 1) nL1 = cnt;
    off = up256(off + es * cnt);
  }
  off = up256(off + es * nL);
  off = up256(off + es * nL);
  off = up256(off + es * nL1);
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
