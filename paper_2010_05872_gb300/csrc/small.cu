// The coarsest levels of a transform in one CTA.  Below a few tens of
// thousands of nodes every per-level kernel is a handful of CTAs whose cost
// is launch and latency; here one CTA (1024 threads) loads the grid of the
// highest small level and every level's tables into shared memory, runs the
// whole decomposition (or recomposition) of the levels below it there, and
// writes the grid back.
//
// Per level transition (tables of the level, Section 2):
//   decomposition : F = R v - (R P) v_c, Thomas solves along each axis,
//                   coarse values v_c + z, coefficients v - Pi(v_c); after
//                   the coarsest level the final coarse values go back into
//                   the nodal positions, coarsest first;
//   recomposition : the coarse grids are gathered from the nodal positions
//                   first; then, coarsest first, F = R w - (R S) w_c, the
//                   solves, c' = Q u - z, and the grid becomes Pi(c') plus the
//                   coefficients.
// These are the same operators as the per-level kernels; only the order of
// the rounding differs.  Every phase is latency-bound on one SM, so each is
// laid out to keep many independent loads in flight with little integer
// work per node:
//   * the load vector is separable: a walk along axis 1 per (fine plane,
//     coarse column) applies the axis-2 and axis-1 rows of R with a
//     five-row window (scratch S = R1 R2 v on every fine plane), then a walk
//     along axis 0 per coarse (row, column) applies R0 to S and subtracts
//     X0 of the axis-1/2 products of X on the nodal planes, writing F in
//     place of S one plane late (a plane of S is no longer read once the
//     walk has passed it);
//   * the coefficient / interpolation pass takes a fine row and one nodal
//     column with the coefficient column to its right, so the axis-0/1
//     interpolant of the two nodal columns is formed once for both nodes;
//   * indices come from multiply-high divisions by per-level constants.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "pdl.cuh"
#include "grid.cuh"
#include "kernels.cuh"
#include "tma.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

// FP32 grids reach 33^3 nodes and take 1024 threads; FP64 ones stay at 17^3
// (shared-memory capacity), where 512 threads with more registers each do.
template <typename T>
constexpr int small_threads() { return sizeof(T) == 4 ? 1024 : 512; }
constexpr int kTabArrays = 7;  // iwl, iwr, rw, X, ta, tm, tc
constexpr int kSmallSegs = kSmallMaxLevels * 3 * kTabArrays;

// Division by a divisor fixed for the launch: q = umulhi(x, m) with
// m = ceil(2^32 / d), exact while x * d < 2^32 (m = 0 stands for d = 1).
struct FastDiv {
  unsigned d, m;
};
FastDiv make_fastdiv(unsigned d) {
  return {d, d <= 1 ? 0u : static_cast<unsigned>((0x100000000ull + d - 1) / d)};
}
__device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return f.m ? static_cast<int>(__umulhi(static_cast<unsigned>(x), f.m)) : x;
}

// Transition i of the launch: fine grid G[i + 1] (n) -> coarse grid G[i] (c).
struct SmallLevel {
  int n[3], c[3];
  int toff[3];  // each axis's table block, elements from the table base
  FastDiv dc2, dc1, dn1;
};

template <typename T>
struct SmallSeg {  // one table array copied to shared memory
  const T* src;
  int dst, count;
};

template <typename T>
struct SmallParams {
  SmallLevel lv[kSmallMaxLevels];
  int goff[kSmallMaxLevels + 1];  // G[i], elements from the shared-memory base
  int boff;                       // load-vector scratch (S, then F)
  int ntop;                       // nodes of the highest grid G[nlev]
  int nseg;
  SmallSeg<T> seg[kSmallSegs];
};

// One axis's tables in shared memory, in this order: iwl, iwr [n],
// rw [5 nc], X [3 nc] (R P or R S by direction), ta, tm, tc [nc].
template <typename T>
struct AxS {
  const T *iwl, *iwr, *rw, *x, *ta, *tm, *tc;
};
__host__ __device__ __forceinline__ int axis_table_size(int n, int nc) { return 2 * n + 11 * nc; }
template <typename T>
__device__ __forceinline__ AxS<T> axis_smem(const T* tab, int off, int n, int nc) {
  AxS<T> a;
  a.iwl = tab + off;
  a.iwr = a.iwl + n;
  a.rw = a.iwr + n;
  a.x = a.rw + 5 * nc;
  a.ta = a.x + 3 * nc;
  a.tm = a.ta + nc;
  a.tc = a.tm + nc;
  return a;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Load vector, first pass: S[j0][k1][k2] = sum_b R1[k1][b] sum_o R2[k2][o]
// v[j0][cpos(k1) + b - 2][cpos(k2) + o - 2] on every fine plane j0 (taps
// outside the grid read as zero).  A thread walks one (j0, k2) line along
// axis 1, forming each fine row's axis-2 sum once and keeping five of them.
template <typename T>
__device__ void lv_rows(const SmallLevel& L, const T* tab, const T* v, T* S) {
  const int n1 = L.n[1], n2 = L.n[2], c1 = L.c[1], c2 = L.c[2];
  const AxS<T> a1 = axis_smem(tab, L.toff[1], n1, c1);
  const AxS<T> a2 = axis_smem(tab, L.toff[2], n2, c2);
  const int items = L.n[0] * c2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int j0 = fdiv(it, L.dc2), k2 = it - j0 * c2;
    const int p2 = cpos(k2, n2);
    int jc[5];
    T wc[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const int jj = p2 + o - 2;
      const bool in = jj >= 0 && jj < n2;
      jc[o] = in ? jj : p2;
      wc[o] = in ? a2.rw[5 * k2 + o] : T(0);
    }
    const T* plane = v + j0 * n1 * n2;
    auto rowsum = [&](int j1) -> T {
      if (j1 < 0 || j1 >= n1) return T(0);
      const T* r = plane + j1 * n2;
      return (wc[0] * r[jc[0]] + wc[1] * r[jc[1]]) + (wc[2] * r[jc[2]] + (wc[3] * r[jc[3]] + wc[4] * r[jc[4]]));
    };
    T w0 = T(0), w1 = T(0), w2 = rowsum(0), w3 = rowsum(1), w4 = rowsum(2);
    int p = 0;
    T* out = S + j0 * c1 * c2 + k2;
    for (int k1 = 0; k1 < c1; ++k1) {
      if (k1 > 0) {
        const int pn = cpos(k1, n1);
        if (pn - p == 2) {
          w0 = w2; w1 = w3; w2 = w4;
          w3 = rowsum(pn + 1);
          w4 = rowsum(pn + 2);
        } else {
          w0 = w1; w1 = w2; w2 = w3; w3 = w4;
          w4 = rowsum(pn + 2);
        }
        p = pn;
      }
      const T* r1 = a1.rw + 5 * k1;
      out[k1 * c2] = (r1[0] * w0 + r1[1] * w1) + (r1[2] * w2 + (r1[3] * w3 + r1[4] * w4));
    }
  }
}

// Load vector, second pass: F[k0][k1][k2] = sum_a R0[k0][a] S[cpos(k0) + a - 2]
// - sum_d X0[k0][d] E[k0 - 1 + d], with E[k] = sum X1 X2 of v on the nodal
// positions of nodal plane k.  A thread walks one coarse (k1, k2) column
// along axis 0 and writes F[k0 - 1] over S once F[k0] is formed: every
// later step reads planes of S above cpos(k0) + 2 >= k0 only.
template <typename T>
__device__ void lv_planes(const SmallLevel& L, const T* tab, const T* v, T* SF) {
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  const int c0 = L.c[0], c1 = L.c[1], c2 = L.c[2];
  const AxS<T> a0 = axis_smem(tab, L.toff[0], n0, c0);
  const AxS<T> a1 = axis_smem(tab, L.toff[1], n1, c1);
  const AxS<T> a2 = axis_smem(tab, L.toff[2], n2, c2);
  const int items = c1 * c2, cs = c1 * c2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int k1 = fdiv(it, L.dc2), k2 = it - k1 * c2;
    int o1[3], o2[3];
    T x1[3], x2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int q1 = k1 - 1 + d, q2 = k2 - 1 + d;
      const bool in1 = q1 >= 0 && q1 < c1, in2 = q2 >= 0 && q2 < c2;
      o1[d] = cpos(in1 ? q1 : k1, n1) * n2;
      x1[d] = in1 ? a1.x[3 * k1 + d] : T(0);
      o2[d] = cpos(in2 ? q2 : k2, n2);
      x2[d] = in2 ? a2.x[3 * k2 + d] : T(0);
    }
    auto E = [&](int k) -> T {
      if (k < 0 || k >= c0) return T(0);
      const T* pl = v + cpos(k, n0) * n1 * n2;
      T s = T(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T* r = pl + o1[b];
        s += x1[b] * (x2[0] * r[o2[0]] + x2[1] * r[o2[1]] + x2[2] * r[o2[2]]);
      }
      return s;
    };
    T* col = SF + k1 * c2 + k2;
    auto sval = [&](int j0) -> T { return (j0 >= 0 && j0 < n0) ? col[j0 * cs] : T(0); };
    T w0 = T(0), w1 = T(0), w2 = sval(0), w3 = sval(1), w4 = sval(2);
    T em = T(0), e0 = E(0), ep = E(1);
    int p = 0;
    T prev = T(0);
    for (int k0 = 0; k0 < c0; ++k0) {
      if (k0 > 0) {
        const int pn = cpos(k0, n0);
        if (pn - p == 2) {
          w0 = w2; w1 = w3; w2 = w4;
          w3 = sval(pn + 1);
          w4 = sval(pn + 2);
        } else {
          w0 = w1; w1 = w2; w2 = w3; w3 = w4;
          w4 = sval(pn + 2);
        }
        p = pn;
        em = e0; e0 = ep;
        ep = E(k0 + 1);
      }
      const T* r0 = a0.rw + 5 * k0;
      const T* xx = a0.x + 3 * k0;
      const T f = ((r0[0] * w0 + r0[1] * w1) + (r0[2] * w2 + (r0[3] * w3 + r0[4] * w4))) -
                  (xx[0] * em + xx[1] * e0 + xx[2] * ep);
      if (k0 > 0) col[(k0 - 1) * cs] = prev;
      prev = f;
    }
    col[(c0 - 1) * cs] = prev;
  }
}

// Thomas solves of M_c along every axis of F (one thread per line); values
// and factors are read eight rows ahead of each recurrence.
template <typename T>
__device__ void solves_small(const SmallLevel& L, const T* tab, T* F) {
  const int c0 = L.c[0], c1 = L.c[1], c2 = L.c[2];
  for (int a = 2; a >= 0; --a) {
    if (L.n[a] > 1) {
      const int nc = L.c[a];
      const AxS<T> ax = axis_smem(tab, L.toff[a], L.n[a], nc);
      const int stride = a == 2 ? 1 : a == 1 ? c2 : c1 * c2;
      const int lines = a == 2 ? c0 * c1 : a == 1 ? c0 * c2 : c1 * c2;
      for (int line = threadIdx.x; line < lines; line += blockDim.x) {
        int base;
        if (a == 2) {
          base = line * c2;
        } else if (a == 1) {
          const int k0 = fdiv(line, L.dc2);
          base = k0 * c1 * c2 + (line - k0 * c2);
        } else {
          base = line;
        }
        T* l = F + base;
        T y = T(0);
        for (int k0 = 0; k0 < nc; k0 += 8) {
          T f[8], ta[8], tm[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = min(k0 + u, nc - 1);
            f[u] = l[k * stride];
            ta[u] = ax.ta[k];
            tm[u] = ax.tm[k];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (k0 + u < nc) {
              y = (f[u] - ta[u] * y) * tm[u];
              l[(k0 + u) * stride] = y;
            }
        }
        T x = T(0);
        for (int k0 = nc - 1; k0 >= 0; k0 -= 8) {
          T yv[8], tc[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = max(k0 - u, 0);
            yv[u] = l[k * stride];
            tc[u] = ax.tc[k];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (k0 - u >= 0) {
              x = yv[u] - tc[u] * x;
              l[(k0 - u) * stride] = x;
            }
        }
      }
    }
    __syncthreads();
  }
}

// Coefficients (decomposition: v -= Pi(v_c) off the nodal positions) or
// interpolation (recomposition: v += Pi(c) off them, v = c on them) for one
// level.  An item is a fine row (j0, j1) and a coarse column k2: the nodal
// column cpos(k2) and, when it is a coefficient column, 2 k2 + 1.  The
// corners are v's nodal positions (decomposition; never written here) or the
// coarse grid G (recomposition).
template <typename T, bool DEC>
__device__ void interp_pass(const SmallLevel& L, const T* tab, T* v, const T* G) {
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  const int c0 = L.c[0], c1 = L.c[1], c2 = L.c[2];
  const AxS<T> a0 = axis_smem(tab, L.toff[0], n0, c0);
  const AxS<T> a1 = axis_smem(tab, L.toff[1], n1, c1);
  const AxS<T> a2 = axis_smem(tab, L.toff[2], n2, c2);
  const int items = n0 * n1 * c2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = fdiv(it, L.dc2), k2 = it - q * c2;
    const int j0 = fdiv(q, L.dn1), j1 = q - j0 * n1;
    const bool q0 = is_coef(j0, n0), q1 = is_coef(j1, n1);
    const int kl0 = q0 ? (j0 >> 1) : nodal_k(j0, n0, c0), kr0 = q0 ? kl0 + 1 : kl0;
    const int kl1 = q1 ? (j1 >> 1) : nodal_k(j1, n1, c1), kr1 = q1 ? kl1 + 1 : kl1;
    const int jc = 2 * k2 + 1;
    const bool hasc = jc < n2 - 1;  // odd and inside the row: a coefficient column
    const int k2r = hasc ? k2 + 1 : k2;
    int rll, rlr, rrl, rrr, cl, cr;
    if (DEC) {
      const int pl0 = cpos(kl0, n0) * n1, pr0 = cpos(kr0, n0) * n1;
      const int pl1 = cpos(kl1, n1), pr1 = cpos(kr1, n1);
      rll = (pl0 + pl1) * n2; rlr = (pl0 + pr1) * n2;
      rrl = (pr0 + pl1) * n2; rrr = (pr0 + pr1) * n2;
      cl = cpos(k2, n2); cr = cpos(k2r, n2);
    } else {
      rll = (kl0 * c1 + kl1) * c2; rlr = (kl0 * c1 + kr1) * c2;
      rrl = (kr0 * c1 + kl1) * c2; rrr = (kr0 * c1 + kr1) * c2;
      cl = k2; cr = k2r;
    }
    const T* cv = DEC ? v : G;
    const T vll = cv[rll + cl], vlr = cv[rlr + cl], vrl = cv[rrl + cl], vrr = cv[rrr + cl];
    const T ull = cv[rll + cr], ulr = cv[rlr + cr], url = cv[rrl + cr], urr = cv[rrr + cr];
    const T wl0 = q0 ? a0.iwl[j0] : T(1), wr0 = q0 ? a0.iwr[j0] : T(0);
    const T wl1 = q1 ? a1.iwl[j1] : T(1), wr1 = q1 ? a1.iwr[j1] : T(0);
    auto lerp01 = [&](T ll, T lr, T rl, T rr) -> T {
      const T a = q1 ? wl1 * ll + wr1 * lr : ll;
      const T b = q1 ? wl1 * rl + wr1 * rr : rl;
      return q0 ? wl0 * a + wr0 * b : a;
    };
    const T rl = lerp01(vll, vlr, vrl, vrr);
    T* row = v + (j0 * n1 + j1) * n2;
    const int jn = cpos(k2, n2);
    if (q0 || q1) {
      if (DEC) row[jn] -= rl;
      else row[jn] += rl;
    } else if (!DEC) {
      row[jn] = rl;
    }
    if (hasc) {
      const T rr = lerp01(ull, ulr, url, urr);
      const T pv = a2.iwl[jc] * rl + a2.iwr[jc] * rr;
      if (DEC) row[jc] -= pv;
      else row[jc] += pv;
    }
  }
}

// The nodal positions of a fine grid (n) and its coarse grid (c): element k
// of the coarse grid and the fine element it sits on.
__device__ __forceinline__ int nodal_index(const SmallLevel& L, int k) {
  const int q = fdiv(k, L.dc2), k2 = k - q * L.c[2];
  const int k0 = fdiv(q, L.dc1), k1 = q - k0 * L.c[1];
  return (cpos(k0, L.n[0]) * L.n[1] + cpos(k1, L.n[1])) * L.n[2] + cpos(k2, L.n[2]);
}

template <typename T, bool DEC>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512, 1)
small_levels_kernel(const __grid_constant__ SmallParams<T> sp, int nlev, T* __restrict__ data) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const T* tab = sm;
  T* top = sm + sp.goff[nlev];
  const int ntop = sp.ntop;
  // Every table and the highest grid through asynchronous copies, all in
  // flight at once.
  for (int s = threadIdx.x >> 5; s < sp.nseg; s += blockDim.x >> 5) {
    const SmallSeg<T> g = sp.seg[s];
    for (int e = threadIdx.x & 31; e < g.count; e += 32) cp_async_elem(sm + g.dst + e, g.src + e);
  }
  constexpr int VEC = 16 / sizeof(T);
  const bool aligned = (reinterpret_cast<uintptr_t>(data) & 15) == 0;
  const int nv = aligned ? ntop / VEC : 0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cp_async_16(top + i * VEC, data + i * VEC);
  for (int i = nv * VEC + threadIdx.x; i < ntop; i += blockDim.x) cp_async_elem(top + i, data + i);
  cp_async_wait_all();
  __syncthreads();

  T* SF = sm + sp.boff;
  if (DEC) {
    for (int i = nlev - 1; i >= 0; --i) {
      const SmallLevel& L = sp.lv[i];
      T* v = sm + sp.goff[i + 1];
      T* G = sm + sp.goff[i];
      lv_rows(L, tab, v, SF);
      __syncthreads();
      lv_planes(L, tab, v, SF);
      __syncthreads();
      solves_small(L, tab, SF);
      const int nc = L.c[0] * L.c[1] * L.c[2];
      for (int k = threadIdx.x; k < nc; k += blockDim.x) G[k] = v[nodal_index(L, k)] + SF[k];
      interp_pass<T, true>(L, tab, v, G);
      __syncthreads();
    }
    // Final coarse values into the nodal positions, coarsest first.
    for (int i = 0; i < nlev; ++i) {
      const SmallLevel& L = sp.lv[i];
      const T* G = sm + sp.goff[i];
      T* v = sm + sp.goff[i + 1];
      const int nc = L.c[0] * L.c[1] * L.c[2];
      for (int k = threadIdx.x; k < nc; k += blockDim.x) v[nodal_index(L, k)] = G[k];
      __syncthreads();
    }
  } else {
    // Coarse grids from the nodal positions, finest first.
    for (int i = nlev - 1; i >= 0; --i) {
      const SmallLevel& L = sp.lv[i];
      const T* v = sm + sp.goff[i + 1];
      T* G = sm + sp.goff[i];
      const int nc = L.c[0] * L.c[1] * L.c[2];
      for (int k = threadIdx.x; k < nc; k += blockDim.x) G[k] = v[nodal_index(L, k)];
      __syncthreads();
    }
    for (int i = 0; i < nlev; ++i) {
      const SmallLevel& L = sp.lv[i];
      T* v = sm + sp.goff[i + 1];
      T* G = sm + sp.goff[i];
      lv_rows(L, tab, v, SF);
      __syncthreads();
      lv_planes(L, tab, v, SF);
      __syncthreads();
      solves_small(L, tab, SF);
      const int nc = L.c[0] * L.c[1] * L.c[2];
      for (int k = threadIdx.x; k < nc; k += blockDim.x) G[k] -= SF[k];
      __syncthreads();
      interp_pass<T, false>(L, tab, v, G);
      __syncthreads();
    }
  }
  if (aligned) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const V* src = reinterpret_cast<const V*>(top);
    V* dst = reinterpret_cast<V*>(data);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = src[i];
  }
  for (int i = nv * VEC + threadIdx.x; i < ntop; i += blockDim.x) data[i] = top[i];
}

// Shared-memory layout (elements of T): every axis table block, the coarse
// grids G[0 .. nlev - 1], the load-vector scratch (n0 c1 c2 of the largest
// transition, which also holds F), then the highest grid on a 16-byte
// boundary.  Fills `sp` when given; returns the bytes.
template <typename T>
size_t small_layout(const LevelK<T>* lv, int nlev, bool dec, SmallParams<T>* sp) {
  constexpr int VEC = 16 / sizeof(T);
  auto up = [](size_t x) { return (x + VEC - 1) / VEC * VEC; };
  size_t off = 0;
  int nseg = 0;
  for (int i = 0; i < nlev; ++i)
    for (int a = 0; a < 3; ++a) {
      const AxisK<T>& ax = lv[i].ax[a];
      const int n = ax.n, nc = ax.nc;
      if (sp) {
        sp->lv[i].toff[a] = static_cast<int>(off);
        const T* src[kTabArrays] = {ax.iwl, ax.iwr, ax.rw, dec ? ax.xd : ax.xr, ax.ta, ax.tm, ax.tc};
        const int cnt[kTabArrays] = {n, n, 5 * nc, 3 * nc, nc, nc, nc};
        int d = static_cast<int>(off);
        for (int t = 0; t < kTabArrays; ++t) {
          if (src[t] != nullptr && cnt[t] > 0) sp->seg[nseg++] = SmallSeg<T>{src[t], d, cnt[t]};
          d += cnt[t];
        }
      }
      off += axis_table_size(n, nc);
    }
  off = up(off);
  size_t scratch = 0;
  for (int i = 0; i < nlev; ++i) {
    const LevelK<T>& L = lv[i];
    if (sp) {
      SmallLevel& s = sp->lv[i];
      for (int a = 0; a < 3; ++a) {
        s.n[a] = L.ax[a].n;
        s.c[a] = L.ax[a].nc;
      }
      s.dc2 = make_fastdiv(L.ax[2].nc);
      s.dc1 = make_fastdiv(L.ax[1].nc);
      s.dn1 = make_fastdiv(L.ax[1].n);
      sp->goff[i] = static_cast<int>(off);
    }
    off += size_t(L.ax[0].nc) * L.ax[1].nc * L.ax[2].nc;
    scratch = std::max(scratch, size_t(L.ax[0].n) * L.ax[1].nc * L.ax[2].nc);
  }
  off = up(off);
  if (sp) sp->boff = static_cast<int>(off);
  off = up(off + scratch);
  const LevelK<T>& Lt = lv[nlev - 1];
  const size_t ntop = size_t(Lt.ax[0].n) * Lt.ax[1].n * Lt.ax[2].n;
  if (sp) {
    sp->goff[nlev] = static_cast<int>(off);
    sp->ntop = static_cast<int>(ntop);
    sp->nseg = nseg;
  }
  off += ntop;
  return sizeof(T) * off;
}

}  // namespace

template <typename T>
size_t small_levels_smem(const LevelK<T>* lv, int nlev) {
  return small_layout<T>(lv, nlev, true, nullptr);
}

template <typename T>
cudaError_t launch_small_levels(const LevelK<T>* lv, int nlev, bool dec, T* data, int level,
                                cudaStream_t s) {
  if (nlev < 1 || nlev > kSmallMaxLevels) return cudaErrorInvalidValue;
  SmallParams<T> sp{};
  const size_t smem = small_layout<T>(lv, nlev, dec, &sp);
  // The multiply-high divisions are exact for every index of these grids.
  if (sp.ntop > kSmallMaxNodes) return cudaErrorInvalidValue;
  TraceScope ts(kKSmallLevels, level, 2.0 * sizeof(T) * double(sp.ntop), s);
  auto kernel = dec ? small_levels_kernel<T, true> : small_levels_kernel<T, false>;
  allow_dynamic_smem(kernel, smem);
  launch_pdl(kernel, dim3(1), dim3(small_threads<T>()), smem, s, sp, nlev, data);
  return cudaGetLastError();
}

template size_t small_levels_smem<float>(const LevelK<float>*, int);
template size_t small_levels_smem<double>(const LevelK<double>*, int);
template cudaError_t launch_small_levels<float>(const LevelK<float>*, int, bool, float*, int,
                                                cudaStream_t);
template cudaError_t launch_small_levels<double>(const LevelK<double>*, int, bool, double*, int,
                                                 cudaStream_t);

}  // namespace mgb
