// The coarsest levels of a transform in one CTA.  Below a few tens of
// thousands of nodes every per-level kernel is a handful of CTAs whose cost
// is launch and latency; here one CTA of 1024 threads loads the grid of the
// highest small level into shared memory, runs the whole decomposition (or
// recomposition) of the levels below it there, and writes the grid back.
//
// Per level transition (tables of the level, Section 2):
//   decomposition : F = R v - (R P) v_c (the load vector, by a direct 5-tap
//                   tensor stencil per coarse node), Thomas solves along each
//                   axis, coarse values v_c + z, coefficients v - Pi(v_c);
//                   after the coarsest level the final coarse values go back
//                   into the nodal positions, coarsest first;
//   recomposition : the coarse grids are gathered from the nodal positions
//                   first; then, coarsest first, F = R w - (R S) w_c, the
//                   solves, c' = Q u - z, and the grid becomes Pi(c') plus the
//                   coefficients.
// These are the same operators as the per-level kernels; only the order of
// the rounding differs.
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
#include "grid.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

constexpr int kSmallThreads = 512;

template <typename T>
struct SmallLevels {
  LevelK<T> lv[kSmallMaxLevels];  // lv[i]: transition of level stop + 1 + i
};

__device__ __forceinline__ int grid_size(const int n[3]) { return n[0] * n[1] * n[2]; }

// F = R v - X v_c on the coarse grid of one transition; v is the fine grid,
// v_c its values on the coarse nodes (read from the nodal positions of v).
// Tap positions are clamped into the grid under zero weights, so every load
// of a node is unconditional and a thread's loads pipeline.
template <typename T>
__device__ void load_vector_small(const LevelK<T>& L, bool dec, const T* v, T* F) {
  const int n1 = L.ax[1].n, n2 = L.ax[2].n;
  const int c1 = L.ax[1].nc, c2 = L.ax[2].nc;
  const int nco = L.ax[0].nc * c1 * c2;
  for (int idx = threadIdx.x; idx < nco; idx += blockDim.x) {
    const int k2 = idx % c2, k01 = idx / c2, k1 = k01 % c1, k0 = k01 / c1;
    const int kk[3] = {k0, k1, k2};
    int j[3][5], q[3][3];
    T w[3][5], x[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const AxisK<T>& ax = L.ax[a];
      const int n = ax.n, nc = ax.nc, k = kk[a], p = cpos(k, n);
      const T* X = dec ? ax.xd : ax.xr;
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int jj = p + o - 2;
        const bool in = jj >= 0 && jj < n;
        j[a][o] = in ? jj : p;
        w[a][o] = in ? __ldg(ax.rw + 5 * k + o) : T(0);
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int qq = k - 1 + d;
        const bool in = qq >= 0 && qq < nc;
        q[a][d] = cpos(in ? qq : k, n);
        x[a][d] = in ? __ldg(X + 3 * k + d) : T(0);
      }
    }
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      T s1 = T(0);
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const T* row = v + (j[0][a] * n1 + j[1][b]) * n2;
        s1 += w[1][b] * ((w[2][0] * row[j[2][0]] + w[2][1] * row[j[2][1]]) +
                         (w[2][2] * row[j[2][2]] + (w[2][3] * row[j[2][3]] + w[2][4] * row[j[2][4]])));
      }
      acc += w[0][a] * s1;
    }
    T xs = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T s1 = T(0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T* row = v + (q[0][a] * n1 + q[1][b]) * n2;
        s1 += x[1][b] * (x[2][0] * row[q[2][0]] + x[2][1] * row[q[2][1]] + x[2][2] * row[q[2][2]]);
      }
      xs += x[0][a] * s1;
    }
    F[idx] = acc - xs;
  }
}

// Thomas solves of M_c along every axis of the coarse grid F (one thread
// per line); values and factors are read eight rows ahead of each
// recurrence, so the chain waits on arithmetic rather than on loads.
template <typename T>
__device__ void solves_small(const LevelK<T>& L, T* F) {
  const int c[3] = {L.ax[0].nc, L.ax[1].nc, L.ax[2].nc};
  for (int a = 2; a >= 0; --a) {
    const AxisK<T>& ax = L.ax[a];
    const int nc = c[a];
    if (L.ax[a].n > 1) {
      const int stride = a == 2 ? 1 : a == 1 ? c[2] : c[1] * c[2];
      const int lines = (c[0] * c[1] * c[2]) / nc;
      for (int line = threadIdx.x; line < lines; line += blockDim.x) {
        // Line index -> (outer, inner) around the solved axis.
        const int inner = line % stride, outer = line / stride;
        T* l = F + outer * nc * stride + inner;
        T y = T(0);
        for (int k0 = 0; k0 < nc; k0 += 8) {
          T f[8], ta[8], tm[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = min(k0 + u, nc - 1);
            f[u] = l[k * stride];
            ta[u] = __ldg(ax.ta + k);
            tm[u] = __ldg(ax.tm + k);
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
            tc[u] = __ldg(ax.tc + k);
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

// Multilinear interpolation at fine node (j0, j1, j2) from coarse values
// `cv` (coarse grid layout, or, with from_fine, the nodal positions of the
// fine grid `cv`): always the 8 corners (a nodal axis repeats its node under
// weights 1 and 0, which passes the value unrounded), all loads issued
// before the arithmetic.
template <typename T>
__device__ __forceinline__ T interp_small(const LevelK<T>& L, const T* cv, bool from_fine, int j0,
                                          int j1, int j2) {
  const int j[3] = {j0, j1, j2};
  int kl[3], kr[3];
  T wl[3], wr[3];
  bool q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const AxisK<T>& ax = L.ax[a];
    q[a] = is_coef(j[a], ax.n);
    kl[a] = q[a] ? (j[a] >> 1) : nodal_k(j[a], ax.n, ax.nc);
    kr[a] = q[a] ? kl[a] + 1 : kl[a];
    wl[a] = q[a] ? __ldg(ax.iwl + j[a]) : T(1);
    wr[a] = q[a] ? __ldg(ax.iwr + j[a]) : T(0);
    if (from_fine) {
      kl[a] = cpos(kl[a], ax.n);
      kr[a] = cpos(kr[a], ax.n);
    }
  }
  const int m1 = from_fine ? L.ax[1].n : L.ax[1].nc, m2 = from_fine ? L.ax[2].n : L.ax[2].nc;
  auto at = [&](int a0, int a1, int a2) { return cv[(a0 * m1 + a1) * m2 + a2]; };
  const T v000 = at(kl[0], kl[1], kl[2]), v001 = at(kl[0], kl[1], kr[2]);
  const T v010 = at(kl[0], kr[1], kl[2]), v011 = at(kl[0], kr[1], kr[2]);
  const T v100 = at(kr[0], kl[1], kl[2]), v101 = at(kr[0], kl[1], kr[2]);
  const T v110 = at(kr[0], kr[1], kl[2]), v111 = at(kr[0], kr[1], kr[2]);
  auto r2 = [&](T a, T b) { return q[2] ? wl[2] * a + wr[2] * b : a; };
  auto r1 = [&](T a, T b) { return q[1] ? wl[1] * a + wr[1] * b : a; };
  const T a0 = r1(r2(v000, v001), r2(v010, v011));
  const T a1 = r1(r2(v100, v101), r2(v110, v111));
  return q[0] ? wl[0] * a0 + wr[0] * a1 : a0;
}

template <typename T, bool DEC>
__global__ void __launch_bounds__(kSmallThreads)
small_levels_kernel(SmallLevels<T> sl, int nlev, T* __restrict__ data) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* base = reinterpret_cast<T*>(smem_raw);
  // Grids G[i], i = 0..nlev (G[nlev] the top), then the load-vector scratch.
  T* G[kSmallMaxLevels + 1];
  int gsz[kSmallMaxLevels + 1];
  {
    size_t off = 0;
    for (int i = 0; i <= nlev; ++i) {
      const LevelK<T>& L = sl.lv[i < nlev ? i : nlev - 1];
      const int d[3] = {i < nlev ? L.ax[0].nc : L.ax[0].n, i < nlev ? L.ax[1].nc : L.ax[1].n,
                        i < nlev ? L.ax[2].nc : L.ax[2].n};
      gsz[i] = grid_size(d);
      G[i] = base + off;
      off += gsz[i];
    }
    base += off;
  }
  T* Ft = base;
  const int ntop = gsz[nlev];
  // Eight loads of a thread in flight at a time (one CTA moves the grid).
  for (int i0 = threadIdx.x; i0 < ntop; i0 += 8 * blockDim.x) {
    T t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      t[u] = i < ntop ? data[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < ntop) G[nlev][i] = t[u];
    }
  }
  __syncthreads();
  if (DEC) {
    for (int i = nlev - 1; i >= 0; --i) {
      const LevelK<T>& L = sl.lv[i];
      T* v = G[i + 1];
      const int n0 = L.ax[0].n, n1 = L.ax[1].n, n2 = L.ax[2].n;
      const int c1 = L.ax[1].nc, c2 = L.ax[2].nc;
      load_vector_small(L, true, v, Ft);
      __syncthreads();
      solves_small(L, Ft);
      for (int k = threadIdx.x; k < gsz[i]; k += blockDim.x) {
        const int k2 = k % c2, k1 = (k / c2) % c1, k0 = k / (c1 * c2);
        G[i][k] = v[(cpos(k0, n0) * n1 + cpos(k1, n1)) * n2 + cpos(k2, n2)] + Ft[k];
      }
      // Coefficients from the (unchanged) nodal values of v.
      for (int x = threadIdx.x; x < gsz[i + 1]; x += blockDim.x) {
        const int j2 = x % n2, j1 = (x / n2) % n1, j0 = x / (n1 * n2);
        if (is_coef(j0, n0) || is_coef(j1, n1) || is_coef(j2, n2))
          v[x] -= interp_small(L, v, true, j0, j1, j2);
      }
      __syncthreads();
    }
    // Final coarse values into the nodal positions, coarsest first.
    for (int i = 0; i < nlev; ++i) {
      const LevelK<T>& L = sl.lv[i];
      const int n0 = L.ax[0].n, n1 = L.ax[1].n, n2 = L.ax[2].n;
      const int c1 = L.ax[1].nc, c2 = L.ax[2].nc;
      for (int k = threadIdx.x; k < gsz[i]; k += blockDim.x) {
        const int k2 = k % c2, k1 = (k / c2) % c1, k0 = k / (c1 * c2);
        G[i + 1][(cpos(k0, n0) * n1 + cpos(k1, n1)) * n2 + cpos(k2, n2)] = G[i][k];
      }
      __syncthreads();
    }
  } else {
    // Coarse grids from the nodal positions, finest first.
    for (int i = nlev - 1; i >= 0; --i) {
      const LevelK<T>& L = sl.lv[i];
      const int n0 = L.ax[0].n, n1 = L.ax[1].n, n2 = L.ax[2].n;
      const int c1 = L.ax[1].nc, c2 = L.ax[2].nc;
      for (int k = threadIdx.x; k < gsz[i]; k += blockDim.x) {
        const int k2 = k % c2, k1 = (k / c2) % c1, k0 = k / (c1 * c2);
        G[i][k] = G[i + 1][(cpos(k0, n0) * n1 + cpos(k1, n1)) * n2 + cpos(k2, n2)];
      }
      __syncthreads();
    }
    for (int i = 0; i < nlev; ++i) {
      const LevelK<T>& L = sl.lv[i];
      T* v = G[i + 1];
      const int n0 = L.ax[0].n, n1 = L.ax[1].n, n2 = L.ax[2].n;
      const int c1 = L.ax[1].nc, c2 = L.ax[2].nc;
      load_vector_small(L, false, v, Ft);
      __syncthreads();
      solves_small(L, Ft);
      for (int k = threadIdx.x; k < gsz[i]; k += blockDim.x) G[i][k] -= Ft[k];
      __syncthreads();
      for (int x = threadIdx.x; x < gsz[i + 1]; x += blockDim.x) {
        const int j2 = x % n2, j1 = (x / n2) % n1, j0 = x / (n1 * n2);
        if (is_coef(j0, n0) || is_coef(j1, n1) || is_coef(j2, n2)) {
          v[x] += interp_small(L, G[i], false, j0, j1, j2);
        } else {
          const int k0 = nodal_k(j0, n0, L.ax[0].nc), k1 = nodal_k(j1, n1, c1);
          v[x] = G[i][(k0 * c1 + k1) * c2 + nodal_k(j2, n2, c2)];
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < ntop; i += blockDim.x) data[i] = G[nlev][i];
}

}  // namespace

template <typename T>
size_t small_levels_smem(const LevelK<T>* lv, int nlev) {
  // Grids of every level (coarsest .. top) and one coarse-sized scratch.
  size_t total = 0, maxc = 0;
  for (int i = 0; i < nlev; ++i) {
    const size_t c = size_t(lv[i].ax[0].nc) * lv[i].ax[1].nc * lv[i].ax[2].nc;
    total += c;
    maxc = std::max(maxc, c);
  }
  total += size_t(lv[nlev - 1].ax[0].n) * lv[nlev - 1].ax[1].n * lv[nlev - 1].ax[2].n;
  return sizeof(T) * (total + maxc);
}

template <typename T>
cudaError_t launch_small_levels(const LevelK<T>* lv, int nlev, bool dec, T* data, int level,
                                cudaStream_t s) {
  if (nlev < 1 || nlev > kSmallMaxLevels) return cudaErrorInvalidValue;
  SmallLevels<T> sl{};
  for (int i = 0; i < nlev; ++i) sl.lv[i] = lv[i];
  const size_t smem = small_levels_smem(lv, nlev);
  const size_t ntop = size_t(lv[nlev - 1].ax[0].n) * lv[nlev - 1].ax[1].n * lv[nlev - 1].ax[2].n;
  TraceScope ts(kKSmallLevels, level, 2.0 * sizeof(T) * double(ntop), s);
  auto kernel = dec ? small_levels_kernel<T, true> : small_levels_kernel<T, false>;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  launch_pdl(kernel, dim3(1), dim3(kSmallThreads), smem, s, sl, nlev, data);
  return cudaGetLastError();
}

template size_t small_levels_smem<float>(const LevelK<float>*, int);
template size_t small_levels_smem<double>(const LevelK<double>*, int);
template cudaError_t launch_small_levels<float>(const LevelK<float>*, int, bool, float*, int,
                                                cudaStream_t);
template cudaError_t launch_small_levels<double>(const LevelK<double>*, int, bool, double*, int,
                                                 cudaStream_t);

}  // namespace mgb
