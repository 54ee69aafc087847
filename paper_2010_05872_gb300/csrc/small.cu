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

constexpr int kSmallThreads = 1024;

template <typename T>
struct SmallLevels {
  LevelK<T> lv[kSmallMaxLevels];  // lv[i]: transition of level stop + 1 + i
};

__device__ __forceinline__ int grid_size(const int n[3]) { return n[0] * n[1] * n[2]; }

// F = R v - X v_c on the coarse grid of one transition; v is the fine grid,
// v_c its values on the coarse nodes (read from the nodal positions of v).
template <typename T>
__device__ void load_vector_small(const LevelK<T>& L, bool dec, const T* v, T* F) {
  const int n0 = L.ax[0].n, n1 = L.ax[1].n, n2 = L.ax[2].n;
  const int c0 = L.ax[0].nc, c1 = L.ax[1].nc, c2 = L.ax[2].nc;
  const T* X0 = dec ? L.ax[0].xd : L.ax[0].xr;
  const T* X1 = dec ? L.ax[1].xd : L.ax[1].xr;
  const T* X2 = dec ? L.ax[2].xd : L.ax[2].xr;
  const int nco = c0 * c1 * c2;
  for (int idx = threadIdx.x; idx < nco; idx += blockDim.x) {
    const int k2 = idx % c2, k1 = (idx / c2) % c1, k0 = idx / (c1 * c2);
    const int p0 = cpos(k0, n0), p1 = cpos(k1, n1), p2 = cpos(k2, n2);
    T r0[5], r1[5], r2[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      r0[o] = __ldg(L.ax[0].rw + 5 * k0 + o);
      r1[o] = __ldg(L.ax[1].rw + 5 * k1 + o);
      r2[o] = __ldg(L.ax[2].rw + 5 * k2 + o);
    }
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const int j0 = p0 + a - 2;
      if (j0 < 0 || j0 >= n0) continue;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const int j1 = p1 + b - 2;
        if (j1 < 0 || j1 >= n1) continue;
        const T* row = v + (j0 * n1 + j1) * n2;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const int j2 = p2 + c - 2;
          if (j2 >= 0 && j2 < n2) s += r2[c] * row[j2];
        }
        acc += r0[a] * r1[b] * s;
      }
    }
    T xs = T(0);
    for (int d0 = 0; d0 < 3; ++d0) {
      const int q0 = k0 - 1 + d0;
      if (q0 < 0 || q0 >= c0) continue;
      const T w0 = __ldg(X0 + 3 * k0 + d0);
      for (int d1 = 0; d1 < 3; ++d1) {
        const int q1 = k1 - 1 + d1;
        if (q1 < 0 || q1 >= c1) continue;
        const T w01 = w0 * __ldg(X1 + 3 * k1 + d1);
        const T* row = v + (cpos(q0, n0) * n1 + cpos(q1, n1)) * n2;
        for (int d2 = 0; d2 < 3; ++d2) {
          const int q2 = k2 - 1 + d2;
          if (q2 >= 0 && q2 < c2) xs += w01 * __ldg(X2 + 3 * k2 + d2) * row[cpos(q2, n2)];
        }
      }
    }
    F[idx] = acc - xs;
  }
}

// Thomas solves of M_c along every axis of the coarse grid F (one thread
// per line).
template <typename T>
__device__ void solves_small(const LevelK<T>& L, T* F) {
  const int c[3] = {L.ax[0].nc, L.ax[1].nc, L.ax[2].nc};
  for (int a = 2; a >= 0; --a) {
    const AxisK<T>& ax = L.ax[a];
    const int nc = c[a];
    const int stride = a == 2 ? 1 : a == 1 ? c[2] : c[1] * c[2];
    const int lines = (c[0] * c[1] * c[2]) / nc;
    for (int line = threadIdx.x; line < lines; line += blockDim.x) {
      // Line index -> (outer, inner) around the solved axis.
      const int inner = line % stride, outer = line / stride;
      T* l = F + outer * nc * stride + inner;
      T y = T(0);
      for (int k = 0; k < nc; ++k) {
        y = (l[k * stride] - __ldg(ax.ta + k) * y) * __ldg(ax.tm + k);
        l[k * stride] = y;
      }
      T x = T(0);
      for (int k = nc - 1; k >= 0; --k) {
        x = l[k * stride] - __ldg(ax.tc + k) * x;
        l[k * stride] = x;
      }
    }
    __syncthreads();
  }
}

// Multilinear interpolation at fine node (j0, j1, j2) from coarse values
// `cv` (coarse grid layout, or, with from_fine, the nodal positions of the
// fine grid `cv`).
template <typename T>
__device__ __forceinline__ T interp_small(const LevelK<T>& L, const T* cv, bool from_fine, int j0,
                                          int j1, int j2) {
  const int n[3] = {L.ax[0].n, L.ax[1].n, L.ax[2].n};
  const int c[3] = {L.ax[0].nc, L.ax[1].nc, L.ax[2].nc};
  const int j[3] = {j0, j1, j2};
  int kl[3], kr[3];
  T wl[3], wr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (is_coef(j[a], n[a])) {
      kl[a] = (j[a] - 1) >> 1;
      kr[a] = kl[a] + 1;
      wl[a] = __ldg(L.ax[a].iwl + j[a]);
      wr[a] = __ldg(L.ax[a].iwr + j[a]);
    } else {
      kl[a] = kr[a] = nodal_k(j[a], n[a], c[a]);
      wl[a] = T(1);
      wr[a] = T(0);
    }
  }
  auto at = [&](int a0, int a1, int a2) -> T {
    if (from_fine) return cv[(cpos(a0, n[0]) * n[1] + cpos(a1, n[1])) * n[2] + cpos(a2, n[2])];
    return cv[(a0 * c[1] + a1) * c[2] + a2];
  };
  T s = T(0);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const T w = ((m & 4) ? wr[0] : wl[0]) * ((m & 2) ? wr[1] : wl[1]) * ((m & 1) ? wr[2] : wl[2]);
    if (w != T(0))
      s += w * at((m & 4) ? kr[0] : kl[0], (m & 2) ? kr[1] : kl[1], (m & 1) ? kr[2] : kl[2]);
  }
  return s;
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
