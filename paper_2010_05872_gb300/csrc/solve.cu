// Batched tridiagonal solves with the coarse mass matrix M_c along every axis
// of a level (Section 2 step 4; Section 5.3 "batched correction computation",
// Section 5.4 precomputed factors): Thomas elimination with the factors of the
// plan, forward y_k = (f_k - a_k y_{k-1}) m_k, backward x_k = y_k - c'_k x_{k+1}.
// The last solve of a level applies its result (correction application).
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

constexpr int kChunk = 8;  // elements of a line loaded together (independent loads)

template <typename T>
__device__ __forceinline__ void apply_x(T* F, T* B, int64_t idx, T x, T old_b, int mode) {
  if (mode == kApplyNone) {
    F[idx] = x;
  } else if (mode == kApplyDecompose) {
    B[idx] = old_b + x;
    F[idx] = old_b;
  } else {
    B[idx] = old_b - x;
  }
}

// Lines along a strided axis: element k of line (outer, inner) sits at
// outer * nc * stride + k * stride + inner.  One thread per line; adjacent
// threads take adjacent `inner`, so every access is a coalesced row access.
// Loads are issued kChunk at a time ahead of the recurrence.
template <typename T>
__global__ void __launch_bounds__(256)
solve_strided_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t outer,
                     int64_t stride, int mode) {
  const int64_t line = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (line >= outer * stride) return;
  const int64_t o = line / stride, in = line - o * stride;
  const int nc = ax.nc;
  T* Fl = F + o * nc * stride + in;
  T* Bl = B ? B + o * nc * stride + in : nullptr;
  T y = T(0);
  for (int k0 = 0; k0 < nc; k0 += kChunk) {
    T f[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      f[j] = (k0 + j < nc) ? Fl[static_cast<int64_t>(k0 + j) * stride] : T(0);
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const int k = k0 + j;
      if (k < nc) {
        y = (f[j] - __ldg(ax.ta + k) * y) * __ldg(ax.tm + k);
        Fl[static_cast<int64_t>(k) * stride] = y;
      }
    }
  }
  T x = T(0);
  for (int k1 = nc - 1; k1 >= 0; k1 -= kChunk) {
    T yv[kChunk], bv[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const int k = k1 - j;
      yv[j] = (k >= 0) ? Fl[static_cast<int64_t>(k) * stride] : T(0);
      bv[j] = (k >= 0 && mode != kApplyNone) ? Bl[static_cast<int64_t>(k) * stride] : T(0);
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const int k = k1 - j;
      if (k >= 0) {
        x = yv[j] - __ldg(ax.tc + k) * x;
        const int64_t idx = static_cast<int64_t>(k) * stride;
        if (mode == kApplyNone) Fl[idx] = x;
        else apply_x(Fl, Bl, idx, x, bv[j], mode);
      }
    }
  }
}

// Lines along the contiguous axis: a CTA stages `rows` whole lines in shared
// memory (threads sweep each line, so loads and stores are coalesced), one
// thread per line solves in place (row pitch nc|1 keeps the threads on
// distinct banks), then the lines go back.
template <typename T>
__global__ void __launch_bounds__(128)
solve_contig_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines, int rows,
                    int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int nc = ax.nc, pitch = nc | 1;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * rows;
  const int64_t left = nlines - first;
  const int nr = static_cast<int>(left < rows ? left : rows);
  // The nr lines are contiguous: stage them as one flat range, 8 loads per
  // thread in flight.  With several lines, nr nc <= 28672 (the launcher's
  // shared-memory budget), so i / nc is exact through (i + 0.5) / nc in FP32:
  // that is at least 1 / (2 nc) from an integer and the estimate is within
  // nr 2^-22 <= 0.007 / nc of it.  A single line needs no division.
  const int total = nr * nc;
  const float inv_nc = 1.0f / static_cast<float>(nc);
  const T* src = F + first * nc;
  for (int base = threadIdx.x; base < total; base += 8 * blockDim.x) {
    T v[8];
    int si[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      si[u] = -1;
      if (i < total) {
        const int r = nr == 1 ? 0 : static_cast<int>((static_cast<float>(i) + 0.5f) * inv_nc);
        si[u] = r * pitch + (i - r * nc);
        v[u] = src[i];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (si[u] >= 0) s[si[u]] = v[u];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    T* l = s + r * pitch;
    T y = T(0);
    for (int k = 0; k < nc; ++k) {
      y = (l[k] - __ldg(ax.ta + k) * y) * __ldg(ax.tm + k);
      l[k] = y;
    }
    T x = T(0);
    for (int k = nc - 1; k >= 0; --k) {
      x = l[k] - __ldg(ax.tc + k) * x;
      l[k] = x;
    }
  }
  __syncthreads();
  T* dstF = F + first * nc;
  T* dstB = B ? B + first * nc : nullptr;
  for (int base = threadIdx.x; base < total; base += 8 * blockDim.x) {
    T bv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      bv[u] = (i < total && mode != kApplyNone) ? dstB[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) {
        const int r = nr == 1 ? 0 : static_cast<int>((static_cast<float>(i) + 0.5f) * inv_nc);
        const T x = s[r * pitch + (i - r * nc)];
        if (mode == kApplyNone) dstF[i] = x;
        else apply_x(dstF, dstB, i, x, bv[u], mode);
      }
    }
  }
}

inline unsigned ceil_div(int64_t a, int64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

}  // namespace

template <typename T>
cudaError_t launch_solves(const LevelK<T>& lv, T* F, T* B, ApplyMode mode, int level,
                          cudaStream_t s) {
  const int64_t c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  int last = 0;
  while (lv.ax[last].n == 1) ++last;  // lowest active axis is solved last
  for (int a = 2; a >= last; --a) {
    const int m = (a == last) ? mode : kApplyNone;
    const double passes = m == kApplyDecompose ? 4.0 : m == kApplyRecompose ? 3.0 : 2.0;
    TraceScope ts(a == 2 ? kKSolveContig : kKSolveStrided, level,
                  sizeof(T) * passes * double(c0) * c1 * c2, s);
    const size_t per_row = sizeof(T) * static_cast<size_t>(c2 | 1);
    if (a == 2 && per_row <= 112 * 1024) {
      const int64_t nlines = c0 * c1;
      int rows = static_cast<int>(std::min<size_t>(128, (112 * 1024) / per_row));
      rows = std::max(rows, 1);
      const size_t smem = per_row * rows;
      cudaFuncSetAttribute(solve_contig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
      solve_contig_kernel<T><<<ceil_div(nlines, rows), 128, smem, s>>>(lv.ax[2], F, B, nlines,
                                                                        rows, m);
    } else {
      // Strided lines; contiguous lines too long for shared memory go here
      // too, as lines of stride 1.
      const int64_t outer = (a == 0) ? 1 : (a == 1) ? c0 : c0 * c1;
      const int64_t stride = (a == 0) ? c1 * c2 : (a == 1) ? c2 : 1;
      solve_strided_kernel<T><<<ceil_div(outer * stride, 256), 256, 0, s>>>(lv.ax[a], F, B, outer,
                                                                            stride, m);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_solves<float>(const LevelK<float>&, float*, float*, ApplyMode, int,
                                          cudaStream_t);
template cudaError_t launch_solves<double>(const LevelK<double>&, double*, double*, ApplyMode, int,
                                           cudaStream_t);

}  // namespace mgb
