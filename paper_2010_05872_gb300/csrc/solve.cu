// Batched tridiagonal solves with the coarse mass matrix M_c along every axis
// of a level (Section 2 step 4; Section 5.3 "batched correction computation",
// Section 5.4 precomputed factors): Thomas elimination with the factors of the
// plan, forward y_k = (f_k - a_k y_{k-1}) m_k, backward x_k = y_k - c'_k x_{k+1}.
// The last solve of a level applies its result (correction application).
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "solve_tile.cuh"
#include "tma.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

// Elements of a line loaded together (independent loads in flight).
template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  static constexpr int value = 32;
};
template <>
struct Chunk<double> {
  static constexpr int value = 16;
};


// Lines along a strided axis: element k of line (outer, inner) sits at
// outer * nc * stride + k * stride + inner.  One thread per line; adjacent
// threads take adjacent `inner`, so every access is a coalesced row access.
// Loads are issued kChunk at a time ahead of the recurrence.
template <typename T>
__global__ void __launch_bounds__(256)
solve_strided_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t outer,
                     int64_t stride, int mode) {
  constexpr int kChunk = Chunk<T>::value;
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

template <typename T>
__global__ void __launch_bounds__(128)
solve_contig_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines, int rows,
                    int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  solve_contig_tile<T>(ax, F, B, nlines, rows, mode, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(128)
solve_contig_tma_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines,
                        int rows, int mode, unsigned int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  solve_contig_tma_tile<T>(ax, F, B, nlines, rows, mode, status, blockIdx.x, smem_raw);
}

// The per-level form keeps its own body (one 32-line group per CTA of
// exactly nseg warps); solve_seg_tile is the same method for the persistent
// batched kernel, with several groups side by side.
template <typename T>
__global__ void __launch_bounds__(32 * kSegWarps, 2)
solve_seg_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines, int64_t S,
                 int64_t block_stride, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = ax.nc, L = ax.seg_len;
  const int nseg = blockDim.x >> 5;
  T* s_tm = reinterpret_cast<T*>(smem_raw);
  T* s_sb = s_tm + nc;
  T* s_sg = s_sb + nc;
  T* s_sy = s_sg + nc;
  T* s_sh = s_sy + nc;
  T* s_c = s_sh + nc;  // nseg x 32 boundary values
  const int tid = threadIdx.x, lane = tid & 31, sgi = tid >> 5;
  for (int k = tid; k < nc; k += blockDim.x) {
    s_tm[k] = ax.tm[k];
    s_sb[k] = ax.sb[k];
    s_sg[k] = ax.sg[k];
    s_sy[k] = ax.sy[k];
    s_sh[k] = ax.sh[k];
  }
  const int64_t line = static_cast<int64_t>(blockIdx.x) * 32 + lane;
  const bool valid = line < nlines;
  const int64_t o = valid ? line / S : 0, in = valid ? line - o * S : 0;
  const int64_t base = o * block_stride + in;
  const int k0 = sgi * L, len = max(0, min(L, nc - k0));
  T v[kSegMax];
  {
    const T* p = F + base + static_cast<int64_t>(k0) * S;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j) {
      v[j] = (valid && j < len) ? *p : T(0);
      p += S;
    }
  }
  __syncthreads();
  // Forward from a zero boundary value.
  T y = T(0);
#pragma unroll
  for (int j = 0; j < kSegMax; ++j) {
    if (j < len) {
      y = s_tm[k0 + j] * v[j] + s_sb[k0 + j] * y;
      v[j] = y;
    }
  }
  s_c[sgi * 32 + lane] = y;
  __syncthreads();
  T Y = T(0);  // final y at the end of the previous segment
  for (int q = 0; q < sgi; ++q) Y = s_c[q * 32 + lane] + s_sg[min(q * L + L, nc) - 1] * Y;
#pragma unroll
  for (int j = 0; j < kSegMax; ++j)
    if (j < len) v[j] += s_sg[k0 + j] * Y;
  __syncthreads();  // every read of the forward boundary values is done
  // Backward from a zero boundary value.
  T x = T(0);
#pragma unroll
  for (int j = kSegMax - 1; j >= 0; --j) {
    if (j < len) {
      x = v[j] + s_sy[k0 + j] * x;
      v[j] = x;
    }
  }
  s_c[sgi * 32 + lane] = x;
  __syncthreads();
  T X = T(0);  // final x at the start of the next segment
  for (int q = nseg - 1; q > sgi; --q) X = s_c[q * 32 + lane] + s_sh[q * L] * X;
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < kSegMax; ++j)
    if (j < len) v[j] += s_sh[k0 + j] * X;
  T* pf = F + base + static_cast<int64_t>(k0) * S;
  if (mode == kApplyNone) {
#pragma unroll
    for (int j = 0; j < kSegMax; ++j) {
      if (j < len) *pf = v[j];
      pf += S;
    }
    return;
  }
  // Apply in groups of 8 (B loads in flight together).
  T* pb = B + base + static_cast<int64_t>(k0) * S;
#pragma unroll
  for (int j0 = 0; j0 < kSegMax; j0 += 8) {
    T bv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) bv[u] = (j0 + u < len) ? pb[static_cast<int64_t>(u) * S] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (j0 + u < len) {
        const int64_t off = static_cast<int64_t>(u) * S;
        if (mode == kApplyDecompose) {
          pb[off] = bv[u] + v[j0 + u];
          pf[off] = bv[u];
        } else {
          pb[off] = bv[u] - v[j0 + u];
        }
      }
    }
    pb += 8 * S;
    pf += 8 * S;
  }
}

inline unsigned ceil_div(int64_t a, int64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

}  // namespace

template <typename T>
cudaError_t launch_solves(const LevelK<T>& lv, T* F, T* B, ApplyMode mode, int level,
                          unsigned int* status, cudaStream_t s) {
  const int64_t c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  int last = 0;
  while (lv.ax[last].n == 1) ++last;  // lowest active axis is solved last
  for (int a = 2; a >= last; --a) {
    const int m = (a == last) ? mode : kApplyNone;
    const double passes = m == kApplyDecompose ? 4.0 : m == kApplyRecompose ? 3.0 : 2.0;
    TraceScope ts(a == 2 ? kKSolveContig : kKSolveStrided, level,
                  sizeof(T) * passes * double(c0) * c1 * c2, s);
    const size_t per_row = sizeof(T) * static_cast<size_t>(c2 | 1);
    const size_t tpad = (3 * sizeof(T) * static_cast<size_t>(c2) + 15) / 16 * 16;
    if (a == 2 && (c2 & 1) && per_row <= 32 * 1024 && c0 * c1 >= 1024) {
      // Odd line length: TMA-staged lines, about 64 KB of lines per CTA.
      const int64_t nlines = c0 * c1;
      const int rows = static_cast<int>(std::max<size_t>(1, std::min<size_t>(128, (64 * 1024) / per_row)));
      const size_t smem = tpad + per_row * rows + 32;
      cudaFuncSetAttribute(solve_contig_tma_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
      solve_contig_tma_kernel<T><<<ceil_div(nlines, rows), 128, smem, s>>>(lv.ax[2], F, B, nlines,
                                                                            rows, m, status);
    } else if (a == 2 && per_row <= 112 * 1024) {
      const int64_t nlines = c0 * c1;
      int rows = static_cast<int>(std::min<size_t>(128, (112 * 1024) / per_row));
      rows = std::max(rows, 1);
      const size_t smem = per_row * rows;
      cudaFuncSetAttribute(solve_contig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
      solve_contig_kernel<T><<<ceil_div(nlines, rows), 128, smem, s>>>(lv.ax[2], F, B, nlines,
                                                                        rows, m);
    } else if (a != 2 && (lv.ax[a].nc + lv.ax[a].seg_len - 1) / lv.ax[a].seg_len <= kSegWarps) {
      // Strided lines in register-resident segments.
      const int nc = lv.ax[a].nc;
      const int nseg = (nc + lv.ax[a].seg_len - 1) / lv.ax[a].seg_len;
      const int64_t S = (a == 0) ? c1 * c2 : c2;
      const int64_t nlines = (a == 0) ? S : c0 * S;
      const size_t smem = sizeof(T) * (5 * static_cast<size_t>(nc) + 32 * static_cast<size_t>(nseg));
      solve_seg_kernel<T><<<ceil_div(nlines, 32), 32 * nseg, smem, s>>>(lv.ax[a], F, B, nlines, S,
                                                                         nc * S, m);
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
                                          unsigned int*, cudaStream_t);
template cudaError_t launch_solves<double>(const LevelK<double>&, double*, double*, ApplyMode, int,
                                           unsigned int*, cudaStream_t);

}  // namespace mgb
