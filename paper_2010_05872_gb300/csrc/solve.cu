// Batched tridiagonal solves with the coarse mass matrix M_c along every axis
// of a level (Section 2 step 4; Section 5.3 "batched correction computation",
// Section 5.4 precomputed factors): Thomas elimination with the factors of the
// plan, forward y_k = (f_k - a_k y_{k-1}) m_k, backward x_k = y_k - c'_k x_{k+1}.
// The last solve of a level applies its result (correction application).
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
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

// Contiguous lines of odd length, staged by one 1D TMA bulk copy: the rows
// lines of a CTA are one contiguous range, copied as its enclosing 16-byte-
// aligned range (the at most 15 bytes past the last whole 16 bytes of the
// array by plain loads); with an odd pitch the threads' lines fall on
// distinct banks.  The Thomas factors come to shared memory too; one thread
// per line solves in place, then the range is written back with coalesced
// stores.  The wait on the copy gives up after 2 s and records the failure
// in `status`.
template <typename T>
__global__ void __launch_bounds__(128)
solve_contig_tma_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines,
                        int rows, int mode, unsigned int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_shift;
  const int nc = ax.nc;
  T* s_ta = reinterpret_cast<T*>(smem_raw);  // nc each
  T* s_tm = s_ta + nc;
  T* s_tc = s_tm + nc;
  const int tpad = ((3 * nc * static_cast<int>(sizeof(T)) + 15) / 16) * 16;
  T* s = reinterpret_cast<T*>(smem_raw + tpad);
  const int64_t first = static_cast<int64_t>(blockIdx.x) * rows;
  const int nr = static_cast<int>(min(static_cast<int64_t>(rows), nlines - first));
  const int total = nr * nc;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t lim = (static_cast<uint64_t>(nlines) * nc * sizeof(T)) & ~15ull;
    const uint64_t sb = static_cast<uint64_t>(first) * nc * sizeof(T);
    const uint64_t eb = sb + static_cast<uint64_t>(total) * sizeof(T);
    const uint64_t ab = sb & ~15ull;
    uint64_t bb = (eb + 15) & ~15ull;
    if (bb > lim) bb = lim;
    const int shift = static_cast<int>((sb - ab) / sizeof(T));
    s_shift = shift;
    const unsigned bytes = bb > ab ? static_cast<unsigned>(bb - ab) : 0u;
    mbar_arrive_expect_tx(&bar, bytes);
    if (bytes) tma_bulk_g2s(s, reinterpret_cast<const char*>(F) + ab, bytes, &bar);
    for (uint64_t x = bb > sb ? bb : sb; x < eb; x += sizeof(T))
      s[shift + static_cast<int>((x - sb) / sizeof(T))] = F[x / sizeof(T)];
  }
  for (int k = tid; k < nc; k += blockDim.x) {
    s_ta[k] = ax.ta[k];
    s_tm[k] = ax.tm[k];
    s_tc[k] = ax.tc[k];
  }
  __syncthreads();
  const bool got = mbar_wait(&bar, 0u, kWaitLimitNs);
  if (__syncthreads_or(!got)) {
    if (tid == 0) *reinterpret_cast<volatile unsigned*>(status) = 1u;
    mbar_wait(&bar, 0u, kWaitLimitNs);
    return;
  }
  const int shift = s_shift;
  if (tid < nr) {
    T* l = s + shift + tid * nc;
    T y = T(0);
#pragma unroll 4
    for (int k = 0; k < nc; ++k) {
      y = (l[k] - s_ta[k] * y) * s_tm[k];
      l[k] = y;
    }
    T x = T(0);
#pragma unroll 4
    for (int k = nc - 1; k >= 0; --k) {
      x = l[k] - s_tc[k] * x;
      l[k] = x;
    }
  }
  __syncthreads();
  T* dstF = F + first * nc;
  T* dstB = B ? B + first * nc : nullptr;
  for (int base = tid; base < total; base += 4 * blockDim.x) {
    T bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * blockDim.x;
      bv[u] = (i < total && mode != kApplyNone) ? dstB[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * blockDim.x;
      if (i < total) {
        const T x = s[shift + i];
        if (mode == kApplyNone) dstF[i] = x;
        else apply_x(dstF, dstB, i, x, bv[u], mode);
      }
    }
  }
}

// Lines along a strided axis, split into segments of up to 32 rows: lane t
// of every warp of a CTA takes line (32 b + t), warp w takes segment w of
// it, so a warp's loads of one row are 32 consecutive words and a thread
// keeps its segment in registers (one read and one write of F per element).
// Both Thomas recurrences are first-order linear, so each segment runs them
// from a zero boundary value and then adds the boundary value's effect, a
// product of recurrence coefficients from the plan: forward, the final y
// at the end of segment s is y_loc + sg_end * (final y at the end of s - 1);
// backward, the final x at the start of s is x_loc + sh_start * (final x at
// the start of s + 1).  The boundary values pass between the warps through
// shared memory.
constexpr int kSegMax = 32;
constexpr int kSegWarps = 9;  // lines of up to 288 rows

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
