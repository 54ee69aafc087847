// Batched tridiagonal solves with the coarse mass matrix M_c along every axis
// of a level (Section 2 step 4; Section 5.3 "batched correction computation",
// Section 5.4 precomputed factors): Thomas elimination with the factors of the
// plan, forward y_k = (f_k - a_k y_{k-1}) m_k, backward x_k = y_k - c'_k x_{k+1}.
// The last solve of a level applies its result (correction application).
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
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
  grid_dep_enter();
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
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  solve_contig_tile<T>(ax, F, B, nlines, rows, mode, blockIdx.x, smem_raw);
}

// The per-level form keeps its own body (one 32-line group per CTA of
// exactly nseg warps; short-lived CTAs let the scheduler overlap one group's
// loads with another's arithmetic); solve_seg_tile is the same method for
// the persistent batched kernel, with several groups side by side.  Here
// warp 0 carries the boundary values across all segments (one pass per
// recurrence) instead of every warp walking the segments before it, and
// offsets are of type IDX (32-bit whenever the coarse grid allows).
template <typename T, typename IDX>
__global__ void __launch_bounds__(32 * kSegWarps, 2)
solve_seg_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, IDX nlines, IDX S,
                 IDX block_stride, int mode) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nc = ax.nc, L = ax.seg_len;
  const int nseg = blockDim.x >> 5;
  T* s_tm = reinterpret_cast<T*>(smem_raw);
  T* s_sb = s_tm + nc;
  T* s_sg = s_sb + nc;
  T* s_sy = s_sg + nc;
  T* s_sh = s_sy + nc;
  T* s_c = s_sh + nc;            // nseg x 32 local boundary values
  T* s_y = s_c + nseg * 32;      // nseg x 32 carried boundary values
  const int tid = threadIdx.x, lane = tid & 31, sgi = tid >> 5;
  for (int k = tid; k < nc; k += blockDim.x) {
    s_tm[k] = ax.tm[k];
    s_sb[k] = ax.sb[k];
    s_sg[k] = ax.sg[k];
    s_sy[k] = ax.sy[k];
    s_sh[k] = ax.sh[k];
  }
  const IDX line = static_cast<IDX>(blockIdx.x) * 32 + lane;
  const bool valid = line < nlines;
  const IDX o = valid ? line / S : 0, in = valid ? line - o * S : 0;
  const int k0 = sgi * L, len = max(0, min(L, nc - k0));
  const IDX base = o * block_stride + in + static_cast<IDX>(k0) * S;
  T v[kSegMax];
#pragma unroll
  for (int j = 0; j < kSegMax; ++j)
    v[j] = (valid && j < len) ? F[base + static_cast<IDX>(j) * S] : T(0);
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
  if (sgi == 0) {  // the final y entering each segment
    T Y = T(0);
    for (int q = 0; q < nseg; ++q) {
      s_y[q * 32 + lane] = Y;
      Y = s_c[q * 32 + lane] + s_sg[min(q * L + L, nc) - 1] * Y;
    }
  }
  __syncthreads();
  {
    const T Y = s_y[sgi * 32 + lane];
#pragma unroll
    for (int j = 0; j < kSegMax; ++j)
      if (j < len) v[j] += s_sg[k0 + j] * Y;
  }
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
  if (sgi == 0) {  // the final x entering each segment from above
    T X = T(0);
    for (int q = nseg - 1; q >= 0; --q) {
      s_y[q * 32 + lane] = X;
      X = s_c[q * 32 + lane] + s_sh[q * L] * X;
    }
  }
  __syncthreads();
  if (!valid) return;
  {
    const T X = s_y[sgi * 32 + lane];
#pragma unroll
    for (int j = 0; j < kSegMax; ++j)
      if (j < len) v[j] += s_sh[k0 + j] * X;
  }
  if (mode == kApplyNone) {
#pragma unroll
    for (int j = 0; j < kSegMax; ++j)
      if (j < len) F[base + static_cast<IDX>(j) * S] = v[j];
    return;
  }
  // Apply in groups of 8 (B loads in flight together).
#pragma unroll
  for (int j0 = 0; j0 < kSegMax; j0 += 8) {
    T bv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      bv[u] = (j0 + u < len) ? B[base + static_cast<IDX>(j0 + u) * S] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (j0 + u < len) {
        const IDX off = base + static_cast<IDX>(j0 + u) * S;
        if (mode == kApplyDecompose) {
          B[off] = bv[u] + v[j0 + u];
          F[off] = bv[u];
        } else {
          B[off] = bv[u] - v[j0 + u];
        }
      }
    }
  }
}

// Contiguous lines of odd length in a persistent, double-buffered form: a
// CTA takes batches of `rows` lines (one contiguous range each) in turn; the
// bulk copy of its next batch (thread 0, enclosing 16-byte-aligned range,
// the at most 15 bytes past the array's last whole 16 bytes by plain loads)
// runs while the current batch is solved (one thread per line, Thomas from
// shared memory with the factors there too; an odd pitch keeps the lines on
// distinct banks) and written back with coalesced stores.  Waits give up
// after 2 s and record the failure in `status`.
template <typename T>
__global__ void __launch_bounds__(128)
solve_contig_pipe_kernel(AxisK<T> ax, T* __restrict__ F, T* __restrict__ B, int64_t nlines,
                         int rows, int bufelems, int mode, unsigned int* __restrict__ status) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_shift[2];
  const int nc = ax.nc;
  T* s_ta = reinterpret_cast<T*>(smem_raw);  // nc each
  T* s_tm = s_ta + nc;
  T* s_tc = s_tm + nc;
  const int tpad = ((3 * nc * static_cast<int>(sizeof(T)) + 15) / 16) * 16;
  T* buf0 = reinterpret_cast<T*>(smem_raw + tpad);  // 2 x bufelems
  const int tid = threadIdx.x;
  const int64_t nbatch = (nlines + rows - 1) / rows;
  const uint64_t lim = (static_cast<uint64_t>(nlines) * nc * sizeof(T)) & ~15ull;
  auto issue = [&](int64_t b, int slot) {  // thread 0
    const int64_t first = b * rows;
    const int nr = static_cast<int>(min(static_cast<int64_t>(rows), nlines - first));
    const uint64_t sb = static_cast<uint64_t>(first) * nc * sizeof(T);
    const uint64_t eb = sb + static_cast<uint64_t>(nr) * nc * sizeof(T);
    const uint64_t ab = sb & ~15ull;
    uint64_t bb = (eb + 15) & ~15ull;
    if (bb > lim) bb = lim;
    const int shift = static_cast<int>((sb - ab) / sizeof(T));
    T* dst = buf0 + static_cast<size_t>(slot) * bufelems;
    s_shift[slot] = shift;
    const unsigned bytes = bb > ab ? static_cast<unsigned>(bb - ab) : 0u;
    mbar_arrive_expect_tx(&bars[slot], bytes);
    if (bytes) tma_bulk_g2s(dst, reinterpret_cast<const char*>(F) + ab, bytes, &bars[slot]);
    for (uint64_t x = bb > sb ? bb : sb; x < eb; x += sizeof(T))
      dst[shift + static_cast<int>((x - sb) / sizeof(T))] = F[x / sizeof(T)];
  };
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    if (blockIdx.x < nbatch) issue(blockIdx.x, 0);
  }
  for (int k = tid; k < nc; k += blockDim.x) {
    s_ta[k] = ax.ta[k];
    s_tm[k] = ax.tm[k];
    s_tc[k] = ax.tc[k];
  }
  __syncthreads();
  unsigned phase = 0u;
  int it = 0;
  for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x, ++it) {
    const int slot = it & 1;
    const int64_t nb = b + gridDim.x;
    if (tid == 0 && nb < nbatch) {
      fence_proxy_async();  // the other buffer's last reads (generic) precede the copy
      issue(nb, slot ^ 1);
    }
    const bool got = mbar_wait(&bars[slot], (phase >> slot) & 1u, kWaitLimitNs);
    if (__syncthreads_or(!got)) {
      if (tid == 0) *reinterpret_cast<volatile unsigned*>(status) = 1u;
      mbar_wait(&bars[slot], (phase >> slot) & 1u, kWaitLimitNs);
      if (nb < nbatch) mbar_wait(&bars[slot ^ 1], (phase >> (slot ^ 1)) & 1u, kWaitLimitNs);
      return;
    }
    phase ^= 1u << slot;
    const int64_t first = b * rows;
    const int nr = static_cast<int>(min(static_cast<int64_t>(rows), nlines - first));
    const int total = nr * nc;
    T* s = buf0 + static_cast<size_t>(slot) * bufelems + s_shift[slot];
    if (tid < nr) thomas_smem(s + tid * nc, s_ta, s_tm, s_tc, nc);
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
          const T x = s[i];
          if (mode == kApplyNone) dstF[i] = x;
          else apply_x(dstF, dstB, i, x, bv[u], mode);
        }
      }
    }
    __syncthreads();  // this buffer may be refilled
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
    // FP64 runs the contiguous axis through the segmented kernel as lines of
    // stride 1: its 16-row chains instead of whole-line Thomas chains, which
    // FP64's FMA latency makes long (and few lines fit a batch).
    const bool seg64 = sizeof(T) == 8 && a == 2 && lv.ax[2].n > 1 &&
                       (c2 + lv.ax[2].seg_len - 1) / lv.ax[2].seg_len <= kSegWarps;
    if (seg64) {
      const int nc = static_cast<int>(c2);
      const int nseg = (nc + lv.ax[2].seg_len - 1) / lv.ax[2].seg_len;
      const int64_t nlines = c0 * c1;
      const size_t smem = sizeof(T) * (5 * static_cast<size_t>(nc) + 64 * static_cast<size_t>(nseg));
      if (c0 * c1 * c2 < (int64_t(1) << 31))
        launch_pdl(solve_seg_kernel<T, int32_t>, dim3(ceil_div(nlines, 32)), dim3(32 * nseg), smem, s,
                   lv.ax[2], F, B, static_cast<int32_t>(nlines), int32_t(1), static_cast<int32_t>(nc), m);
      else
        launch_pdl(solve_seg_kernel<T, int64_t>, dim3(ceil_div(nlines, 32)), dim3(32 * nseg), smem, s,
                   lv.ax[2], F, B, nlines, int64_t(1), static_cast<int64_t>(nc), m);
    } else if (a == 2 && (c2 & 1) && per_row <= 16 * 1024 && c0 * c1 >= 1024) {
      // Odd line length: persistent double-buffered TMA batches of about
      // 32 KB of lines, three CTAs per SM.
      const int64_t nlines = c0 * c1;
      const int rows = static_cast<int>(std::max<size_t>(1, std::min<size_t>(128, (32 * 1024) / per_row)));
      const int vec = 16 / static_cast<int>(sizeof(T));
      const int bufelems = ((rows * static_cast<int>(c2) + 2 * vec) + vec - 1) / vec * vec;
      const size_t smem = tpad + 2 * sizeof(T) * static_cast<size_t>(bufelems);
      allow_dynamic_smem(solve_contig_pipe_kernel<T>, smem);
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_contig_pipe_kernel<T>, 128, smem);
      const int64_t nbatch = (nlines + rows - 1) / rows;
      const unsigned grid = static_cast<unsigned>(std::max<int64_t>(
          1, std::min<int64_t>(nbatch, 152 * static_cast<int64_t>(std::max(per_sm, 1)))));
      launch_pdl(solve_contig_pipe_kernel<T>, dim3(grid), dim3(128), smem, s, lv.ax[2], F, B,
                 nlines, rows, bufelems, m, status);
    } else if (a == 2 && per_row <= 112 * 1024) {
      const int64_t nlines = c0 * c1;
      int rows = static_cast<int>(std::min<size_t>(128, (112 * 1024) / per_row));
      rows = std::max(rows, 1);
      const size_t smem = per_row * rows;
      allow_dynamic_smem(solve_contig_kernel<T>, smem);
      launch_pdl(solve_contig_kernel<T>, dim3(ceil_div(nlines, rows)), dim3(128), smem, s, lv.ax[2],
                 F, B, nlines, rows, m);
    } else if (a != 2 && (lv.ax[a].nc + lv.ax[a].seg_len - 1) / lv.ax[a].seg_len <= kSegWarps) {
      // Strided lines in register-resident segments.
      const int nc = lv.ax[a].nc;
      const int nseg = (nc + lv.ax[a].seg_len - 1) / lv.ax[a].seg_len;
      const int64_t S = (a == 0) ? c1 * c2 : c2;
      const int64_t nlines = (a == 0) ? S : c0 * S;
      const size_t smem = sizeof(T) * (5 * static_cast<size_t>(nc) + 64 * static_cast<size_t>(nseg));
      if (c0 * c1 * c2 < (int64_t(1) << 31))
        launch_pdl(solve_seg_kernel<T, int32_t>, dim3(ceil_div(nlines, 32)), dim3(32 * nseg), smem, s,
                   lv.ax[a], F, B, static_cast<int32_t>(nlines), static_cast<int32_t>(S),
                   static_cast<int32_t>(nc * S), m);
      else
        launch_pdl(solve_seg_kernel<T, int64_t>, dim3(ceil_div(nlines, 32)), dim3(32 * nseg), smem, s,
                   lv.ax[a], F, B, nlines, S, nc * S, m);
    } else {
      // Strided lines; contiguous lines too long for shared memory go here
      // too, as lines of stride 1.
      const int64_t outer = (a == 0) ? 1 : (a == 1) ? c0 : c0 * c1;
      const int64_t stride = (a == 0) ? c1 * c2 : (a == 1) ? c2 : 1;
      launch_pdl(solve_strided_kernel<T>, dim3(ceil_div(outer * stride, 256)), dim3(256), 0, s,
                 lv.ax[a], F, B, outer, stride, m);
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
