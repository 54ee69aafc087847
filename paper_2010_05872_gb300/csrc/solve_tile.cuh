// Tiles (CTA work units) of the batched tridiagonal solves, shared by the
// per-level kernels and the persistent batched kernel.  See solve.cu for
// the methods.  `tile` plays the role of the block index and `smem_raw` is
// the dynamic shared memory; any block at least as large as the launcher's
// runs a tile.
#pragma once

#include <cstdint>

#include "kernels.cuh"
#include "tma.cuh"

namespace mgb {

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

// Thomas elimination of one line held in shared memory, in place: forward
// y_k = (f_k - a_k y_{k-1}) m_k, backward x_k = y_k - c'_k x_{k+1}.  Values
// and factors are read eight at a time ahead of the recurrence, so the chain
// waits on arithmetic, not on shared-memory latency.
template <typename T>
__device__ __forceinline__ void thomas_smem(T* l, const T* ta, const T* tm, const T* tc, int nc) {
  T y = T(0);
  int k = 0;
  for (; k + 8 <= nc; k += 8) {
    T f[8], a[8], m[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      f[j] = l[k + j];
      a[j] = ta[k + j];
      m[j] = tm[k + j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      y = (f[j] - a[j] * y) * m[j];
      l[k + j] = y;
    }
  }
  for (; k < nc; ++k) {
    y = (l[k] - ta[k] * y) * tm[k];
    l[k] = y;
  }
  T x = T(0);
  k = nc - 1;
  for (; k >= 7; k -= 8) {
    T v[8], c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = l[k - j];
      c[j] = tc[k - j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x = v[j] - c[j] * x;
      l[k - j] = x;
    }
  }
  for (; k >= 0; --k) {
    x = l[k] - tc[k] * x;
    l[k] = x;
  }
}

// Lines along the contiguous axis: a CTA stages `rows` whole lines in shared
// memory (threads sweep each line, so loads and stores are coalesced), one
// thread per line solves in place (row pitch nc|1 keeps the threads on
// distinct banks), then the lines go back.
template <typename T>
__device__ __forceinline__ void solve_contig_tile(const AxisK<T>& ax, T* __restrict__ F,
                                                  T* __restrict__ B, int64_t nlines, int rows,
                                                  int mode, int tile, unsigned char*) {
  // The dynamic shared memory of the launch (every tile starts at its base).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int nc = ax.nc, pitch = nc | 1;
  const int64_t first = static_cast<int64_t>(tile) * rows;
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
template <typename T, bool PERSIST = false>
__device__ __forceinline__ void solve_contig_tma_tile(const AxisK<T>& ax, T* __restrict__ F,
                                                      T* __restrict__ B, int64_t nlines, int rows,
                                                      int mode, unsigned int* __restrict__ status,
                                                      int tile, unsigned char*) {
  // The dynamic shared memory of the launch (every tile starts at its base).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_shift;
  const int nc = ax.nc;
  T* s_ta = reinterpret_cast<T*>(smem_raw);  // nc each
  T* s_tm = s_ta + nc;
  T* s_tc = s_tm + nc;
  const int tpad = ((3 * nc * static_cast<int>(sizeof(T)) + 15) / 16) * 16;
  T* s = reinterpret_cast<T*>(smem_raw + tpad);
  const int64_t first = static_cast<int64_t>(tile) * rows;
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
      s[shift + static_cast<int>((x - sb) / sizeof(T))] = PERSIST ? __ldcg(F + x / sizeof(T)) : F[x / sizeof(T)];
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
  if (tid < nr) thomas_smem(s + shift + tid * nc, s_ta, s_tm, s_tc, nc);
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
  if (PERSIST && tid == 0) mbar_inval(&bar);
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
constexpr int kSegMax = 16;
constexpr int kSegWarps = 18;  // lines of up to 288 rows

template <typename T, bool MULTI = false>
__device__ __forceinline__ void solve_seg_tile(const AxisK<T>& ax, T* __restrict__ F,
                                               T* __restrict__ B, int64_t nlines, int64_t S,
                                               int64_t block_stride, int mode, int tile,
                                               unsigned char*, int gpp = 1) {
  // The dynamic shared memory of the launch (every tile starts at its base).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // gpp groups of 32 lines side by side: warps [g nseg, (g + 1) nseg) take
  // group g of the tile (tile gpp + g); warps beyond gpp nseg idle.
  const int nc = ax.nc, L = ax.seg_len;
  const int nseg = MULTI ? (nc + L - 1) / L : static_cast<int>(blockDim.x >> 5);
  T* s_tm = reinterpret_cast<T*>(smem_raw);
  T* s_sb = s_tm + nc;
  T* s_sg = s_sb + nc;
  T* s_sy = s_sg + nc;
  T* s_sh = s_sy + nc;
  const int tid = threadIdx.x, lane = tid & 31;
  // MULTI: gpp groups side by side (a persistent CTA); otherwise the block
  // has exactly nseg warps and takes one group.
  const int gslot = MULTI ? min((tid >> 5) / nseg, gpp) : 0;
  const int sgi = !MULTI ? (tid >> 5) : gslot < gpp ? (tid >> 5) - gslot * nseg : nseg;
  const int gsel = MULTI ? min(gslot, gpp - 1) : 0;
  T* s_c = s_sh + nc + static_cast<size_t>(gsel) * nseg * 32;  // nseg x 32 per group
  for (int k = tid; k < nc; k += blockDim.x) {
    s_tm[k] = ax.tm[k];
    s_sb[k] = ax.sb[k];
    s_sg[k] = ax.sg[k];
    s_sy[k] = ax.sy[k];
    s_sh[k] = ax.sh[k];
  }
  const int64_t line = MULTI ? (static_cast<int64_t>(tile) * gpp + gsel) * 32 + lane
                             : static_cast<int64_t>(tile) * 32 + lane;
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
  if (!MULTI || sgi < nseg) s_c[sgi * 32 + lane] = y;
  __syncthreads();
  T Y = T(0);  // final y at the end of the previous segment
  for (int q = 0; q < (MULTI ? min(sgi, nseg) : sgi); ++q)
    Y = s_c[q * 32 + lane] + s_sg[min(q * L + L, nc) - 1] * Y;
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
  if (!MULTI || sgi < nseg) s_c[sgi * 32 + lane] = x;
  __syncthreads();
  T X = T(0);  // final x at the start of the next segment
  for (int q = nseg - 1; q > sgi; --q) X = s_c[q * 32 + lane] + s_sh[q * L] * X;
  if (!valid || (MULTI && sgi >= nseg)) return;
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

}  // namespace mgb
