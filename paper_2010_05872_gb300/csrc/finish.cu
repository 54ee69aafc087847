// In-place finishing pass over a level-l grid (Section 2):
//   decomposition : coefficient nodes get v - Pi(v on N_{l-1}) (the saved
//                   nodal values), nodal nodes get the final coarser values;
//   recomposition : coefficient nodes get u_mc + Pi(coarse values), nodal
//                   nodes get the coarse values.
// Layout of the work: a CTA takes kRows consecutive fine rows (j0, j1) and a
// chunk of up to kCols columns.  Every row first gets its "combined" coarse
// row in shared memory: the up to 4 coarse rows its corners come from,
// weighted by the axis-0 and axis-1 interpolation weights.  Then one thread
// per fine column walks the rows; its column data (nodal or coefficient,
// coarse index, axis-2 weights) stays in registers and its kRows loads are
// issued together.
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
#include "finish_tile.cuh"
#include "grid.cuh"
#include "kernels.cuh"
#include "tma.cuh"
#include "trace.hpp"

namespace mgb {
namespace {


constexpr int kRows = 16;
constexpr int kCols = 640;           // even
constexpr int kMaxThreads = kCols;
constexpr int kCW = kCols / 2 + 1;   // combined coarse values per row and chunk

template <typename T>
__global__ void __launch_bounds__(kMaxThreads)
finish_kernel(LevelK<T> lv, const T* __restrict__ nodal_src, const T* __restrict__ interp_src,
              T sign, T* __restrict__ fine) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* crow = reinterpret_cast<T*>(smem_raw);  // kRows x kCW
  __shared__ int64_t s_nodal[kRows];         // coarse row offset (fully nodal rows) or -1
  __shared__ int64_t s_o00[kRows];           // coarse row of the (low, low) corner
  __shared__ int s_q[kRows];                 // bit 1: axis-0 coefficient, bit 0: axis-1
  __shared__ T s_w[kRows][4];                // corner weights

  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int64_t nrows = static_cast<int64_t>(n0) * n1;
  const int64_t ngroups = (nrows + kRows - 1) / kRows;
  const int nchunks = (n2 + kCols - 1) / kCols;
  const int tid = threadIdx.x;

  for (int64_t b = blockIdx.x; b < ngroups * nchunks; b += gridDim.x) {
    const int64_t rg = b / nchunks;
    const int cx = static_cast<int>(b - rg * nchunks);
    const int64_t r0 = rg * kRows;
    const int R = static_cast<int>(min(static_cast<int64_t>(kRows), nrows - r0));
    const int jlo = cx * kCols, jhi = min(jlo + kCols, n2);  // fine columns [jlo, jhi)
    const int klo = jlo / 2, khi = min(jhi / 2, c2 - 1);      // coarse columns [klo, khi]
    const int kw = khi - klo + 1;

    // Row data, one thread per row: corner coarse row, weights, and the
    // coarse row of fully nodal rows.
    if (tid < R) {
      const int64_t rr = r0 + tid;
      const int j0 = static_cast<int>(rr / n1), j1 = static_cast<int>(rr - static_cast<int64_t>(j0) * n1);
      const bool q0 = is_coef(j0, n0), q1 = is_coef(j1, n1);
      const int a0 = q0 ? (j0 - 1) >> 1 : nodal_k(j0, n0, c0);
      const int a1 = q1 ? (j1 - 1) >> 1 : nodal_k(j1, n1, c1);
      const T wl0 = q0 ? lv.ax[0].iwl[j0] : T(1), wr0 = q0 ? lv.ax[0].iwr[j0] : T(0);
      const T wl1 = q1 ? lv.ax[1].iwl[j1] : T(1), wr1 = q1 ? lv.ax[1].iwr[j1] : T(0);
      const int64_t o00 = (static_cast<int64_t>(a0) * c1 + a1) * c2;
      s_o00[tid] = o00;
      s_nodal[tid] = (q0 || q1) ? -1 : o00;
      s_q[tid] = (q0 ? 2 : 0) | (q1 ? 1 : 0);
      s_w[tid][0] = wl0 * wl1;
      s_w[tid][1] = wl0 * wr1;
      s_w[tid][2] = wr0 * wl1;
      s_w[tid][3] = wr0 * wr1;
    }
    __syncthreads();
    // Combined coarse rows: items (row, coarse column) flat, 8 per thread in
    // flight.  i / kw (i < kRows kw, kw <= kCW) is exact through
    // (i + 0.5) / kw in FP32: that quotient is at least 1 / (2 kw) from an
    // integer and the FP32 estimate is within kRows 2^-22 of it.
    {
      const int items = R * kw;
      const float inv_kw = 1.0f / static_cast<float>(kw);
      for (int base = tid; base < items; base += 8 * blockDim.x) {
        T v[8];
        int slot[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = base + u * blockDim.x;
          slot[u] = -1;
          v[u] = T(0);
          if (i < items) {
            const int rl = static_cast<int>((static_cast<float>(i) + 0.5f) * inv_kw);
            const int k = i - rl * kw;
            const int q = s_q[rl];
            const T* s00 = interp_src + s_o00[rl] + klo + k;
            T x = s_w[rl][0] * s00[0];
            if (q & 1) x += s_w[rl][1] * s00[c2];
            if (q & 2) {
              const T* s10 = s00 + static_cast<int64_t>(c1) * c2;
              x += s_w[rl][2] * s10[0];
              if (q & 1) x += s_w[rl][3] * s10[c2];
            }
            v[u] = x;
            slot[u] = rl * kCW + k;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (slot[u] >= 0) crow[slot[u]] = v[u];
      }
    }
    __syncthreads();

    const int j2 = jlo + tid;
    if (j2 < jhi) {
      const bool q2 = is_coef(j2, n2);
      const int kn = nodal_k(j2, n2, c2);  // coarse index (nodal column)
      const int km = (j2 >> 1) - klo;      // left coarse neighbour (coefficient column)
      const T wl2 = q2 ? lv.ax[2].iwl[j2] : T(1), wr2 = q2 ? lv.ax[2].iwr[j2] : T(0);
      const int kl = q2 ? km : kn - klo, kr = q2 ? km + 1 : kn - klo;
      T f[kRows];
#pragma unroll
      for (int rl = 0; rl < kRows; ++rl)
        if (rl < R) f[rl] = fine[(r0 + rl) * n2 + j2];
#pragma unroll
      for (int rl = 0; rl < kRows; ++rl) {
        if (rl < R) {
          const int64_t no = s_nodal[rl];
          T out;
          if (no >= 0 && !q2) {
            out = nodal_src[no + kn];
          } else {
            const T* cr = crow + rl * kCW;
            out = f[rl] + sign * (wl2 * cr[kl] + wr2 * cr[kr]);
          }
          fine[(r0 + rl) * n2 + j2] = out;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Marching form for 2D and 3D levels whose rows fit one CTA.  A CTA owns the
// fine rows of T1 coarse rows along axis 1 (all columns, or a column chunk of
// a 2D level) and walks pairs of fine planes (2m, 2m+1) along axis 0.  Per
// pair it needs the fine rows of both planes and coarse planes m and m+1;
// each arrives by one 1D TMA bulk copy (its enclosing 16-byte-aligned range,
// offset kept, no byte past an array's end requested, ragged ends by plain
// loads), the next pair's data while the current pair is computed.  One
// thread per fine column: its axis-2 data stays in registers, rows are walked
// with uniform row data, each output is one coalesced store.
// ---------------------------------------------------------------------------
template <typename T, int NS, int T1C>
__global__ void __launch_bounds__(kFMaxThreads, sizeof(T) == 4 ? 2 : 1)
finish_march_kernel(LevelK<T> lv, const T* __restrict__ nodal_src,
                    const T* __restrict__ interp_src, T sign, T* __restrict__ fine,
                    FinishGeom g, unsigned int* __restrict__ status) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  finish_march_tile<T, NS, T1C>(lv, nodal_src, interp_src, sign, fine, g, status, blockIdx.x,
                                smem_raw);
}

}  // namespace

template <typename T>
cudaError_t launch_finish(const LevelK<T>& lv_in, const T* nodal_src, const T* interp_src, T sign,
                          T* fine, int level, unsigned int* status, cudaStream_t s) {
  const LevelK<T>& lv = lv_in;
  const int64_t nf_all = int64_t(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  const double ncs_all = double(lv.ax[0].nc) * lv.ax[1].nc * lv.ax[2].nc;
  if (!(lv.ax[0].n == 1 && lv.ax[1].n == 1) && nf_all >= (int64_t(1) << 17)) {
    LevelK<T> mv = lv_in;
    if (mv.ax[0].n == 1) std::swap(mv.ax[0], mv.ax[1]);  // 2D: march along the rows
    FinishGeom g{};
    if (finish_geometry(mv, g)) {
      TraceScope ts(sign < T(0) ? kKFinishDec : kKFinishRec, level,
                    sizeof(T) * (2 * double(nf_all) + (nodal_src == interp_src ? 1 : 2) * ncs_all), s);
      constexpr int NS = FinishCfg<T>::NS;
      const size_t smem =
          sizeof(T) * (2 * NS * static_cast<size_t>(g.FBUF) +
                       (nodal_src == interp_src ? 1 : 2) * (NS + 1) * static_cast<size_t>(g.CBUF));
      auto kernel = finish_march_kernel<T, NS, FinishCfg<T>::T1>;
      allow_dynamic_smem(kernel, smem);
      int per_sm = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, g.threads, smem);
      per_sm = std::max(per_sm, 1);
      const int npairs = (mv.ax[0].n + 1) / 2;
      g.t0 = march_chunk(npairs, g.nb1 * g.nb2, 152 * per_sm, 1);
      g.nb0 = (npairs + g.t0 - 1) / g.t0;
      launch_pdl(kernel, dim3(static_cast<unsigned>(g.nb0 * g.nb1 * g.nb2)), dim3(g.threads), smem,
                 s, mv, nodal_src, interp_src, sign, fine, g, status);
      return cudaGetLastError();
    }
  }
  const int n2 = lv.ax[2].n;
  const int64_t nrows = static_cast<int64_t>(lv.ax[0].n) * lv.ax[1].n;
  const int64_t work = ((nrows + kRows - 1) / kRows) * ((n2 + kCols - 1) / kCols);
  const int threads = 32 * ((std::min(n2, kCols) + 31) / 32);
  const size_t smem = sizeof(T) * kRows * kCW;
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(work, 1 << 30));
  const double nf = double(nrows) * n2;
  const double ncs = double(lv.ax[0].nc) * lv.ax[1].nc * lv.ax[2].nc;
  TraceScope ts(sign < T(0) ? kKFinishDec : kKFinishRec, level,
                sizeof(T) * (2 * nf + (nodal_src == interp_src ? 1 : 2) * ncs), s);
  allow_dynamic_smem(finish_kernel<T>, smem);
  launch_pdl(finish_kernel<T>, dim3(grid), dim3(threads), smem, s, lv, nodal_src, interp_src, sign,
             fine);
  return cudaGetLastError();
}

template cudaError_t launch_finish<float>(const LevelK<float>&, const float*, const float*, float,
                                          float*, int, unsigned int*, cudaStream_t);
template cudaError_t launch_finish<double>(const LevelK<double>&, const double*, const double*,
                                           double, double*, int, unsigned int*, cudaStream_t);

}  // namespace mgb
