// Sampled prediction-error sums of the adaptive stopping level (Section 4.2,
// Algorithm 1's sampled prediction errors) on one level-l grid.
//
// The sampled blocks are the cells of the level-(l-1) grid whose index is a
// multiple of 4 along every axis (one block in four per dimension); a cell
// spans level-l indices cpos(b) .. cpos(b + 1), 3 nodes (2 for the end cell
// of an even axis).  Over the coefficient nodes of those blocks (nodes off
// N_{l-1}, 19 in a full 3^3 block) the kernel sums, in FP64,
//   E_Lorenzo += |Lorenzo prediction - v| + 1.22 tau0          (Eq. lorenzo)
//   E_interp  += |multilinear interpolation - v| + p tau0      (Eq. interp)
// with p = 0.369, 0.259, 0.182 for edge, plane and cube nodes (one, two or
// three midpoint coordinates).  The predictions and residuals are formed in
// the grid's own precision (FP32 arithmetic runs at a far higher rate than
// FP64 on this part) and each block's residual sum is added in FP64.  The Lorenzo prediction is the signed sum of
// the 7 neighbours with some indices lowered by one (+ for an odd number of
// lowered indices); neighbours outside the grid count as 0.  Interpolation
// uses the level's own weights (the transform's iwl / iwr tables), of which
// the 1/2, 1/4, 1/8 stencils of Eq. (multilinear_interp) are the uniform
// case.
//
// One thread per sampled block (grid-stride, its 4^3 neighbourhood in
// registers), per-CTA partial sums reduced in a fixed order by a second
// single-CTA kernel: the result does not depend on timing.
#include <climits>
#include <cstdint>

#include "pdl.cuh"
#include "grid.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

constexpr int kPThreads = 256;
constexpr double kLorenzoPenalty = 1.22;
__constant__ double kInterpPenalty[4] = {0.0, 0.369, 0.259, 0.182};

template <typename T>
__global__ void __launch_bounds__(kPThreads)
prediction_errors_kernel(LevelK<T> lv, const T* __restrict__ v, int nsampled, int m1, int m2,
                         double tau0, double* __restrict__ partial) {
  grid_dep_enter();
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  double el = 0.0, ei = 0.0;
  // One thread per sampled block: its 4 x 4 x 4 neighbourhood (the block
  // and the row / column / plane before it, 0 outside the grid) is loaded
  // into registers, then the 27 node slots are evaluated from there.
  for (int sidx = blockIdx.x * blockDim.x + threadIdx.x; sidx < nsampled;
       sidx += gridDim.x * blockDim.x) {
    const int s2 = sidx % m2, s1 = (sidx / m2) % m1, s0 = sidx / (m1 * m2);
    const int lo[3] = {cpos(4 * s0, n0), cpos(4 * s1, n1), cpos(4 * s2, n2)};
    const int hi[3] = {cpos(4 * s0 + 1, n0), cpos(4 * s1 + 1, n1), cpos(4 * s2 + 1, n2)};
    T w[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = lo[0] - 1 + a, j = lo[1] - 1 + b, k = lo[2] - 1 + c;
          const bool in = i >= 0 && j >= 0 && k >= 0 && i <= hi[0] && j <= hi[1] && k <= hi[2];
          w[a][b][c] = in ? __ldg(v + (static_cast<int64_t>(i) * n1 + j) * n2 + k) : T(0);
        }
    // The cell midpoint of each axis (if any) and its interpolation weights.
    bool mid[3];
    T wl[3], wr[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int nd = d == 0 ? n0 : d == 1 ? n1 : n2;
      mid[d] = hi[d] - lo[d] == 2 && is_coef(lo[d] + 1, nd);
      wl[d] = mid[d] ? lv.ax[d].iwl[lo[d] + 1] : T(0);
      wr[d] = mid[d] ? lv.ax[d].iwr[lo[d] + 1] : T(0);
    }
    if (mid[0] && mid[1] && mid[2]) {
      // A full 3^3 block (all but the end cells of even axes): the
      // interpolant by tensor steps from the 8 corners (window rows 1 and 3),
      // axis 2, then 1, then 0; the node's prediction is the last step along
      // its midpoint axes.
      T m2[2][2], m1[2][3], m0[3][3];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
          m2[a][b] = wl[2] * w[1 + 2 * a][1 + 2 * b][1] + wr[2] * w[1 + 2 * a][1 + 2 * b][3];
      auto p1 = [&](int a, int b, int c) {  // value at (row a in {0,1}, b in {0,1}, c in 0..2)
        return c == 1 ? m2[a][b] : w[1 + 2 * a][1 + 2 * b][1 + c];
      };
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) m1[a][c] = wl[1] * p1(a, 0, c) + wr[1] * p1(a, 1, c);
      auto p0 = [&](int a, int b, int c) {  // a in {0,1}, b in 0..2, c in 0..2
        return b == 1 ? m1[a][c] : p1(a, b >> 1, c);
      };
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) m0[b][c] = wl[0] * p0(0, b, c) + wr[0] * p0(1, b, c);
      T sl = T(0), si = T(0);
#pragma unroll
      for (int oi = 0; oi < 3; ++oi)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj)
#pragma unroll
          for (int ok = 0; ok < 3; ++ok) {
            if (oi != 1 && oj != 1 && ok != 1) continue;  // a corner
            const int a = oi + 1, b = oj + 1, c = ok + 1;
            const T x = w[a][b][c];
            const T lor = w[a][b][c - 1] + w[a][b - 1][c] + w[a - 1][b][c] - w[a][b - 1][c - 1] -
                          w[a - 1][b][c - 1] - w[a - 1][b - 1][c] + w[a - 1][b - 1][c - 1];
            const T ip = oi == 1 ? m0[oj][ok] : oj == 1 ? m1[oi >> 1][ok] : m2[oi >> 1][oj >> 1];
            sl += abs(lor - x);
            si += abs(ip - x);
          }
      // 19 nodes: 12 edge, 6 plane, 1 cube.
      el += static_cast<double>(sl) + 19.0 * kLorenzoPenalty * tau0;
      ei += static_cast<double>(si) +
            (12.0 * kInterpPenalty[1] + 6.0 * kInterpPenalty[2] + kInterpPenalty[3]) * tau0;
      continue;
    }
#pragma unroll
    for (int oi = 0; oi < 3; ++oi)
#pragma unroll
      for (int oj = 0; oj < 3; ++oj)
#pragma unroll
        for (int ok = 0; ok < 3; ++ok) {
          const bool c0 = oi == 1 && mid[0], c1 = oj == 1 && mid[1], c2 = ok == 1 && mid[2];
          const int mids = int(c0) + int(c1) + int(c2);
          if (mids == 0 || lo[0] + oi > hi[0] || lo[1] + oj > hi[1] || lo[2] + ok > hi[2]) continue;
          const int a = oi + 1, b = oj + 1, c = ok + 1;
          const T x = w[a][b][c];
          const T lor = w[a][b][c - 1] + w[a][b - 1][c] + w[a - 1][b][c] - w[a][b - 1][c - 1] -
                        w[a - 1][b][c - 1] - w[a - 1][b - 1][c] + w[a - 1][b - 1][c - 1];
          // Multilinear interpolation from the cell's corner nodes: along an
          // axis where the node sits in the middle of the block the window
          // rows 1, 2, 3 weigh (wl, 0, wr) at a midpoint and (0, 1, 0) at
          // the nodal end of a 2-node cell; elsewhere the node's own row.
          T f0[3], f1[3], f2[3];
          f0[0] = c0 ? wl[0] : T(0); f0[1] = c0 ? T(0) : T(1); f0[2] = c0 ? wr[0] : T(0);
          f1[0] = c1 ? wl[1] : T(0); f1[1] = c1 ? T(0) : T(1); f1[2] = c1 ? wr[1] : T(0);
          f2[0] = c2 ? wl[2] : T(0); f2[1] = c2 ? T(0) : T(1); f2[2] = c2 ? wr[2] : T(0);
          T ip = T(0);
#pragma unroll
          for (int u0 = 0; u0 < 3; ++u0) {
            if (oi != 1 && u0 != 1) continue;
            const int ra = oi == 1 ? 1 + u0 : a;
            const T g0 = oi == 1 ? f0[u0] : T(1);
#pragma unroll
            for (int u1 = 0; u1 < 3; ++u1) {
              if (oj != 1 && u1 != 1) continue;
              const int rb = oj == 1 ? 1 + u1 : b;
              const T g1 = oj == 1 ? f1[u1] : T(1);
#pragma unroll
              for (int u2 = 0; u2 < 3; ++u2) {
                if (ok != 1 && u2 != 1) continue;
                const int rc = ok == 1 ? 1 + u2 : c;
                const T g2 = ok == 1 ? f2[u2] : T(1);
                ip += g0 * g1 * g2 * w[ra][rb][rc];
              }
            }
          }
          el += static_cast<double>(abs(lor - x)) + kLorenzoPenalty * tau0;
          ei += static_cast<double>(abs(ip - x)) + kInterpPenalty[mids] * tau0;
        }
  }
  // Fixed-order CTA reduction.
  __shared__ double s_el[kPThreads], s_ei[kPThreads];
  s_el[threadIdx.x] = el;
  s_ei[threadIdx.x] = ei;
  __syncthreads();
  for (int h = kPThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_el[threadIdx.x] += s_el[threadIdx.x + h];
      s_ei[threadIdx.x] += s_ei[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s_el[0];
    partial[2 * blockIdx.x + 1] = s_ei[0];
  }
}

__global__ void __launch_bounds__(kPThreads)
prediction_errors_final_kernel(const double* __restrict__ partial, int nblocks,
                               double* __restrict__ result) {
  grid_dep_enter();
  __shared__ double s_el[kPThreads], s_ei[kPThreads];
  double el = 0.0, ei = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    el += partial[2 * i];
    ei += partial[2 * i + 1];
  }
  s_el[threadIdx.x] = el;
  s_ei[threadIdx.x] = ei;
  __syncthreads();
  for (int h = kPThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_el[threadIdx.x] += s_el[threadIdx.x + h];
      s_ei[threadIdx.x] += s_ei[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = s_el[0];
    result[1] = s_ei[0];
  }
}

}  // namespace

template <typename T>
cudaError_t launch_prediction_errors(const LevelK<T>& lv, const T* v, double tau0, double* partial,
                                     double* result, int level, cudaStream_t s) {
  // Sampled cells per axis: indices 0, 4, 8, .. below nc - 1.
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = (lv.ax[a].nc - 2) / 4 + 1;
  const int64_t nsampled = int64_t(m[0]) * m[1] * m[2];
  if (nsampled > INT32_MAX) return cudaErrorInvalidValue;
  const int blocks = static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>(kMinmaxBlocks, (nsampled + kPThreads - 1) / kPThreads)));
  // 19 nodes and their 7 + up to 8 neighbours per full block.
  TraceScope ts(kKPredErr, level, sizeof(T) * 27.0 * double(nsampled), s);
  ts.more_kernels(1);
  launch_pdl(prediction_errors_kernel<T>, dim3(blocks), dim3(kPThreads), 0, s, lv, v,
             static_cast<int>(nsampled), m[1], m[2], tau0, partial);
  launch_pdl(prediction_errors_final_kernel, dim3(1), dim3(kPThreads), 0, s,
             static_cast<const double*>(partial), blocks, result);
  return cudaGetLastError();
}

template cudaError_t launch_prediction_errors<float>(const LevelK<float>&, const float*, double,
                                                     double*, double*, int, cudaStream_t);
template cudaError_t launch_prediction_errors<double>(const LevelK<double>&, const double*, double,
                                                      double*, double*, int, cudaStream_t);

}  // namespace mgb
