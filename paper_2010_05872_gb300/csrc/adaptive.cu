// Sampled prediction-error sums of the adaptive stopping level (Section 4.2,
// Algorithm 1 lines 4-9) on one level-l grid.
//
// The sampled blocks are the cells of the level-(l-1) grid whose index is a
// multiple of 4 along every axis (one block in four per dimension); a cell
// spans level-l indices cpos(b) .. cpos(b + 1), 3 nodes (2 for the end cell
// of an even axis).  Over the coefficient nodes of those blocks (nodes off
// N_{l-1}, 19 in a full 3^3 block) the kernel sums, in FP64,
//   E_Lorenzo += |Lorenzo prediction - v| + 1.22 tau0          (Eq. lorenzo)
//   E_interp  += |multilinear interpolation - v| + p tau0      (Eq. interp)
// with p = 0.369, 0.259, 0.182 for edge, plane and cube nodes (one, two or
// three midpoint coordinates).  The Lorenzo prediction is the signed sum of
// the 7 neighbours with some indices lowered by one (+ for an odd number of
// lowered indices); neighbours outside the grid count as 0.  Interpolation
// uses the level's own weights (the transform's iwl / iwr tables), of which
// the 1/2, 1/4, 1/8 stencils of Eq. (multilinear_interp) are the uniform
// case.
//
// One thread per sampled block (grid-stride), per-CTA partial sums reduced
// in a fixed order by a second single-CTA kernel: the result does not depend
// on timing.
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
prediction_errors_kernel(LevelK<T> lv, const T* __restrict__ v, int64_t nsampled, int m1, int m2,
                         double tau0, double* __restrict__ partial) {
  grid_dep_enter();
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  double el = 0.0, ei = 0.0;
  for (int64_t sidx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; sidx < nsampled;
       sidx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int s2 = static_cast<int>(sidx % m2);
    const int s1 = static_cast<int>((sidx / m2) % m1);
    const int s0 = static_cast<int>(sidx / (static_cast<int64_t>(m1) * m2));
    const int lo0 = cpos(4 * s0, n0), hi0 = cpos(4 * s0 + 1, n0);
    const int lo1 = cpos(4 * s1, n1), hi1 = cpos(4 * s1 + 1, n1);
    const int lo2 = cpos(4 * s2, n2), hi2 = cpos(4 * s2 + 1, n2);
    for (int i = lo0; i <= hi0; ++i) {
      const bool c0 = is_coef(i, n0);
      for (int j = lo1; j <= hi1; ++j) {
        const bool c1 = is_coef(j, n1);
        for (int k = lo2; k <= hi2; ++k) {
          const bool c2 = is_coef(k, n2);
          const int mids = int(c0) + int(c1) + int(c2);
          if (mids == 0) continue;
          auto at = [&](int a, int b, int c) -> double {
            return (a < 0 || b < 0 || c < 0)
                       ? 0.0
                       : static_cast<double>(v[(static_cast<int64_t>(a) * n1 + b) * n2 + c]);
          };
          const double x = at(i, j, k);
          const double lor = at(i, j, k - 1) + at(i, j - 1, k) + at(i - 1, j, k) -
                             at(i, j - 1, k - 1) - at(i - 1, j, k - 1) - at(i - 1, j - 1, k) +
                             at(i - 1, j - 1, k - 1);
          // Multilinear interpolation from the cell's corner nodes.
          int p0[2] = {i, i}, p1[2] = {j, j}, p2[2] = {k, k};
          double w0[2] = {1.0, 0.0}, w1[2] = {1.0, 0.0}, w2[2] = {1.0, 0.0};
          if (c0) {
            p0[0] = i - 1; p0[1] = i + 1;
            w0[0] = static_cast<double>(lv.ax[0].iwl[i]); w0[1] = static_cast<double>(lv.ax[0].iwr[i]);
          }
          if (c1) {
            p1[0] = j - 1; p1[1] = j + 1;
            w1[0] = static_cast<double>(lv.ax[1].iwl[j]); w1[1] = static_cast<double>(lv.ax[1].iwr[j]);
          }
          if (c2) {
            p2[0] = k - 1; p2[1] = k + 1;
            w2[0] = static_cast<double>(lv.ax[2].iwl[k]); w2[1] = static_cast<double>(lv.ax[2].iwr[k]);
          }
          double ip = 0.0;
          for (int a = 0; a < (c0 ? 2 : 1); ++a)
            for (int b = 0; b < (c1 ? 2 : 1); ++b)
              for (int c = 0; c < (c2 ? 2 : 1); ++c)
                ip += w0[a] * w1[b] * w2[c] * at(p0[a], p1[b], p2[c]);
          el += fabs(lor - x) + kLorenzoPenalty * tau0;
          ei += fabs(ip - x) + kInterpPenalty[mids] * tau0;
        }
      }
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
  const int blocks = static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>(kMinmaxBlocks, (nsampled + kPThreads - 1) / kPThreads)));
  // 19 nodes and their 7 + up to 8 neighbours per full block.
  TraceScope ts(kKPredErr, level, sizeof(T) * 27.0 * double(nsampled), s);
  ts.more_kernels(1);
  launch_pdl(prediction_errors_kernel<T>, dim3(blocks), dim3(kPThreads), 0, s, lv, v, nsampled,
             m[1], m[2], tau0, partial);
  launch_pdl(prediction_errors_final_kernel, dim3(1), dim3(kPThreads), 0, s,
             static_cast<const double*>(partial), blocks, result);
  return cudaGetLastError();
}

template cudaError_t launch_prediction_errors<float>(const LevelK<float>&, const float*, double,
                                                     double*, double*, int, cudaStream_t);
template cudaError_t launch_prediction_errors<double>(const LevelK<double>&, const double*, double,
                                                      double*, double*, int, cudaStream_t);

}  // namespace mgb
