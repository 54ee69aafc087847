// sm_103a kernels of level-wise quantization (Section 4.1; Algorithm 1 lines
// 17-22), dequantization and the value range that scales a relative bound.
#include <cfloat>
#include <cmath>

#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFlagNonfinite = 1u;
constexpr unsigned kFlagOverflow = 2u;

// Nearest integer with ties away from zero.  y - trunc(y) is exact in binary
// floating point, so comparing it with 0.5 decides the rounding exactly.
__device__ __forceinline__ long long round_half_away(double y) {
  const double t = trunc(y);
  const double fr = y - t;
  long long k = static_cast<long long>(t);
  if (fr >= 0.5) k += 1;
  else if (fr <= -0.5) k -= 1;
  return k;
}

// One CTA row loop over (j0, j1); threads sweep the contiguous axis.  The
// level of node (j0, j1, j2) is the max of the per-axis first-appearance
// levels, raised to the stopping level.
template <typename T>
__global__ void __launch_bounds__(kThreads)
quantize_kernel(const T* __restrict__ coeffs, int64_t* __restrict__ labels,
                const uint8_t* __restrict__ lev0, const uint8_t* __restrict__ lev1,
                const uint8_t* __restrict__ lev2, int64_t n0, int64_t n1, int64_t n2, int stop,
                LevelTable tab, unsigned int* __restrict__ flags) {
  const int64_t nrows = n0 * n1;
  unsigned bad = 0;
  for (int64_t r = blockIdx.y; r < nrows; r += gridDim.y) {
    const int64_t j0 = r / n1, j1 = r - j0 * n1;
    const int l01 = max(max(static_cast<int>(lev0[j0]), static_cast<int>(lev1[j1])), stop);
    const int64_t row = r * n2;
    for (int64_t j2 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j2 < n2;
         j2 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const int l = max(l01, static_cast<int>(lev2[j2]));
      const double x = static_cast<double>(coeffs[row + j2]);
      long long k = 0;
      if (!isfinite(x)) {
        bad |= kFlagNonfinite;
      } else {
        const double y = x / tab.q[l];
        if (fabs(y) >= 4611686018427387904.0) bad |= kFlagOverflow;  // 2^62
        else k = round_half_away(y);
      }
      labels[row + j2] = k;
    }
  }
  if (bad) atomicOr(flags, bad);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
dequantize_kernel(const int64_t* __restrict__ labels, T* __restrict__ coeffs,
                  const uint8_t* __restrict__ lev0, const uint8_t* __restrict__ lev1,
                  const uint8_t* __restrict__ lev2, int64_t n0, int64_t n1, int64_t n2, int stop,
                  LevelTable tab) {
  const int64_t nrows = n0 * n1;
  for (int64_t r = blockIdx.y; r < nrows; r += gridDim.y) {
    const int64_t j0 = r / n1, j1 = r - j0 * n1;
    const int l01 = max(max(static_cast<int>(lev0[j0]), static_cast<int>(lev1[j1])), stop);
    const int64_t row = r * n2;
    for (int64_t j2 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j2 < n2;
         j2 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const int l = max(l01, static_cast<int>(lev2[j2]));
      coeffs[row + j2] = static_cast<T>(static_cast<double>(labels[row + j2]) * tab.q[l]);
    }
  }
}

// Block-wide min/max into per-block partials; non-finite elements flagged.
template <typename T>
__global__ void __launch_bounds__(kThreads)
minmax_partial_kernel(const T* __restrict__ data, int64_t count, double* __restrict__ partial,
                      unsigned int* __restrict__ flags) {
  __shared__ double smin[kThreads], smax[kThreads];
  double mn = DBL_MAX, mx = -DBL_MAX;
  unsigned bad = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = static_cast<double>(data[i]);
    if (!isfinite(v)) { bad = kFlagNonfinite; continue; }
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  if (bad) atomicOr(flags, bad);
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = smin[0];
    partial[2 * blockIdx.x + 1] = smax[0];
  }
}

__global__ void __launch_bounds__(kThreads)
minmax_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ result) {
  __shared__ double smin[kThreads], smax[kThreads];
  double mn = DBL_MAX, mx = -DBL_MAX;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    mn = fmin(mn, partial[2 * i]);
    mx = fmax(mx, partial[2 * i + 1]);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = smin[0];
    result[1] = smax[0];
  }
}

dim3 row_grid(int64_t n0, int64_t n1, int64_t n2) {
  const int64_t bx = (n2 + kThreads - 1) / kThreads;
  const int64_t nrows = n0 * n1;
  unsigned gx = static_cast<unsigned>(bx < 64 ? bx : 64);
  unsigned gy = static_cast<unsigned>(nrows < 65535 ? nrows : 65535);
  return dim3(gx, gy);
}

}  // namespace

template <typename T>
cudaError_t launch_quantize(const T* coeffs, int64_t* labels, const uint8_t* lev0,
                            const uint8_t* lev1, const uint8_t* lev2, int64_t n0, int64_t n1,
                            int64_t n2, int stop_level, const LevelTable& tab,
                            unsigned int* flags, cudaStream_t s) {
  TraceScope ts(kKQuantize, -1, double(n0) * n1 * n2 * (sizeof(T) + 8), s);
  quantize_kernel<T><<<row_grid(n0, n1, n2), kThreads, 0, s>>>(coeffs, labels, lev0, lev1, lev2,
                                                                n0, n1, n2, stop_level, tab, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dequantize(const int64_t* labels, T* coeffs, const uint8_t* lev0,
                              const uint8_t* lev1, const uint8_t* lev2, int64_t n0, int64_t n1,
                              int64_t n2, int stop_level, const LevelTable& tab, cudaStream_t s) {
  TraceScope ts(kKDequantize, -1, double(n0) * n1 * n2 * (sizeof(T) + 8), s);
  dequantize_kernel<T><<<row_grid(n0, n1, n2), kThreads, 0, s>>>(labels, coeffs, lev0, lev1, lev2,
                                                                  n0, n1, n2, stop_level, tab);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_minmax(const T* data, int64_t count, double* partial, unsigned int* flags,
                          double* result, cudaStream_t s) {
  int64_t blocks = (count + kThreads - 1) / kThreads;
  if (blocks > kMinmaxBlocks) blocks = kMinmaxBlocks;
  if (blocks < 1) blocks = 1;
  TraceScope ts(kKMinmax, -1, double(count) * sizeof(T), s);
  minmax_partial_kernel<T><<<static_cast<unsigned>(blocks), kThreads, 0, s>>>(data, count, partial,
                                                                             flags);
  minmax_final_kernel<<<1, kThreads, 0, s>>>(partial, static_cast<int>(blocks), result);
  return cudaGetLastError();
}

#define MGB_INST(T)                                                                              \
  template cudaError_t launch_quantize<T>(const T*, int64_t*, const uint8_t*, const uint8_t*,   \
                                          const uint8_t*, int64_t, int64_t, int64_t, int,        \
                                          const LevelTable&, unsigned int*, cudaStream_t);       \
  template cudaError_t launch_dequantize<T>(const int64_t*, T*, const uint8_t*, const uint8_t*, \
                                            const uint8_t*, int64_t, int64_t, int64_t, int,      \
                                            const LevelTable&, cudaStream_t);                    \
  template cudaError_t launch_minmax<T>(const T*, int64_t, double*, unsigned int*, double*,     \
                                        cudaStream_t);
MGB_INST(float)
MGB_INST(double)
#undef MGB_INST

}  // namespace mgb
