// The coarse part's Lorenzo coder (the coarse part's coder in Algorithm 1;
// Section 4.2, Eq. (lorenzo)), as an exact integer transform of the coarse block's labels.
//
// The labels of N_{l~} are the linear quantization of Q_{l~}u with bin
// 2 tau_{l~}; replacing each by its Lorenzo residual r = q - pred(q) (pred
// the signed sum of the lower neighbours in the coarse grid, 0 outside it)
// predicts from the reconstructed values and leaves small codes for a
// smooth coarse part.  The arithmetic is 64-bit wrap-around, so the
// transform is a bijection; its inverse is a cumulative sum along every
// axis (the residual operator is the product of the backward differences).
//
// Encoding: the residuals of all coarse nodes are formed from the labels in
// place (read-only) into a compact array, then scattered back.  Decoding:
// the residuals are gathered, summed along axis 2, 1 and 0 (a thread per
// line), and scattered back.
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

struct Block {
  const int32_t* p[3];  // finest positions of the block's nodes per axis
  int m[3];             // block shape
  int64_t n1, n2;       // finest sizes of axes 1 and 2
};

__device__ __forceinline__ int64_t at(const Block& b, int i, int j, int k) {
  return (int64_t(b.p[0][i]) * b.n1 + b.p[1][j]) * b.n2 + b.p[2][k];
}

__global__ void __launch_bounds__(256)
lorenzo_residual_kernel(const int64_t* __restrict__ labels, Block b, uint64_t* __restrict__ out) {
  grid_dep_enter();
  const int64_t total = int64_t(b.m[0]) * b.m[1] * b.m[2];
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(t % b.m[2]);
    const int j = static_cast<int>((t / b.m[2]) % b.m[1]);
    const int i = static_cast<int>(t / (int64_t(b.m[1]) * b.m[2]));
    auto q = [&](int a, int c, int e) -> uint64_t {
      return (a < 0 || c < 0 || e < 0) ? 0ull : static_cast<uint64_t>(labels[at(b, a, c, e)]);
    };
    out[t] = q(i, j, k) - q(i, j, k - 1) - q(i, j - 1, k) - q(i - 1, j, k) + q(i, j - 1, k - 1) +
             q(i - 1, j, k - 1) + q(i - 1, j - 1, k) - q(i - 1, j - 1, k - 1);
  }
}

__global__ void __launch_bounds__(256)
block_gather_kernel(const int64_t* __restrict__ labels, Block b, uint64_t* __restrict__ out) {
  grid_dep_enter();
  const int64_t total = int64_t(b.m[0]) * b.m[1] * b.m[2];
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(t % b.m[2]);
    const int j = static_cast<int>((t / b.m[2]) % b.m[1]);
    const int i = static_cast<int>(t / (int64_t(b.m[1]) * b.m[2]));
    out[t] = static_cast<uint64_t>(labels[at(b, i, j, k)]);
  }
}

__global__ void __launch_bounds__(256)
block_scatter_kernel(const uint64_t* __restrict__ in, Block b, int64_t* __restrict__ labels) {
  grid_dep_enter();
  const int64_t total = int64_t(b.m[0]) * b.m[1] * b.m[2];
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(t % b.m[2]);
    const int j = static_cast<int>((t / b.m[2]) % b.m[1]);
    const int i = static_cast<int>(t / (int64_t(b.m[1]) * b.m[2]));
    labels[at(b, i, j, k)] = static_cast<int64_t>(in[t]);
  }
}

// Cumulative sum along one axis of the compact block (a thread per line).
__global__ void __launch_bounds__(256)
block_cumsum_kernel(uint64_t* __restrict__ v, int m0, int m1, int m2, int axis) {
  grid_dep_enter();
  const int64_t len = axis == 0 ? m0 : axis == 1 ? m1 : m2;
  const int64_t stride = axis == 0 ? int64_t(m1) * m2 : axis == 1 ? m2 : 1;
  const int64_t lines = int64_t(m0) * m1 * m2 / len;
  for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < lines;
       l += int64_t(gridDim.x) * blockDim.x) {
    // Line l -> its first element: the index with the summed axis at 0.
    const int64_t inner = l % stride, outer = l / stride;
    uint64_t* p = v + outer * len * stride + inner;
    uint64_t acc = 0;
    for (int64_t e = 0; e < len; ++e) {
      acc += p[e * stride];
      p[e * stride] = acc;
    }
  }
}

unsigned grid_for(int64_t n) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256)));
}

}  // namespace

cudaError_t launch_lorenzo(bool encode, int64_t* labels, const int64_t* dims3,
                           const int32_t* const* pos, const int64_t* shape3, uint64_t* tmp,
                           cudaStream_t s) {
  Block b;
  for (int a = 0; a < 3; ++a) {
    b.p[a] = pos[a];
    b.m[a] = static_cast<int>(shape3[a]);
  }
  b.n1 = dims3[1];
  b.n2 = dims3[2];
  const int64_t total = shape3[0] * shape3[1] * shape3[2];
  TraceScope ts(kKLorenzo, -1, 16.0 * double(total), s);
  if (encode) {
    ts.more_kernels(1);
    launch_pdl(lorenzo_residual_kernel, dim3(grid_for(total)), dim3(256), 0, s,
               static_cast<const int64_t*>(labels), b, tmp);
  } else {
    ts.more_kernels(4);
    launch_pdl(block_gather_kernel, dim3(grid_for(total)), dim3(256), 0, s,
               static_cast<const int64_t*>(labels), b, tmp);
    for (int a = 2; a >= 0; --a)
      launch_pdl(block_cumsum_kernel, dim3(grid_for(total / std::max<int64_t>(1, shape3[a]))),
                 dim3(256), 0, s, tmp, b.m[0], b.m[1], b.m[2], a);
  }
  launch_pdl(block_scatter_kernel, dim3(grid_for(total)), dim3(256), 0, s,
             static_cast<const uint64_t*>(tmp), b, labels);
  return cudaGetLastError();
}

}  // namespace mgb
