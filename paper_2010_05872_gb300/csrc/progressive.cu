// Progressive recomposition and analysis on a reduced representation
// (Section 1, data refactoring; Section 6.2.2, iso-surface use case).
//
// gather_level_kernel copies the nodes of N_k out of an array in the finest
// layout into a compact level-k grid (positions from the plan), so that the
// recomposition of the levels up to k can run on the reduced grid alone.
//
// iso_area_kernel measures the iso-surface v = iso of a 3D grid function by
// marching tetrahedra: each cell is split into the 6 tetrahedra around its
// main diagonal (corner 0 to corner 7, corner c at offsets (c>>2 & 1,
// c>>1 & 1, c & 1)), v is linear on each, a vertex is above when v > iso,
// and the surface crosses an edge joining an above and a below vertex at
// the root of the linear interpolant.  One vertex apart gives a triangle,
// two apart a quadrilateral split along the diagonal from the (below 0,
// above 0) edge point to the (below 1, above 1) one.  The geometry is
// formed in the grid's precision and each cell's area is added in FP64;
// per-CTA partial sums are reduced in a fixed order.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <limits>

#include "pdl.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

constexpr int kIThreads = 256;

template <typename T>
__global__ void __launch_bounds__(256)
gather_level_kernel(const T* __restrict__ src, int64_t n1, int64_t n2, const int32_t* __restrict__ p0,
                    const int32_t* __restrict__ p1, const int32_t* __restrict__ p2, int m0, int m1,
                    int m2, T* __restrict__ dst) {
  grid_dep_enter();
  const int64_t total = int64_t(m0) * m1 * m2;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i2 = static_cast<int>(t % m2);
    const int i1 = static_cast<int>((t / m2) % m1);
    const int i0 = static_cast<int>(t / (int64_t(m1) * m2));
    dst[t] = src[(int64_t(p0[i0]) * n1 + p1[i1]) * n2 + p2[i2]];
  }
}

template <typename T>
__device__ __forceinline__ T tri_area(const T a[3], const T b[3], const T c[3]) {
  const T u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
  const T w0 = c[0] - a[0], w1 = c[1] - a[1], w2 = c[2] - a[2];
  const T x = u1 * w2 - u2 * w1, y = u2 * w0 - u0 * w2, z = u0 * w1 - u1 * w0;
  return T(0.5) * sqrt(x * x + y * y + z * z);
}

// Area of the iso-surface inside one tetrahedron (vertices q, values f,
// classification up).
template <typename T>
__device__ T tet_area(const T q[4][3], const T f[4], const bool up[4], T iso) {
  int nu = 0;
  for (int i = 0; i < 4; ++i) nu += up[i];
  if (nu == 0 || nu == 4) return T(0);
  auto cross = [&](int a, int b, T out[3]) {
    const T t = (iso - f[a]) / (f[b] - f[a]);
    for (int d = 0; d < 3; ++d) out[d] = q[a][d] + t * (q[b][d] - q[a][d]);
  };
  if (nu == 1 || nu == 3) {
    // The lone vertex and the other three, in increasing index order.
    const bool lone_up = nu == 1;
    int one = 0;
    for (int i = 0; i < 4; ++i)
      if (up[i] == lone_up) one = i;
    T pts[3][3];
    int m = 0;
    for (int i = 0; i < 4; ++i)
      if (i != one) cross(one, i, pts[m++]);
    return tri_area(pts[0], pts[1], pts[2]);
  }
  int dn[2], upv[2], a = 0, b = 0;
  for (int i = 0; i < 4; ++i) {
    if (up[i]) upv[b++] = i;
    else dn[a++] = i;
  }
  T q0[3], q1[3], q2[3], q3[3];
  cross(dn[0], upv[0], q0);
  cross(dn[0], upv[1], q1);
  cross(dn[1], upv[1], q2);
  cross(dn[1], upv[0], q3);
  return tri_area(q0, q1, q2) + tri_area(q0, q2, q3);
}

__constant__ int kTets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

template <typename T>
__global__ void __launch_bounds__(kIThreads)
iso_area_kernel(const T* __restrict__ v, int n0, int n1, int n2, const double* __restrict__ x0,
                const double* __restrict__ x1, const double* __restrict__ x2, T iso_cls, T iso,
                double* __restrict__ partial) {
  grid_dep_enter();
  const int64_t cells = int64_t(n0 - 1) * (n1 - 1) * (n2 - 1);
  double acc = 0.0;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < cells;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(t % (n2 - 1));
    const int j = static_cast<int>((t / (n2 - 1)) % (n1 - 1));
    const int i = static_cast<int>(t / (int64_t(n1 - 1) * (n2 - 1)));
    T f[8];
    bool up[8];
    int nu = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      f[c] = v[(int64_t(i + (c >> 2 & 1)) * n1 + (j + (c >> 1 & 1))) * n2 + (k + (c & 1))];
      up[c] = f[c] > iso_cls;
      nu += up[c];
    }
    if (nu == 0 || nu == 8) continue;
    const T px[2] = {T(x0[i]), T(x0[i + 1])}, py[2] = {T(x1[j]), T(x1[j + 1])},
            pz[2] = {T(x2[k]), T(x2[k + 1])};
    T cell = T(0);
    for (int tt = 0; tt < 6; ++tt) {
      T q[4][3], fv[4];
      bool uv[4];
      for (int m = 0; m < 4; ++m) {
        const int c = kTets[tt][m];
        q[m][0] = px[c >> 2 & 1];
        q[m][1] = py[c >> 1 & 1];
        q[m][2] = pz[c & 1];
        fv[m] = f[c];
        uv[m] = up[c];
      }
      cell += tet_area(q, fv, uv, iso);
    }
    acc += static_cast<double>(cell);
  }
  __shared__ double s_a[kIThreads];
  s_a[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kIThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s_a[threadIdx.x] += s_a[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s_a[0];
}

__global__ void __launch_bounds__(kIThreads)
sum_partials_kernel(const double* __restrict__ partial, int n, double* __restrict__ result) {
  grid_dep_enter();
  __shared__ double s_a[kIThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  s_a[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kIThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s_a[threadIdx.x] += s_a[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) result[0] = s_a[0];
}

}  // namespace

template <typename T>
cudaError_t launch_gather_level(const T* src, const int64_t* dims3, const int32_t* const* pos,
                                const int64_t* shape3, T* dst, cudaStream_t s) {
  const int64_t total = shape3[0] * shape3[1] * shape3[2];
  const unsigned grid =
      static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(4 * 152 * 8, (total + 255) / 256)));
  TraceScope ts(kKGather, -1, 2.0 * sizeof(T) * double(total), s);
  launch_pdl(gather_level_kernel<T>, dim3(grid), dim3(256), 0, s, src, dims3[1], dims3[2], pos[0],
             pos[1], pos[2], static_cast<int>(shape3[0]), static_cast<int>(shape3[1]),
             static_cast<int>(shape3[2]), dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iso_area(const T* v, const int64_t* dims3, const double* const* x, double iso,
                            double* partial, double* result, cudaStream_t s) {
  // Classification v > iso in the grid's precision: against the largest
  // value of T not above iso, which gives the same answer as comparing the
  // widened value with iso.
  T iso_cls = static_cast<T>(iso);
  if (static_cast<double>(iso_cls) > iso) iso_cls = std::nextafter(iso_cls, -std::numeric_limits<T>::infinity());
  const int64_t cells = (dims3[0] - 1) * (dims3[1] - 1) * (dims3[2] - 1);
  const int blocks = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>(kMinmaxBlocks, (cells + kIThreads - 1) / kIThreads)));
  TraceScope ts(kKIsoArea, -1, sizeof(T) * double(dims3[0] * dims3[1] * dims3[2]), s);
  ts.more_kernels(1);
  launch_pdl(iso_area_kernel<T>, dim3(blocks), dim3(kIThreads), 0, s, v, static_cast<int>(dims3[0]),
             static_cast<int>(dims3[1]), static_cast<int>(dims3[2]), x[0], x[1], x[2], iso_cls,
             static_cast<T>(iso), partial);
  launch_pdl(sum_partials_kernel, dim3(1), dim3(kIThreads), 0, s,
             static_cast<const double*>(partial), blocks, result);
  return cudaGetLastError();
}

template cudaError_t launch_gather_level<float>(const float*, const int64_t*, const int32_t* const*,
                                                const int64_t*, float*, cudaStream_t);
template cudaError_t launch_gather_level<double>(const double*, const int64_t*,
                                                 const int32_t* const*, const int64_t*, double*,
                                                 cudaStream_t);
template cudaError_t launch_iso_area<float>(const float*, const int64_t*, const double* const*,
                                            double, double*, double*, cudaStream_t);
template cudaError_t launch_iso_area<double>(const double*, const int64_t*, const double* const*,
                                             double, double*, double*, cudaStream_t);

}  // namespace mgb
