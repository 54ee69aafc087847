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
// per-CTA partial sums are reduced in a fixed order.  A CTA takes whole rows
// of cells (fixed (i, j)), its threads running along the contiguous axis.
#include <algorithm>
#include <cfloat>
#include <climits>
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

// A tetrahedron vertex: position and value.
template <typename T>
struct TV {
  T x, y, z, f;
};

template <typename T>
__device__ __forceinline__ TV<T> pick(bool c, const TV<T>& a, const TV<T>& b) {
  return {c ? a.x : b.x, c ? a.y : b.y, c ? a.z : b.z, c ? a.f : b.f};
}

// Crossing of the iso-surface on the edge from vertex a to vertex b.
template <typename T>
__device__ __forceinline__ void edge_cross(const TV<T>& a, const TV<T>& b, T iso, T out[3]) {
  const T t = (iso - a.f) / (b.f - a.f);
  out[0] = a.x + t * (b.x - a.x);
  out[1] = a.y + t * (b.y - a.y);
  out[2] = a.z + t * (b.z - a.z);
}

// Area of the iso-surface inside one tetrahedron (vertices v, up[i] when
// v[i] is above), in one code path for every case: the vertices are put in
// the order below-first, each side in index order (slots s0..s3); with nu
// vertices above, the polygon's corners lie on the edges
//   nu = 2: (s0,s2) (s0,s3) (s1,s3) (s1,s2), split along the first to third,
//   nu = 1: (s3,s0) (s3,s1) (s3,s2), nu = 3: (s0,s1) (s0,s2) (s0,s3),
// a triangle being a quadrilateral with its last corner repeated.
template <typename T>
__device__ T tet_area(const TV<T> v[4], const bool up[4], T iso) {
  int nu = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) nu += up[i];
  if (nu == 0 || nu == 4) return T(0);
  const int nd = 4 - nu;
  int slot[4], cu = 0, cd = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    slot[i] = up[i] ? nd + cu : cd;
    cu += up[i];
    cd += !up[i];
  }
  TV<T> sv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    sv[k] = pick(slot[0] == k, v[0], pick(slot[1] == k, v[1], pick(slot[2] == k, v[2], v[3])));
  const bool quad = nu == 2, one_up = nu == 1;
  // Edge endpoints (first, second) of the four corners.
  const TV<T> a0 = quad ? sv[0] : (one_up ? sv[3] : sv[0]);
  const TV<T> b0 = quad ? sv[2] : (one_up ? sv[0] : sv[1]);
  const TV<T> a1 = quad ? sv[0] : (one_up ? sv[3] : sv[0]);
  const TV<T> b1 = quad ? sv[3] : (one_up ? sv[1] : sv[2]);
  const TV<T> a2 = quad ? sv[1] : (one_up ? sv[3] : sv[0]);
  const TV<T> b2 = quad ? sv[3] : (one_up ? sv[2] : sv[3]);
  const TV<T> a3 = quad ? sv[1] : a2;
  const TV<T> b3 = quad ? sv[2] : b2;
  T q0[3], q1[3], q2[3], q3[3];
  edge_cross(a0, b0, iso, q0);
  edge_cross(a1, b1, iso, q1);
  edge_cross(a2, b2, iso, q2);
  edge_cross(a3, b3, iso, q3);
  return tri_area(q0, q1, q2) + tri_area(q0, q2, q3);
}

template <typename T>
__global__ void __launch_bounds__(kIThreads)
iso_area_kernel(const T* __restrict__ v, int n0, int n1, int n2, const double* __restrict__ x0,
                const double* __restrict__ x1, const double* __restrict__ x2, T iso_cls, T iso,
                double* __restrict__ partial) {
  grid_dep_enter();
  // A CTA takes rows of cells (i, j) in turn; each warp classifies 32
  // consecutive cells of a row at a time and appends the ones the surface
  // crosses (a vertex above and one not), in order, to a 64-entry ring in
  // shared memory; whenever 32 are pending, every lane measures one.  The
  // order of the work, and so of the sums, depends on the data only.
  __shared__ int s_q[kIThreads / 32][64][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int (*q)[2] = s_q[warp];
  int head = 0, pending = 0;  // ring: oldest entry, entries waiting (<= 31 between steps)
  const int rows = (n0 - 1) * (n1 - 1), rowlen = n2 - 1;
  const int64_t plane = int64_t(n1) * n2;
  double acc = 0.0;
  auto corner = [&](int r, int k, int c) -> T {
    const int i = r / (n1 - 1), j = r - i * (n1 - 1);
    return v[int64_t(i + (c >> 2 & 1)) * plane + int64_t(j + (c >> 1 & 1)) * n2 + (k + (c & 1))];
  };
  // Area of the surface inside cell (r, k).
  auto measure = [&](int r, int k) -> T {
    const int i = r / (n1 - 1), j = r - i * (n1 - 1);
    T f[8];
    bool up[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      f[c] = corner(r, k, c);
      up[c] = f[c] > iso_cls;
    }
    const T px[2] = {T(x0[i]), T(x0[i + 1])}, py[2] = {T(x1[j]), T(x1[j + 1])},
            pz[2] = {T(x2[k]), T(x2[k + 1])};
    const int tets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                            {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
    T cell = T(0);
#pragma unroll
    for (int tt = 0; tt < 6; ++tt) {
      TV<T> tv[4];
      bool uv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int c = tets[tt][m];
        tv[m] = {px[c >> 2 & 1], py[c >> 1 & 1], pz[c & 1], f[c]};
        uv[m] = up[c];
      }
      cell += tet_area(tv, uv, iso);
    }
    return cell;
  };
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    for (int k0 = warp * 32; k0 < rowlen; k0 += nwarps * 32) {
      const int k = k0 + lane;
      bool hit = false;
      if (k < rowlen) {
        int nu = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) nu += corner(r, k, c) > iso_cls;
        hit = nu != 0 && nu != 8;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int at = (head + pending + __popc(m & ((1u << lane) - 1u))) & 63;
        q[at][0] = r;
        q[at][1] = k;
      }
      pending += __popc(m);
      __syncwarp();
      if (pending >= 32) {
        const int at = (head + lane) & 63;
        const int rr = q[at][0], kk = q[at][1];
        __syncwarp();  // read before the slots are reused
        acc += static_cast<double>(measure(rr, kk));
        head = (head + 32) & 63;
        pending -= 32;
      }
    }
  }
  if (lane < pending) {
    const int at = (head + lane) & 63;
    acc += static_cast<double>(measure(q[at][0], q[at][1]));
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
  const int64_t rows = (dims3[0] - 1) * (dims3[1] - 1);
  if (rows > INT32_MAX) return cudaErrorInvalidValue;
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kMinmaxBlocks, rows)));
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
