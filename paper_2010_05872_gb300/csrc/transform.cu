// Generic tiled load-vector kernel of one level transition l -> l-1 (Section
// 2 step 4, Section 5.2): coefficients, mass multiply and restriction fused
// on a 3D tile staged in shared memory.  Used for 1D levels and for levels
// too small or too wide for the marching kernel of load_vector.cu.
#include <algorithm>

#include "pdl.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {

namespace {

__device__ __forceinline__ int cpos(int k, int n) { return min(2 * k, n - 1); }
__device__ __forceinline__ bool is_coef(int j, int n) { return (j & 1) && (j != n - 1); }
__device__ __forceinline__ int nodal_k(int j, int n, int nc) { return j == n - 1 ? nc - 1 : (j >> 1); }

constexpr int kThreads = 256;

struct Tile {
  int t0, t1, t2;  // coarse nodes per CTA along each axis
};

template <typename T>
Tile pick_tile(const LevelK<T>& lv) {
  if (lv.ax[0].n == 1 && lv.ax[1].n == 1) return {1, 1, 512};
  if (lv.ax[0].n == 1) return {1, 8, 64};
  return {2, 4, 32};
}

inline int region(int tk, int n) { return n == 1 ? 1 : 2 * tk + 3; }

// ---------------------------------------------------------------------------
// Load vector: w (coefficients or stored u_mc) -> F = (R0 x R1 x R2) w.
// One CTA per coarse tile; the fine region it needs (tile +-2 fine nodes) is
// staged in shared memory, w is formed there, and the separable 5-tap
// restriction runs axis 2, then 1, then 0 on the staged data.
// ---------------------------------------------------------------------------
template <typename T, bool DEC>
__global__ void __launch_bounds__(kThreads)
load_vector_kernel(LevelK<T> lv, const T* __restrict__ fine, T* __restrict__ coarse,
                   T* __restrict__ F, int tk0, int tk1, int tk2) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int K0 = blockIdx.z * tk0, K1 = blockIdx.y * tk1, K2 = blockIdx.x * tk2;
  const int T0 = min(tk0, c0 - K0), T1 = min(tk1, c1 - K1), T2 = min(tk2, c2 - K2);
  const int lo0 = max(2 * K0 - 2, 0), hi0 = min(2 * (K0 + T0 - 1) + 2, n0 - 1);
  const int lo1 = max(2 * K1 - 2, 0), hi1 = min(2 * (K1 + T1 - 1) + 2, n1 - 1);
  const int lo2 = max(2 * K2 - 2, 0), hi2 = min(2 * (K2 + T2 - 1) + 2, n2 - 1);
  const int S0 = hi0 - lo0 + 1, S1 = hi1 - lo1 + 1, S2 = hi2 - lo2 + 1;
  const int S12 = S1 * S2, S = S0 * S12;
  T* sv = smem;
  T* sw = sv + S;
  T* g1 = sw + S;              // S0 x S1 x T2
  T* g2 = g1 + S0 * S1 * T2;   // S0 x T1 x T2

  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const int a = i / S12, r = i - a * S12, b = r / S2, c = r - b * S2;
    sv[i] = fine[(static_cast<int64_t>(lo0 + a) * n1 + (lo1 + b)) * n2 + (lo2 + c)];
  }
  __syncthreads();

  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const int a = i / S12, r = i - a * S12, b = r / S2, c = r - b * S2;
    const int j0 = lo0 + a, j1 = lo1 + b, j2 = lo2 + c;
    const bool q0 = is_coef(j0, n0), q1 = is_coef(j1, n1), q2 = is_coef(j2, n2);
    T w;
    if (!(q0 || q1 || q2)) {
      w = T(0);
      const int k0 = nodal_k(j0, n0, c0), k1 = nodal_k(j1, n1, c1), k2 = nodal_k(j2, n2, c2);
      if (k0 >= K0 && k0 < K0 + T0 && k1 >= K1 && k1 < K1 + T1 && k2 >= K2 && k2 < K2 + T2 &&
          cpos(k0, n0) == j0 && cpos(k1, n1) == j1 && cpos(k2, n2) == j2)
        coarse[(static_cast<int64_t>(k0) * c1 + k1) * c2 + k2] = sv[i];
    } else if (DEC) {
      // Multilinear interpolant from the 2^m coarse corners (m = number of
      // axes along which the node is a coefficient node).
      const T wl0 = q0 ? lv.ax[0].iwl[j0] : T(1), wr0 = q0 ? lv.ax[0].iwr[j0] : T(0);
      const T wl1 = q1 ? lv.ax[1].iwl[j1] : T(1), wr1 = q1 ? lv.ax[1].iwr[j1] : T(0);
      const T wl2 = q2 ? lv.ax[2].iwl[j2] : T(1), wr2 = q2 ? lv.ax[2].iwr[j2] : T(0);
      const int o0 = q0 ? S12 : 0, o1 = q1 ? S2 : 0, o2 = q2 ? 1 : 0;
      const T* p = sv + i;
      T acc = T(0);
#pragma unroll
      for (int e0 = 0; e0 < 2; ++e0) {
        const T w0 = e0 ? wr0 : wl0;
        const int d0 = e0 ? o0 : -o0;
        if (e0 && !q0) continue;
#pragma unroll
        for (int e1 = 0; e1 < 2; ++e1) {
          const T w1 = e1 ? wr1 : wl1;
          const int d1 = e1 ? o1 : -o1;
          if (e1 && !q1) continue;
          T acc2 = T(0);
          if (q2) acc2 = wl2 * p[d0 + d1 - o2] + wr2 * p[d0 + d1 + o2];
          else acc2 = p[d0 + d1];
          acc += w0 * w1 * acc2;
        }
      }
      w = sv[i] - acc;
    } else {
      w = sv[i];
    }
    sw[i] = w;
  }
  __syncthreads();

  // Axis 2 restriction: g1[a][b][t] = sum_o rw2[k2][o] w[a][b][cpos(k2)+o-2]
  {
    const T* rw = lv.ax[2].rw;
    const int cnt = S0 * S1 * T2;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int ab = i / T2, t = i - ab * T2;
      const int k = K2 + t;
      const int c = cpos(k, n2) - lo2;
      const T* src = sw + ab * S2;
      T acc = T(0);
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int cc = c + o - 2;
        if (cc >= 0 && cc < S2) acc += rw[k * 5 + o] * src[cc];
      }
      g1[i] = acc;
    }
  }
  __syncthreads();
  // Axis 1 restriction: g2[a][t1][t2]
  {
    const T* rw = lv.ax[1].rw;
    const int cnt = S0 * T1 * T2;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int a = i / (T1 * T2), r = i - a * (T1 * T2), t1 = r / T2, t2 = r - t1 * T2;
      const int k = K1 + t1;
      const int c = cpos(k, n1) - lo1;
      T acc = T(0);
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int cc = c + o - 2;
        if (cc >= 0 && cc < S1) acc += rw[k * 5 + o] * g1[(a * S1 + cc) * T2 + t2];
      }
      g2[i] = acc;
    }
  }
  __syncthreads();
  // Axis 0 restriction and store.
  {
    const T* rw = lv.ax[0].rw;
    const int cnt = T0 * T1 * T2;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int t0 = i / (T1 * T2), r = i - t0 * (T1 * T2), t1 = r / T2, t2 = r - t1 * T2;
      const int k = K0 + t0;
      const int c = cpos(k, n0) - lo0;
      T acc = T(0);
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int cc = c + o - 2;
        if (cc >= 0 && cc < S0) acc += rw[k * 5 + o] * g2[(cc * T1 + t1) * T2 + t2];
      }
      F[(static_cast<int64_t>(k) * c1 + (K1 + t1)) * c2 + (K2 + t2)] = acc;
    }
  }
}

inline unsigned ceil_div(int64_t a, int64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

}  // namespace

template <typename T>
cudaError_t launch_load_vector(const LevelK<T>& lv, bool dec, const T* fine, T* coarse, T* F,
                               int level, unsigned int* status, cudaStream_t s) {
  const double nfine = double(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  const double ncoarse = double(lv.ax[0].nc) * lv.ax[1].nc * lv.ax[2].nc;
  if (load_vector_march_supported(lv)) {
    TraceScope ts(dec ? kKLoadVectorDec : kKLoadVectorRec, level,
                  sizeof(T) * (nfine + 2 * ncoarse), s);
    return launch_load_vector_march(lv, dec, fine, coarse, F, status, s);
  }
  const Tile t = pick_tile(lv);
  const int tk0 = lv.ax[0].n == 1 ? 1 : t.t0, tk1 = lv.ax[1].n == 1 ? 1 : t.t1, tk2 = t.t2;
  const int S0 = region(tk0, lv.ax[0].n), S1 = region(tk1, lv.ax[1].n), S2 = region(tk2, lv.ax[2].n);
  const size_t smem = sizeof(T) * (2 * static_cast<size_t>(S0) * S1 * S2 +
                                   static_cast<size_t>(S0) * S1 * tk2 +
                                   static_cast<size_t>(S0) * tk1 * tk2);
  dim3 grid(ceil_div(lv.ax[2].nc, tk2), ceil_div(lv.ax[1].nc, tk1), ceil_div(lv.ax[0].nc, tk0));
  const double nf = double(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  const double ncs = double(lv.ax[0].nc) * lv.ax[1].nc * lv.ax[2].nc;
  TraceScope ts(dec ? kKLoadVectorDec : kKLoadVectorRec, level, sizeof(T) * (nf + 2 * ncs), s);
  if (dec) {
    allow_dynamic_smem(load_vector_kernel<T, true>, smem);
    launch_pdl(load_vector_kernel<T, true>, dim3(grid), dim3(kThreads), smem, s, lv, fine, coarse,
               F, tk0, tk1, tk2);
  } else {
    allow_dynamic_smem(load_vector_kernel<T, false>, smem);
    launch_pdl(load_vector_kernel<T, false>, dim3(grid), dim3(kThreads), smem, s, lv, fine, coarse,
               F, tk0, tk1, tk2);
  }
  return cudaGetLastError();
}

template cudaError_t launch_load_vector<float>(const LevelK<float>&, bool, const float*, float*,
                                               float*, int, unsigned int*, cudaStream_t);
template cudaError_t launch_load_vector<double>(const LevelK<double>&, bool, const double*,
                                                double*, double*, int, unsigned int*, cudaStream_t);



}  // namespace mgb
