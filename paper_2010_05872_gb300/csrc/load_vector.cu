// Marching load-vector kernel for the level-l grids of 2D and 3D fields
// (Section 2 step 4 and Section 5.2: coefficient computation, mass multiply
// and restriction to the coarse load vector, fused).
//
// What is computed.  With R = R0 x R1 x R2 the load-vector restriction
// P^T M_f of each axis (5 fine taps per coarse node) and v_c the values of
// `fine` on the coarse nodes N_{l-1}:
//   decomposition : F = R (v - Pi v_c) = R v - (R P) v_c,
//   recomposition : F = R (v with its N_{l-1} values zeroed) = R v - (R S) v_c,
// where P is the prolongation (Pi on the coarse values) and S places coarse
// values on their fine nodes.  R P (the coarse mass matrix in the load-vector
// scaling) and R S are tridiagonal on the coarse grid and tensor products,
// built per axis on the host from the same tables as R.  So a plane of v
// needs only two separable passes, R v over every fine node and X v_c over
// the nodal ones, and no interpolant is formed.  The values of `fine` on
// N_{l-1} are gathered into `coarse` on the way.
//
// Work split: a CTA owns T1 coarse rows along axis 1 and all coarse columns
// of axis 2 (for 2D levels, a chunk of them), and marches through a chunk of
// fine planes along axis 0.  The 2 T1 + 3 fine rows a CTA needs from one
// plane are contiguous in memory, so a plane enters shared memory by one 1D
// TMA bulk copy (cp.async.bulk, completion on an mbarrier) of the enclosing
// 16-byte-aligned range, issued by thread 0; NS plane buffers cycle with
// NS - 1 copies in flight.  Bytes past the end of the array are never
// requested; the at most 15 bytes there come in by plain loads.  Virtual rows
// and columns outside the grid read finite data (zeroed buffers or
// neighbouring rows) under zero weights.
//
// A thread owns coarse column k2 and reads the 5 fine values around it in
// every staged row: one 5-tap sum for R2 and, on nodal rows of nodal planes,
// one for X2.  Row s of the tile feeds the three coarse rows it can touch
// with weights from a per-CTA table (compile-time row loop), and each
// finished plane feeds the three coarse planes it can touch, accumulated in
// registers; a coarse plane is stored to F once its last fine plane has
// passed.  Waits on the mbarriers give up after 2 s, record the failure in
// `status` and end the CTA.
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
#include "kernels.cuh"
#include "lv_tile.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

template <typename T, bool DEC, int NS, int T1C, bool THREE, int CPT, bool REG>
__global__ void __launch_bounds__(kLvMaxThreads)
load_vector_march_kernel(LevelK<T> lv, const T* __restrict__ fine, T* __restrict__ coarse,
                         T* __restrict__ F, MarchGeom g, uint64_t fine_count,
                         unsigned int* __restrict__ status) {
  grid_dep_enter();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  load_vector_march_tile<T, DEC, NS, T1C, THREE, false, CPT, 1, REG>(lv, fine, coarse, F, g, fine_count, status,
                                                 blockIdx.x, smem_raw);
}

}  // namespace

// Whether a level's grid stays in L2 (it then takes the MarchCfg *_L2 shape
// and short marches).
template <typename T>
bool l2_resident(const LevelK<T>& lv) {
  const uint64_t count = uint64_t(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  return count * sizeof(T) <= kL2ResidentBytes;
}

template <typename T>
bool load_vector_march_supported(const LevelK<T>& lv_in) {
  // 2D and 3D levels large enough to fill the GPU (1D and tiny levels use
  // the generic tiled kernel).
  using C = MarchCfg<T>;
  const int64_t nf = int64_t(lv_in.ax[0].n) * lv_in.ax[1].n * lv_in.ax[2].n;
  if (lv_in.ax[0].n == 1 && lv_in.ax[1].n == 1) return false;
  if (nf < (int64_t(1) << 17)) return false;
  LevelK<T> lv = lv_in;
  if (lv.ax[0].n == 1) std::swap(lv.ax[0], lv.ax[1]);
  MarchGeom g{};
  return l2_resident(lv) ? plan_geometry(lv, g, C::CPT_L2, C::T1_L2, C::NS_L2)
                         : plan_geometry(lv, g, C::CPT, C::T1, C::NS);
}

template <typename T, int NS, int T1C, int CPT>
cudaError_t launch_march_shape(const LevelK<T>& lv, bool dec, const T* fine, T* coarse, T* F,
                               unsigned int* status, cudaStream_t s) {
  const int c0 = lv.ax[0].nc;
  MarchGeom g{};
  if (!plan_geometry(lv, g, CPT, T1C, NS)) return cudaErrorInvalidConfiguration;
  const bool three = lv.ax[1].n > 1;
  const size_t smem = sizeof(T) * static_cast<size_t>(NS) * g.BUF;
  using KernelFn = void (*)(LevelK<T>, const T*, T*, T*, MarchGeom, uint64_t, unsigned int*);
  KernelFn kernel;
  // Odd axes (every 2^k + 1 grid): coarse nodes at 2k, zero taps skipped.
  const bool reg = (lv.ax[0].n & 1) && (lv.ax[1].n & 1) && (lv.ax[2].n & 1);
  if (three)
    kernel = dec ? (reg ? load_vector_march_kernel<T, true, NS, T1C, true, CPT, true>
                        : load_vector_march_kernel<T, true, NS, T1C, true, CPT, false>)
                 : (reg ? load_vector_march_kernel<T, false, NS, T1C, true, CPT, true>
                        : load_vector_march_kernel<T, false, NS, T1C, true, CPT, false>);
  else
    kernel = dec ? (reg ? load_vector_march_kernel<T, true, NS, T1C, false, CPT, true>
                        : load_vector_march_kernel<T, true, NS, T1C, false, CPT, false>)
                 : (reg ? load_vector_march_kernel<T, false, NS, T1C, false, CPT, true>
                        : load_vector_march_kernel<T, false, NS, T1C, false, CPT, false>);
  allow_dynamic_smem(kernel, smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, g.threads, smem);
  per_sm = std::max(per_sm, 1);
  // Coarse planes per CTA: the shortest longest march over the waves (a CTA
  // marches 2 t0 + 3 fine planes).
  const uint64_t count = uint64_t(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  g.t0 = march_chunk(c0, g.nb2 * g.nb1, 152 * per_sm, 2);
  g.nb0 = (c0 + g.t0 - 1) / g.t0;
  const unsigned grid = static_cast<unsigned>(g.nb0 * g.nb1 * g.nb2);
  launch_pdl(kernel, dim3(grid), dim3(g.threads), smem, s, lv, fine, coarse, F, g, count, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load_vector_march(const LevelK<T>& lv_in, bool dec, const T* fine, T* coarse,
                                     T* F, unsigned int* status, cudaStream_t s) {
  using C = MarchCfg<T>;
  // A 2D level (1, n1, n2) marches along its rows: view it as (n1, 1, n2).
  LevelK<T> lv = lv_in;
  if (lv.ax[0].n == 1) std::swap(lv.ax[0], lv.ax[1]);
  return l2_resident(lv)
             ? launch_march_shape<T, C::NS_L2, C::T1_L2, C::CPT_L2>(lv, dec, fine, coarse, F, status, s)
             : launch_march_shape<T, C::NS, C::T1, C::CPT>(lv, dec, fine, coarse, F, status, s);
}

template bool load_vector_march_supported<float>(const LevelK<float>&);
template bool load_vector_march_supported<double>(const LevelK<double>&);
template cudaError_t launch_load_vector_march<float>(const LevelK<float>&, bool, const float*,
                                                     float*, float*, unsigned int*, cudaStream_t);
template cudaError_t launch_load_vector_march<double>(const LevelK<double>&, bool, const double*,
                                                      double*, double*, unsigned int*,
                                                      cudaStream_t);

}  // namespace mgb
