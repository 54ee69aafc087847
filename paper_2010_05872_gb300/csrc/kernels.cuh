// Device-side views of the plan tables and the launchers of the transform
// kernels (`level` is the fine level of the transition, used to tag the
// kernel timing trace).  Every grid is handled as 3D (n0, n1, n2) with n2 contiguous;
// padded leading axes have n = nc = 1 and identity tables.
#pragma once

#include <algorithm>
#include <climits>

#include <cstdint>
#include <cuda_runtime.h>

namespace mgb {

template <typename T>
struct AxisK {
  const T* iwl;  // [n]  left interpolation weight of coefficient nodes
  const T* iwr;  // [n]  right interpolation weight of coefficient nodes
  const T* rw;   // [nc*5] load-vector weights on fine offsets -2..+2
  const T* xd;   // [nc*3] R P on coarse nodes k-1, k, k+1 (decomposition)
  const T* xr;   // [nc*3] R S on coarse nodes k-1, k, k+1 (recomposition)
  const T* ta;   // [nc] Thomas: sub-diagonal
  const T* tm;   // [nc] Thomas: reciprocal pivot
  const T* tc;   // [nc] Thomas: eliminated super-diagonal
  const T* sb;   // [nc] segmented forward recurrence: y_k = tm_k f_k + sb_k y_{k-1}
  const T* sg;   // [nc] product of sb over the segment up to k
  const T* sy;   // [nc] segmented backward recurrence: x_k = y_k + sy_k x_{k+1}
  const T* sh;   // [nc] product of sy from k to the segment end
  int n;
  int nc;
  int seg_len;   // rows per segment (the last may be shorter)
};

template <typename T>
struct LevelK {
  AxisK<T> ax[3];
};

// How the last tridiagonal solve of a level writes its result x.
enum ApplyMode : int {
  kApplyNone = 0,       // F <- x
  kApplyDecompose = 1,  // B <- B + x and F <- old B  (B held u on N_{l-1})
  kApplyRecompose = 2,  // B <- B - x                 (B held Q_{l-1}u)
};

// Load vector of one level, read-only on `fine` (level-l grid, n0 x n1 x n2):
//   dec = true : w = fine - Pi(fine at nodal nodes) on coefficient nodes
//   dec = false: w = fine on coefficient nodes (fine holds u_mc)
//   w = 0 on nodal nodes; F = (R0 x R1 x R2) w on the coarse grid; and the
//   nodal values of `fine` are gathered into `coarse` (nc0 x nc1 x nc2).
// `status` receives 1 if a bounded device-side wait gave up.
template <typename T>
cudaError_t launch_load_vector(const LevelK<T>& lv, bool dec, const T* fine, T* coarse, T* F,
                               int level, unsigned int* status, cudaStream_t s);

// The marching TMA-staged form of the load vector (load_vector.cu), used for
// 2D and 3D levels that fill the GPU.
template <typename T>
bool load_vector_march_supported(const LevelK<T>& lv);
template <typename T>
cudaError_t launch_load_vector_march(const LevelK<T>& lv, bool dec, const T* fine, T* coarse,
                                     T* F, unsigned int* status, cudaStream_t s);

// Batched Thomas solves of M_c along every axis (2, then 1, then 0), the
// last one applying its result to B as `mode` says.
template <typename T>
cudaError_t launch_solves(const LevelK<T>& lv, T* F, T* B, ApplyMode mode, int level,
                          unsigned int* status, cudaStream_t s);

// In-place finishing pass over the level-l grid `fine`:
//   nodal nodes       : fine <- nodal_src[k]
//   coefficient nodes : fine <- fine + sign * Pi(interp_src)
// Decomposition: nodal_src = B_{l-1} (final coarse values), interp_src =
// F_{l-1} (saved u on N_{l-1}), sign = -1.  Recomposition: nodal_src =
// interp_src = B_{l-1} (the interpolant's coarse values), sign = +1.
template <typename T>
cudaError_t launch_finish(const LevelK<T>& lv, const T* nodal_src, const T* interp_src, T sign,
                          T* fine, int level, unsigned int* status, cudaStream_t s);

// The coarsest levels stop + 1 .. stop + nlev of a transform in one CTA
// (small.cu): `data` is the level-(stop + nlev) grid, decomposed (dec) or
// recomposed in place; lv[i] is the transition of level stop + 1 + i.
constexpr int kSmallMaxLevels = 10;
constexpr int64_t kSmallMaxNodes = 40000;  // nodes of the highest small level
constexpr size_t kSmallMaxSmem = 220 * 1024;  // its shared memory (every level and table)
template <typename T>
size_t small_levels_smem(const LevelK<T>* lv, int nlev);
template <typename T>
cudaError_t launch_small_levels(const LevelK<T>* lv, int nlev, bool dec, T* data, int level,
                                cudaStream_t s);

// Quantization / dequantization / value range (quantize.cu).  The field is
// viewed as `rows` rows (j0, j1) of n2 contiguous elements; lev01 holds the
// level of each row, lev2 that of each column.
struct LevelTable {
  double q[48];   // bin width 2 tau_l per level
  float rq[48];   // fl32(1 / q_l), or NaN where that is not a normal float
  float qf[48];   // fl32(q_l)
  float dqf[48];  // fl32(q_l - fl32(q_l))
};
// Level tolerances formed on the device (Eq. LinfTau) from a range that
// stays there: tau = rel (max - min), t0 = (1 - kappa) tau / ((1 - kpow) C)
// and t_l = kappa t_{l-1} above the stopping level, the host's operations
// in the host's order (IEEE FP64, no contraction), so the table equals the
// one the host builds from the same tau.
struct RelTol {
  const double* range;   // device [min, max]; NULL: the kernels use the host table
  double rel, C, kappa, kpow;
  int L, stop;
  unsigned int* flags;   // receives 4 if tau is not positive and finite
};
template <typename T>
cudaError_t launch_quantize(const T* coeffs, int64_t* labels, const uint8_t* lev01,
                            const uint8_t* lev2, int64_t rows, int64_t n2, int stop_level,
                            const LevelTable& tab, unsigned int* flags, cudaStream_t s,
                            const RelTol* rt = nullptr);
template <typename T>
cudaError_t launch_dequantize(const int64_t* labels, T* coeffs, const uint8_t* lev01,
                              const uint8_t* lev2, int64_t rows, int64_t n2, int stop_level,
                              const LevelTable& tab, cudaStream_t s, const RelTol* rt = nullptr);
template <typename T>
cudaError_t launch_minmax(const T* data, int64_t count, double* partial, unsigned int* flags,
                          double* result, cudaStream_t s);
constexpr int kMinmaxBlocks = 1216;  // 8 x 152 SMs

// Sampled sums (E_Lorenzo, E_interp) of the adaptive stopping level over the
// level-l grid `v` (the n of lv's axes; 3D), with the level tolerance tau0,
// written to result[0..1] (device); `partial` holds 2 x kMinmaxBlocks
// doubles of scratch.
// The labels' packed stream (pack.cu): chunks of kPackChunk labels.
constexpr int kPackChunk = 1024;
// Bytes before the payload: the count, one width byte per chunk, padding.
size_t pack_header_bytes(int64_t n);
// Encode n device labels into `out` (8-byte aligned, at least
// pack_header_bytes(n) + 8 n bytes); `words` (ceil(n / kPackChunk)
// uint64) is scratch; *total_words (device) receives the payload words.
cudaError_t launch_pack_labels(const int64_t* labels, int64_t n, uint8_t* out, uint64_t* words,
                               uint64_t* total_words, cudaStream_t s);
// Decode a validated stream of n labels.
cudaError_t launch_unpack_labels(const uint8_t* in, int64_t n, uint64_t* words, uint64_t* total_words,
                                 int64_t* labels, cudaStream_t s);

// Lorenzo residuals (encode) of the labels of a level's nodes (positions
// pos[a], block shape shape3) in an array of the finest layout (dims3), in
// place, or their inverse (decode); `tmp` holds the block's element count
// of uint64 scratch.
cudaError_t launch_lorenzo(bool encode, int64_t* labels, const int64_t* dims3,
                           const int32_t* const* pos, const int64_t* shape3, uint64_t* tmp,
                           cudaStream_t s);

// Copy the nodes of a level out of an array in the finest layout (dims3)
// into a compact grid of shape3, with per-axis node positions pos[a].
template <typename T>
cudaError_t launch_gather_level(const T* src, const int64_t* dims3, const int32_t* const* pos,
                                const int64_t* shape3, T* dst, cudaStream_t s);
// Iso-surface area of the 3D grid function v (dims3, axis coordinates
// x[a] on the device) at `iso`, into result[0] (device); `partial` holds
// kMinmaxBlocks doubles of scratch.
template <typename T>
cudaError_t launch_iso_area(const T* v, const int64_t* dims3, const double* const* x, double iso,
                            double* partial, double* result, cudaStream_t s);

template <typename T>
cudaError_t launch_prediction_errors(const LevelK<T>& lv, const T* v, double tau0, double* partial,
                                     double* result, int level, cudaStream_t s);

// Planes (or plane pairs) per CTA of a marching kernel over `units` planes
// with `cols` CTAs per plane chunk and `slots` resident CTAs on the GPU: the
// chunk that minimises the longest march, waves x (chunk + halo).  A chunk
// re-reads `halo` planes and each wave runs as long as its CTAs' marches, so
// this trades halo work against wave count; on the 513^3 finest level it
// takes one wave of 26-plane chunks (load vector 197 -> 182 us against
// chunks of 9 in three waves).
inline int march_chunk(int units, int cols, int slots, int halo) {
  int best = units;
  int64_t best_t = INT64_MAX;
  for (int t0 = 1; t0 <= units; ++t0) {
    const int64_t ctas = int64_t((units + t0 - 1) / t0) * cols;
    const int64_t t = ((ctas + slots - 1) / slots) * (t0 + halo);
    if (t < best_t) { best_t = t; best = t0; }
  }
  return best;
}
constexpr size_t kL2ResidentBytes = size_t(96) << 20;  // levels below this take the L2 tile shape

}  // namespace mgb
