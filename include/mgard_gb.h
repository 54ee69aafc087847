/*
 * mgard_gb.h -- C ABI of the GB300 (sm_103a) MGARD+ hot path: multilevel
 * decomposition / recomposition of 1-3D tensor-product grids and level-wise
 * quantization of the multilevel coefficients (Liang et al., arXiv
 * 2010.05872).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays are C order (the last axis is contiguous), dims[0] the slowest.
 *    Every axis needs at least 3 nodes; 1 <= ndim <= 3; the last axis may
 *    have up to 2^30 nodes, every other axis up to 2^18.
 *  - `dims`, `coords`, `coords[i]` and every `*_out` pointer are HOST
 *    pointers.  `data`, `coeffs`, `labels` and `workspace` are DEVICE
 *    pointers owned by the caller; the library never frees them.
 *  - `coords` may be NULL, and so may any `coords[i]`: that axis is then
 *    uniform.  Results do not depend on the scale or origin of the
 *    coordinates.  Given coordinates must be finite and strictly increasing.
 *  - `dtype` is MGARD_F32 or MGARD_F64: the element type of `data`/`coeffs`
 *    and the arithmetic type of the transform (level tolerances, bin widths
 *    and quantization are always FP64).
 *  - `stop_level` is the stopping level l~ of Algorithm 1 (0 <= l~ <= L):
 *    levels L..l~+1 are decomposed and the nodes of N_{l~} keep Q_{l~}u.
 *    0 is the full depth; L leaves the data unchanged.
 *  - The grid hierarchy (Section 2): every axis is coarsened at every level by
 *    keeping its even nodes, plus its last node when its length is even
 *    (n -> n/2 + 1); L is the number of steps until the shortest axis has 3
 *    nodes.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it and the calls return without waiting, except
 *    mgard_quantize and mgard_value_range, which wait for their own flags,
 *    and mgard_quantize_status, which waits to read them.
 *  - Calls on different streams may run at the same time from different
 *    host threads (say one field's compression while another's is
 *    decompressed, so that the two directions of the host link overlap).
 *    A call that waits keeps its flag word, reduction buffers and pinned
 *    mirrors per (device, stream) and holds no lock that a call on another
 *    stream needs while it waits; only mgard_decompose_adaptive waits under
 *    a per-device lock.  That per-stream scratch (about 20 KB) is made by a
 *    stream's first such call, so make that call outside any stream capture.
 *    It is keyed by the handle: threads that all pass NULL or
 *    cudaStreamPerThread share one scratch and take turns on its waits.
 *    mgard_decompose_noalloc is the exception: its calls share one array
 *    per device and must not overlap (see there).
 *  - The first call for a given (device, dims, coords, dtype) builds a plan
 *    (host FP64 tables, uploaded once with cudaMalloc/cudaMemcpy) and caches
 *    it until mgard_release_plans().  Make that first call outside any CUDA
 *    stream capture.
 *  - Return value: MGARD_OK (0) or one of the negative MGARD_ERR_* codes;
 *    mgard_error_string() names it.  Argument errors are detected before
 *    any work is enqueued.
 */
#ifndef MGARD_GB_H
#define MGARD_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { MGARD_F32 = 0, MGARD_F64 = 1 };

enum {
  MGARD_OK = 0,
  MGARD_ERR_ARG = -1,       /* NULL or misaligned pointer, bad dtype/ndim, tau <= 0 */
  MGARD_ERR_SHAPE = -2,     /* ndim outside 1..3, or an axis outside 3..2^30 (the last)
                               or 3..2^18 (the others) */
  MGARD_ERR_COORDS = -3,    /* coordinates not finite or not strictly increasing */
  MGARD_ERR_LEVEL = -4,     /* stop_level outside [0, L] */
  MGARD_ERR_WORKSPACE = -5, /* workspace NULL, misaligned or smaller than required */
  MGARD_ERR_OVERFLOW = -6,  /* a label would reach 2^62 in magnitude */
  MGARD_ERR_NONFINITE = -7, /* NaN or Inf in the input of quantize / value_range */
  MGARD_ERR_CUDA = -8,      /* a CUDA runtime call or kernel launch failed */
  MGARD_ERR_TIMEOUT = -9    /* a bounded device-side wait gave up */
};

/* Number of decomposition levels L of the hierarchy of `dims`. */
int mgard_num_levels(int ndim, const int64_t* dims, int* L_out);

/* Device workspace (bytes) that mgard_decompose / mgard_recompose need for
 * `dims` and `dtype`: the compact level-l grids and load vectors of every
 * coarser level (about 2/7 of the field for 3D).  The workspace must be
 * 256-byte aligned; its contents on entry do not matter. */
int mgard_workspace_size(int ndim, const int64_t* dims, int dtype, size_t* bytes);

/* Level tolerances tau_l, l = 0..L (host array of L+1 doubles; entries below
 * stop_level repeat tau_{l~}).  Eq. (LinfTau) of Section 4.1 with the
 * stopping level of Algorithm 1:
 *   tau_{l~} = (1 - k) tau_linf / ((1 - k^(L+1-l~)) C_Linf),
 *   tau_l = k tau_{l-1},  k = sqrt(2^ndim),
 * and C_Linf = 1 + max over decomposed levels of an upper bound of the
 * coefficient-to-correction max norm, computed from the coordinates (the
 * paper does not print the constant; the bound keeps the guarantee
 * |u - u~|_inf <= tau_linf of Eq. (LInfNormEstimator)).  tau_linf is
 * absolute and must be > 0. */
int mgard_level_tolerances(int ndim, const int64_t* dims, const double* const* coords,
                           int stop_level, double tau_linf, double* tau_out);

/* Multilevel decomposition, in place (Section 2, decomposition steps 1-6).
 * On return `data` holds u_mc indexed by the finest grid: at a node of
 * N*_l (l > l~) the coefficient (I - Pi_{l-1}) Q_l u, at a node of N_{l~}
 * the value of Q_{l~} u.  Per level: coefficient computation, load vector
 * (mass multiply + restriction, Lemma 1 generalised to any coordinates),
 * batched tridiagonal mass-matrix solves along every axis (Section 5.3-5.4),
 * correction application.  `workspace` needs mgard_workspace_size() bytes;
 * `ws_bytes` is its size. */
int mgard_decompose(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                    int stop_level, void* data, void* workspace, size_t ws_bytes,
                    void* stream);

/* The other bin-width rules of Section 4.1.  mgard_level_tolerances_mode
 * writes L + 1 level tolerances (entries below stop_level repeat
 * tau_{l~}) for mode 0: the geometric rule of mgard_level_tolerances (Eq.
 * LinfTau, tau an L-inf bound); 1: the L-inf-optimal widths, tau_l =
 * tau / C_Linf * #N*_l / #N_L (#N*_l the nodes new at level l, the whole
 * coarse block at the stopping level), the same L-inf guarantee; 2: tau an
 * L2 bound on the reconstruction error, tau_l = tau / (C_L2 h_l^d
 * #N_L)^(1/2) with C_L2 = 1 and h_l^d the product over the axes of the
 * largest integral of a level-l hat function (the reconstruction's error
 * components are L2-orthogonal across levels, so the bound holds with
 * that constant).  Host only.  mgard_quantize_levels and
 * mgard_dequantize_levels are mgard_quantize / mgard_dequantize with the
 * level tolerances given (tau_levels, host, L + 1 values, those from
 * stop_level on positive and finite, else MGARD_ERR_ARG). */
int mgard_level_tolerances_mode(int ndim, const int64_t* dims, const double* const* coords,
                                int stop_level, double tau, int mode, double* tau_out);
int mgard_quantize_levels(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                          int stop_level, const double* tau_levels, const void* coeffs,
                          int64_t* labels, void* stream);
int mgard_dequantize_levels(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                            int stop_level, const double* tau_levels, const int64_t* labels,
                            void* coeffs, void* stream);

/* Adaptive decomposition, in place (Section 4.2; the stopping-level search
 * of Algorithm 1):
 * for l = L, L-1, .., 1 the level-l grid is sampled (the cells of the
 * level-(l-1) grid with every index a multiple of 4, i.e. one 3^3 block in
 * four per dimension) and, over the coefficient nodes of the sampled blocks,
 * E_Lorenzo = sum |Lorenzo prediction - u| + 1.22 tau_0 (Eq. lorenzo) and
 * E_interp = sum |multilinear interpolation - u| + p tau_0 (Eq. interp;
 * p = 0.369 / 0.259 / 0.182 at edge / plane / cube nodes) are summed in
 * FP64 (the per-node residuals in the grid's precision), with tau_0 the
 * tolerance of level l were it the stopping level
 * (tau_linf absolute, > 0) and Lorenzo neighbours outside the grid
 * taken as 0.  If E_Lorenzo < E_interp the decomposition stops at l~ = l;
 * otherwise level l is decomposed and the loop goes on; l~ = 0 when no level
 * stops it.  On return *stop_out = l~ and `data` equals mgard_decompose with
 * stop_level = l~ (up to FP rounding order); recompose and quantize it with
 * that stop level.  sums_out (host, may be NULL) receives 2 (L + 1) doubles:
 * (E_Lorenzo, E_interp) of level l at [2l], [2l + 1], NaN for levels not
 * sampled.  3D grids only (the paper's penalty factors are for 3D):
 * MGARD_ERR_SHAPE otherwise.  Synchronizes `stream` once per sampled level.
 * Workspace and other errors as mgard_decompose. */
int mgard_decompose_adaptive(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                             double tau_linf, void* data, void* workspace, size_t ws_bytes,
                             int* stop_out, double* sums_out, void* stream);

/* The level-`level` grid of the hierarchy of `dims` (0 <= level <= L): its
 * shape (ndim values into shape_out) and, when coords_out is not NULL, the
 * coordinates of its nodes, axis after axis (sum of the shape entries
 * doubles; uniform axes give the finest node indices).  Host only.
 * MGARD_ERR_LEVEL for a level outside [0, L]. */
int mgard_level_grid(int ndim, const int64_t* dims, const double* const* coords, int level,
                     int64_t* shape_out, double* coords_out);

/* Progressive recomposition (Section 1, data refactoring): from `data`, the
 * decomposition of a field with `stop_level` (finest layout, device,
 * read-only), write Q_k u, the field's projection onto the level-k grid
 * (k = level, stop_level <= k <= L), to `out` (device, the compact level-k
 * grid of mgard_level_grid's shape, C order).  Only the components of
 * levels stop_level .. k are read and recomposed, so the cost is that of the
 * level-k grid.  The workspace needs mgard_workspace_size of the level-k
 * shape (at most that of the field); `out` must not overlap `data`.
 * MGARD_ERR_LEVEL for k outside [stop_level, L]; other errors as
 * mgard_recompose. */
int mgard_recompose_partial(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                            int stop_level, int level, const void* data, void* out, void* workspace,
                            size_t ws_bytes, void* stream);

/* Area of the iso-surface data = iso of a 3D grid function (Section 6.2.2's
 * analysis on reduced representations), with the grid's coordinates (NULL:
 * node indices): every cell is split into the 6 tetrahedra around its main
 * diagonal and the function taken linear on each (marching tetrahedra; a
 * vertex counts as above when its value exceeds iso), planar surfaces are
 * measured exactly.  Geometry in the data's precision, sum in FP64, fixed
 * summation order.  Waits for `stream`; *area_out receives the area.
 * MGARD_ERR_SHAPE unless ndim = 3; MGARD_ERR_ARG for a non-finite iso. */
int mgard_iso_area(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                   const void* data, double iso, double* area_out, void* stream);

/* Multilevel recomposition, in place: the exact inverse of mgard_decompose
 * with the same dims, coords, dtype and stop_level (Section 2, recomposition
 * steps 1-5).  Same workspace rule. */
int mgard_recompose(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                    int stop_level, void* data, void* workspace, size_t ws_bytes,
                    void* stream);

/* Level-wise quantization (Section 4.1; Algorithm 1's quantization).  For
 * every node x of the finest grid, with l the least level such that x is in
 * N_l, raised to stop_level: labels[x] = round(coeffs[x] / (2 tau_l)) with
 * ties away from zero, in FP64 (IEEE division).  `coeffs` (dtype) and
 * `labels` (int64, same element count) are device arrays.  If
 * `tau_levels_out` is not NULL it receives tau_0..tau_L (host, L+1
 * doubles).  Waits for the stream and returns MGARD_ERR_NONFINITE /
 * MGARD_ERR_OVERFLOW if any coefficient was not finite or any label would
 * reach 2^62 in magnitude (the labels are then incomplete). */
int mgard_quantize(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                   int stop_level, double tau_linf, const void* coeffs, int64_t* labels,
                   double* tau_levels_out, void* stream);

/* mgard_quantize without its wait (Section 4.1, the same labels): the call
 * enqueues the quantization on `stream` and returns; whether a coefficient
 * was not finite or a label would reach 2^62 is gathered in a word of the
 * device's context over every such call on the device (all streams) until
 * mgard_quantize_status reads it.  For a pipeline that checks once per
 * batch of work instead of once per call. */
int mgard_quantize_async(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, double tau_linf, const void* coeffs, int64_t* labels,
                         double* tau_levels_out, void* stream);

/* Waits for `stream`, then reports and clears what the asynchronous
 * quantizations since the last call gathered: MGARD_ERR_NONFINITE,
 * MGARD_ERR_OVERFLOW, MGARD_ERR_ARG (a level tolerance formed on the device
 * was not positive and finite), or MGARD_ERR_TIMEOUT if a bounded device
 * wait gave up meanwhile; MGARD_OK otherwise.  The stream must be one that follows all of
 * those quantizations (the flags are read on it). */
int mgard_quantize_status(void* stream);

/* Bin centres: coeffs[x] = labels[x] * (2 tau_l), computed in FP64 and
 * rounded to dtype (Section 4.1).  Arguments as for mgard_quantize. */
int mgard_dequantize(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                     int stop_level, double tau_linf, const int64_t* labels, void* coeffs,
                     void* stream);

/* min and max of a device array of `count` elements of dtype, as doubles in
 * minmax_out[0], minmax_out[1] (host).  The value range max - min scales a
 * relative error bound into the absolute tau of the other calls.  Waits for
 * the stream; MGARD_ERR_NONFINITE if an element is NaN or Inf. */
int mgard_value_range(int64_t count, int dtype, const void* data, double* minmax_out,
                      void* stream);

/* A relative error bound carried through on the device (Section 4.1, Eq.
 * LinfTau with tau = rel_bound x (max - min)), so a pipeline of range,
 * decomposition, quantization, dequantization and recomposition needs no
 * wait.  mgard_value_range_async writes min and max of the array to
 * `range` (device, two doubles, 8-byte aligned) and gathers a NaN / Inf
 * element as mgard_quantize_async does (MGARD_ERR_NONFINITE from
 * mgard_quantize_status).  mgard_quantize_rel_async and
 * mgard_dequantize_rel are mgard_quantize_async and mgard_dequantize with
 * tau read from `range` on the device: every CTA forms the level
 * tolerances itself with the host's operations in the host's order, so the
 * labels and values equal those of the host calls given tau = rel_bound x
 * (max - min) computed in FP64.  A tau that is not positive and finite
 * (e.g. a constant array) is reported by mgard_quantize_status as
 * MGARD_ERR_ARG.  The range's partial sums use a buffer of the stream's
 * own, so range calls on different streams may overlap. */
int mgard_value_range_async(int64_t count, int dtype, const void* data, double* range,
                            void* stream);
int mgard_quantize_rel_async(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                             int stop_level, double rel_bound, const double* range,
                             const void* coeffs, int64_t* labels, void* stream);
int mgard_dequantize_rel(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, double rel_bound, const double* range,
                         const int64_t* labels, void* coeffs, void* stream);

/* Host-buffer forms of decompose / recompose: copy `host_in` (pinned or
 * pageable host memory, the field's element count of dtype) to the device
 * buffer `dev_data`, transform it there in place, and copy the result to
 * `host_out` (may equal host_in).  The stream is synchronised before
 * returning.  Other arguments as for mgard_decompose. */
int mgard_decompose_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, const void* host_in, void* host_out, void* dev_data,
                         void* workspace, size_t ws_bytes, void* stream);
int mgard_recompose_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, const void* host_in, void* host_out, void* dev_data,
                         void* workspace, size_t ws_bytes, void* stream);

/* Host-buffer compression round trip (Algorithm 1 with a fixed stopping
 * level and the uniform quantizer of Section 4.1 also on Q_{l~}u in place of
 * the external compressor; the lossless back end stays outside):
 * mgard_compress_host copies `host_field` to `dev_data`, takes the value
 * range on the device, sets tau_linf = rel_bound * (max - min) (a constant
 * field uses rel_bound * |value|, or rel_bound if it is 0), decomposes,
 * quantizes into `dev_labels` (int64, element count of the field) and copies
 * the labels to `host_labels`; *tau_out receives tau_linf.
 * mgard_decompress_host copies `host_labels` to `dev_labels`, dequantizes
 * into `dev_data`, recomposes and copies the field to `host_field`.  Both
 * synchronise the stream before returning; the error codes are those of the
 * calls they chain. */
int mgard_compress_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                        int stop_level, double rel_bound, const void* host_field,
                        int64_t* host_labels, double* tau_out, void* dev_data, int64_t* dev_labels,
                        void* workspace, size_t ws_bytes, void* stream);
int mgard_decompress_host(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                          int stop_level, double tau_linf, const int64_t* host_labels,
                          void* host_field, void* dev_data, int64_t* dev_labels, void* workspace,
                          size_t ws_bytes, void* stream);

/* The coarse part's Lorenzo coder (the coarse part's coder in Algorithm 1;
 * Section 4.2 Eq. lorenzo) as an exact transform of the labels: mgard_lorenzo_encode
 * replaces the labels q of the coarse block N_{stop_level} (in the finest
 * layout, device, in place) by q - pred(q), pred the signed sum of the
 * lower neighbours in the coarse grid (0 outside it), in 64-bit
 * wrap-around arithmetic; mgard_lorenzo_decode is its inverse (cumulative
 * sums along every axis).  The coarse labels are the linear quantization of
 * Q_{l~}u, so the prediction uses the reconstructed values; a smooth coarse
 * part leaves small residuals for the lossless stage.  Other labels are
 * untouched.  Asynchronous on `stream`. */
int mgard_lorenzo_encode(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, int64_t* labels, void* stream);
int mgard_lorenzo_decode(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                         int stop_level, int64_t* labels, void* stream);

/* The labels' lossless stage (Section 4.1: labels go to a lossless coder;
 * the last step of Algorithm 1).  This library's coder packs the labels in chunks
 * of 1024: zigzag codes (0, -1, 1, -2, .. -> 0, 1, 2, 3, ..) in the chunk's
 * width w (bit length of its largest code), least significant bit first.
 * Stream (little-endian): uint64 count | one width byte per chunk | zero
 * padding to 8 bytes | per chunk ceil(n_c w / 64) 64-bit words.
 * mgard_pack_bound: the largest stream of `count` labels (host only).
 * mgard_pack_labels: encode `count` device labels into the device buffer
 * `out` (8-byte aligned, capacity >= mgard_pack_bound, else
 * MGARD_ERR_WORKSPACE); *bytes_out receives the stream size; waits for
 * `stream`.  mgard_unpack_labels: decode a device stream of `bytes` bytes
 * into `count` device labels; the header is read back and checked (count,
 * widths <= 64, size), MGARD_ERR_ARG if it does not match; waits for the
 * header only. */
int mgard_pack_bound(int64_t count, size_t* bytes);
int mgard_pack_labels(int64_t count, const int64_t* labels, void* out, size_t capacity,
                      size_t* bytes_out, void* stream);
int mgard_unpack_labels(const void* in, size_t bytes, int64_t count, int64_t* labels, void* stream);

/* mgard_compress_host / mgard_decompress_host with the packed label stream
 * crossing between host and device instead of int64 labels: compress
 * quantizes into dev_labels, replaces the coarse block's labels by their
 * Lorenzo residuals (mgard_lorenzo_encode), packs into dev_stream (8-byte
 * aligned, at least mgard_pack_bound(count) bytes) and copies the stream
 * (its size in *stream_bytes, at most host_capacity, else
 * MGARD_ERR_WORKSPACE) to host_stream; decompress checks the host stream's
 * header, copies it to dev_stream, unpacks into dev_labels, undoes the
 * Lorenzo residuals, dequantizes, recomposes and copies the field to
 * host_field.  Both synchronise the stream before returning. */
int mgard_compress_host_packed(int ndim, const int64_t* dims, const double* const* coords,
                               int dtype, int stop_level, double rel_bound, const void* host_field,
                               void* host_stream, size_t host_capacity, size_t* stream_bytes,
                               double* tau_out, void* dev_data, int64_t* dev_labels,
                               void* dev_stream, size_t dev_capacity, void* workspace,
                               size_t ws_bytes, void* stream);
int mgard_decompress_host_packed(int ndim, const int64_t* dims, const double* const* coords,
                                 int dtype, int stop_level, double tau_linf,
                                 const void* host_stream, size_t stream_bytes, void* host_field,
                                 void* dev_data, int64_t* dev_labels, void* dev_stream,
                                 size_t dev_capacity, void* workspace, size_t ws_bytes,
                                 void* stream);

/* Four-dimensional grids (the tensor-product hierarchy of Section 2 with
 * d = 4; QMCPACK's data in Section 6 has this shape class).  dims[4] gives
 * the axes, slowest first (C order), each in 3..2^20 nodes; coords is NULL
 * (uniform) or four arrays of strictly increasing coordinates.  The
 * hierarchy halves every axis together, n -> n / 2 + 1, while the smallest
 * axis has more than 3 nodes; mgard_num_levels_4d gives its L.
 * mgard_decompose_4d / mgard_recompose_4d overwrite `data` (device, dtype
 * elements) in place with u_mc (the same layout as the 1-3D calls: the
 * coefficients at their nodes, Q_{l~}u at the nodes of N_{l~}) and back; the
 * workspace (device, 256-byte aligned, mgard_workspace_size_4d bytes) holds
 * the compact grids of the levels below L, two arrays of #N_L elements and
 * one of #N_{L-1}.  Per level they run one pass that forms the coefficients
 * in place (the interpolant from up to 16 coarse nodes) or adds the
 * interpolant back, four restriction passes and four Thomas passes (the
 * operators applied axis by axis), not the fused 1-3D kernels.  mgard_level_tolerances_4d writes the
 * L+1 tolerances of Eq. (LinfTau) with kappa = sqrt(2^4) = 4 and the C_Linf
 * bound of the four axes (entries below stop_level repeat tau_{l~}).
 * mgard_quantize_4d / mgard_dequantize_4d are the level-wise quantizer and
 * its inverse on a 4D u_mc (labels int64, device; bin width 2 tau_l, labels
 * and values exactly those of the FP64 definition, as for 1-3D); quantize
 * waits for the stream and returns MGARD_ERR_NONFINITE / MGARD_ERR_OVERFLOW
 * as mgard_quantize does; dequantize is enqueued on the stream.  Errors: MGARD_ERR_SHAPE for
 * an axis outside 3..2^20 or 2^31 nodes or more (32-bit index arithmetic), MGARD_ERR_COORDS,
 * MGARD_ERR_LEVEL, MGARD_ERR_WORKSPACE, MGARD_ERR_ARG as for the 1-3D calls. */
int mgard_num_levels_4d(const int64_t* dims, int* L_out);
int mgard_workspace_size_4d(const int64_t* dims, int dtype, size_t* bytes);
int mgard_level_tolerances_4d(const int64_t* dims, const double* const* coords, int stop_level,
                              double tau_linf, double* tau_out);
int mgard_decompose_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                       void* data, void* workspace, size_t ws_bytes, void* stream);
int mgard_recompose_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                       void* data, void* workspace, size_t ws_bytes, void* stream);
int mgard_quantize_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                      double tau_linf, const void* coeffs, int64_t* labels, double* tau_levels_out,
                      void* stream);
int mgard_dequantize_4d(const int64_t* dims, const double* const* coords, int dtype, int stop_level,
                        double tau_linf, const int64_t* labels, void* coeffs, void* stream);

/* Canonical Huffman coding of the labels (a reading of the lossless encoder
 * that Algorithm 1 ends with, which the paper does not name), the labels'
 * order-0 entropy and the cost model of Section 4.1.
 * Stream (little-endian): uint64 N | uint32 K = 32817 | uint32 longest code
 * length (<= 31) | K bytes of code lengths per symbol (0 = unused) | zero
 * padding to 8 bytes | per chunk of 1024 labels a uint32 payload word count
 * | zero padding to 8 bytes | the chunks' 64-bit payload words.  Symbol of a label: its zigzag
 * code z (0, -1, 1, -2, .. -> 0, 1, 2, 3, ..) when z < 2^15, else 32768 +
 * b - 16 for z of bit length b, followed by the b - 1 low bits of z.  Code
 * lengths: Huffman's construction with leaves ordered by (count, symbol),
 * merged nodes queued in creation order, a leaf taken on a tie; a code
 * longer than 31 bits halves every used count (at least 1) and rebuilds.
 * Canonical codes, written most significant bit first from bit 0 of the
 * chunk's first word, extra bits after the code, least significant first.
 * mgard_huffman_bound: an upper bound on the stream size of `count` labels.
 * mgard_huffman_encode: labels (device int64, `count`) -> stream at `out`
 * (device, 8-byte aligned, `capacity` bytes, else MGARD_ERR_WORKSPACE);
 * *bytes_out receives its size; waits for the stream (the histogram is
 * read on the host to build the code).
 * mgard_huffman_decode: the inverse; MGARD_ERR_ARG if the stream does not
 * match `count` and `bytes` or is not a valid code (checked on the host
 * from its header and in the kernel while reading); waits for the stream.
 * mgard_label_entropy: -sum p log2 p over the distinct label values, in
 * bits per label (0 for no labels); waits for the stream.
 * mgard_huffman_lengths: host only, the code lengths of `nsym` (<= 65536)
 * symbol counts by the rule above.
 * mgard_cost_model: host only, sum_l #N*_l log2(range / q_l) with
 * q_l = 2 tau_levels[l] for l = stop_level .. L (N_{l~} counted whole at the
 * stopping level), `range` the range of the multilevel coefficients. */
int mgard_huffman_bound(int64_t count, size_t* bytes);
int mgard_huffman_encode(int64_t count, const int64_t* labels, void* out, size_t capacity,
                         size_t* bytes_out, void* stream);
int mgard_huffman_decode(const void* in, size_t bytes, int64_t count, int64_t* labels, void* stream);
int mgard_label_entropy(int64_t count, const int64_t* labels, double* bits_per_label, void* stream);
int mgard_huffman_lengths(int nsym, const uint64_t* counts, uint8_t* lengths);
int mgard_cost_model(int ndim, const int64_t* dims, int stop_level, const double* tau_levels,
                     double range, double* bits);

/* Free every cached plan (device tables included) of the current device.
 * Call it only while no other host thread is inside a call of this library
 * on the device: a call in progress may hold one of the freed plans. */
int mgard_release_plans(void);

/* Batched form: many 3D FP32 fields of uneven shape on uniform grids,
 * decomposed (or recomposed) at full depth in ONE persistent kernel launch
 * replayed as a CUDA graph (Section 2's level loop for every field; the
 * per-field kernels' tiles scheduled across the fields).  The paper runs
 * fields one at a time; batching them is an interface choice of this
 * library.
 *  - dims3: host array of 3 * nfields sizes (n0, n1, n2 per field, C order,
 *    n2 <= 288).  data: host array of nfields device pointers (FP32 fields,
 *    transformed in place; same layout and result as mgard_decompose /
 *    mgard_recompose with stop_level 0 and NULL coords).  workspace: device,
 *    256-byte aligned, at least mgard_batch_workspace_size bytes (one
 *    per-field workspace after another).
 *  - The first call for a (shapes, data pointers, workspace) set builds the
 *    schedule and the graph (device memory is allocated then, and plans are
 *    cached as for the per-field calls); later calls only launch the graph on
 *    `stream`.  Make the first call outside any stream capture.
 *  - mgard_batch_autotune times candidate tile shapes (coarse planes per
 *    load-vector tile, plane pairs per finish tile, lines per contiguous
 *    solve tile
 *    and 32-line groups per segmented solve tile) with decompose + recompose
 *    on the fields (restored afterwards from a device copy), keeps the
 *    fastest for these shapes and writes it to choice_out[4] (may be NULL).
 *    It synchronizes `stream`.
 *  - A device-side wait that gives up (2 s) is reported by the next
 *    mgard_quantize / mgard_value_range as MGARD_ERR_TIMEOUT.
 *  - mgard_batch_release frees every batched schedule and graph.
 *  - mgard_batch_stats waits for the device and copies, for the batched
 *    launch issued last, per tile kind (load vector dec, load vector rec,
 *    contiguous solve with bulk copy, contiguous solve, segmented solve,
 *    finish) three counters: tiles run, SM cycles spent before a tile
 *    started (waiting for its stage's dependency, taking the descriptor) and
 *    SM cycles running tiles; `n` must be at least 18. */
int mgard_batch_workspace_size(int nfields, const int64_t* dims3, size_t* bytes);
int mgard_batch_decompose(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                          size_t ws_bytes, void* stream);
int mgard_batch_recompose(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                          size_t ws_bytes, void* stream);
int mgard_batch_autotune(int nfields, const int64_t* dims3, void* const* data, void* workspace,
                         size_t ws_bytes, void* stream, int* choice_out);
int mgard_batch_release(void);
int mgard_batch_stats(uint64_t* out, int n);

/* Test support for the bounded device-side waits (no counterpart in the
 * paper).  Launches the batched kernel with a one-item schedule whose
 * dependency can never be met (the item waits for a tile of its own stage)
 * and a wait limit of `limit_ns` (0 < limit_ns <= 1e9) instead of 2 s: the
 * kernel's wait gives up, sets the per-device status word and ends without
 * running a tile, so the next mgard_quantize / mgard_value_range on this
 * device returns MGARD_ERR_TIMEOUT (and clears the word).  Allocates and
 * frees a few hundred bytes of device memory; synchronizes `stream`.
 * Returns MGARD_ERR_ARG for a limit out of range, MGARD_ERR_CUDA on a CUDA
 * error, else MGARD_OK. */
int mgard_batch_wait_selftest(int64_t limit_ns, void* stream);

/* Serving: a request loop with continuous batching on the current device
 * (an interface of this library; the paper compresses one field per call).
 * A request is a whole compression (host field -> value range, decomposition
 * at stop_level, level-wise quantization at rel_bound x range -> host
 * labels; Section 2, Section 4.1) or a whole decompression (host labels and
 * the absolute bound tau used at compression -> dequantization,
 * recomposition -> host field), on uniform grids (NULL coords).
 *  - mgard_server_create starts a scheduler thread owning `slots` streams.
 *    Requests are admitted in arrival order as soon as a stream is free and
 *    their device memory (field, labels, workspace; drawn from the device's
 *    stream-ordered memory pool, kept for reuse up to the budget) fits in
 *    `hbm_budget` bytes beside the admitted ones; admitted requests overlap
 *    on the device.  Plans stay resident in the plan cache.
 *  - mgard_server_submit queues a request (the host buffers must stay valid
 *    until its completion is polled; pinned buffers let copies overlap) and
 *    returns its id; a request that alone exceeds the budget is rejected with
 *    MGARD_ERR_WORKSPACE.
 *  - mgard_server_poll returns up to `max` completed requests in completion
 *    order: id, status (MGARD_OK or an error code), latency in seconds from
 *    submission to the scheduler seeing the last device work end, and the
 *    absolute bound tau used (compression) or given (decompression).  Any
 *    output array may be NULL.
 *  - mgard_server_drain waits (up to timeout_s seconds) until no request is
 *    queued or running; mgard_server_counters writes {queued, running, bytes
 *    in use, peak running, peak bytes in use}; mgard_server_destroy drains and
 *    stops the thread. */
enum { MGARD_OP_COMPRESS = 1, MGARD_OP_DECOMPRESS = 2 };
typedef struct {
  int op;             /* MGARD_OP_COMPRESS or MGARD_OP_DECOMPRESS */
  int ndim;
  int64_t dims[3];    /* the first ndim entries are used */
  int dtype;          /* MGARD_F32 or MGARD_F64 */
  int stop_level;
  double rel_bound;   /* compression: bound relative to max - min of the field */
  double tau;         /* decompression: absolute bound used at compression */
  const void* host_in;  /* compression: field; decompression: int64 labels */
  void* host_out;       /* compression: int64 labels; decompression: field */
} mgard_request;
int mgard_server_create(size_t hbm_budget, int slots, void** server);
int mgard_server_submit(void* server, const mgard_request* req, int64_t* id_out);
int mgard_server_poll(void* server, int max, int64_t* ids, int* status, double* latency_s,
                      double* tau, int* count_out);
int mgard_server_drain(void* server, double timeout_s);
int mgard_server_counters(void* server, int64_t* out5);
int mgard_server_destroy(void* server);

/* Allocation-free decomposition.  The paper has no counterpart: this is an
 * interface for callers that must not allocate device memory while they
 * compress -- e.g. an in-situ simulation that has reserved nearly all of HBM
 * for its own state, where a cudaMalloc could fail and may wait for work in
 * flight on other streams.  The result equals mgard_decompose's (same
 * kernels, same rounding).
 *  - No workspace argument: the level workspace and the plan tables live in
 *    one static device array of 32 MiB per device.  Shapes whose tables plus
 *    workspace (about 2/7 of the field in 3D) do not fit are rejected with
 *    MGARD_ERR_WORKSPACE before any work is enqueued (e.g. up to ~110 MB of
 *    FP32 field).
 *  - The calls allocate nothing: no cudaMalloc, cudaFree, pinned host
 *    memory or allocating library.  The array and this library's kernels
 *    are part of the library's device code, which the CUDA runtime loads
 *    when it is first needed (lazily, the default since CUDA 12.2): the
 *    first call on a device, which also looks up the array's device address
 *    (cudaGetSymbolAddress, checked), is where the 32 MiB and the code are
 *    reserved (at library load under CUDA_MODULE_LOADING=EAGER).  Make one
 *    small warm-up call at start-up, before the memory is committed
 *    elsewhere and outside any stream capture; later calls reserve nothing.
 *    A call with a new (dims, coords, dtype) builds host tables and copies
 *    them into the array with cudaMemcpyAsync from pageable memory.
 *  - Only the array's first word (the wait-timeout status) must start at
 *    zero; each call clears it on `stream` before its kernels run.
 *  - Calls share the one array per device: two calls whose work overlaps on
 *    the device (other streams, other host threads, or a new shape while an
 *    earlier call's kernels still run) race on it.  Order them on one stream
 *    or synchronize between them.
 *  - `timed_out` may be NULL: the call returns once the work is enqueued and
 *    a bounded device-side wait that gave up is not reported (the next call
 *    clears the status word; the field may then be partly transformed).
 *    Otherwise the call waits for `stream`, sets *timed_out to 1 if such a
 *    wait gave up (then returns MGARD_ERR_TIMEOUT), else 0.
 * Arguments, layout and the other errors are those of mgard_decompose. */
int mgard_decompose_noalloc(int ndim, const int64_t* dims, const double* const* coords, int dtype,
                            int stop_level, void* data, int* timed_out, void* stream);

/* Kernel timing trace (host-side bookkeeping, no effect on results).
 * mgard_trace_enable(1) clears earlier records and starts bracketing every
 * kernel launch of this library with CUDA events on the launch stream;
 * mgard_trace_enable(0) stops.  mgard_trace_read waits for the recorded
 * events and returns one row per (kernel kind, fine level; -1 for the
 * level-free kernels) with the launch count, the summed device time in ms and
 * the summed algorithmic bytes (each input read once, each output written
 * once); up to max_rows rows are written, *rows_out receives the number of
 * rows available; a row's launch count is the number of traced calls of
 * that kind (a call can launch more than one kernel).
 * mgard_trace_kernel_name names a kind.  mgard_trace_kernel_launches returns
 * the number of kernels this library launched while tracing was on since the
 * last mgard_trace_enable(1).
 * mgard_trace_select(kind, level, any_level) limits the bracketing to the
 * launches of one kernel kind (and, unless any_level is nonzero, of one
 * level), so that the events of the other launches do not perturb a timed
 * region; kind < 0 brackets every launch again (the default).  Launches of
 * every kind are still counted.  Returns MGARD_ERR_ARG for an unknown kind. */
int mgard_trace_enable(int on);
int mgard_trace_select(int kind, int level, int any_level);
int64_t mgard_trace_kernel_launches(void);
int mgard_trace_read(int max_rows, int* kind, int* level, int64_t* launches, double* total_ms,
                     double* bytes, int* rows_out);
const char* mgard_trace_kernel_name(int kind);

/* Arithmetic roof of an element type on the current device (measurement
 * support; no counterpart in the paper): times a kernel of independent
 * dependent-FMA chains (8 per thread, 8 CTAs of 256 threads per SM) with
 * CUDA events on `stream` and writes the best of three runs in flop/s (an
 * FMA counts 2) to *flops_per_s.  The FP64 path of this library is bound by
 * this rate rather than by HBM bandwidth on parts with few FP64 units.
 * Allocates a small device buffer; synchronizes `stream`.  MGARD_ERR_ARG
 * for a bad dtype or a NULL output, MGARD_ERR_CUDA on a CUDA error. */
int mgard_trace_fma_rate(int dtype, double* flops_per_s, void* stream);

/* Static description of an error code. */
const char* mgard_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* MGARD_GB_H */
