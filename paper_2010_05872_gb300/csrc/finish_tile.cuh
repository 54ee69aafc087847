// The marching finish tile (what each CTA of the finish kernel computes),
// shared by the per-level kernel and the persistent batched kernel.  See
// finish.cu for the method.
#pragma once

#include <algorithm>
#include <cstdint>

#include "grid.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace mgb {

constexpr int kFMaxThreads = 576;

// Pipeline depth and coarse rows per CTA along axis 1, per element type:
// NS stages of (two fine planes, one coarse plane) with NS - 1 in flight.
template <typename T>
struct FinishCfg;
template <>
struct FinishCfg<float> {
  static constexpr int NS = 2, T1 = 4;
};
template <>
struct FinishCfg<double> {
  static constexpr int NS = 2, T1 = 4;
};

struct FinishGeom {
  int t1, tc2, t0;       // coarse rows per CTA, fine columns per chunk, plane pairs per CTA
  int nb0, nb1, nb2;     // CTAs along axes 0, 1, 2
  int FBUF, CBUF;        // elements of a fine-plane buffer and of a coarse-plane buffer
  int threads;
  int groups;            // row groups (see finish_march_tile)
  int gthreads;          // threads per row group
};

// Marching form: a CTA owns fine plane pairs [M0, M1) (planes 2m, 2m + 1) of
// up to 2 T1C fine rows and a chunk of fine columns, one thread per column.
// Stage m brings fine planes 2m, 2m + 1 and coarse plane m + 1 (the first
// stage also coarse plane M0) with 1D bulk copies of the contiguous row
// range; coarse planes sit in a ring of NS + 1 buffers.
//
// The interpolant is separable (Section 2, multilinear Pi): a thread first
// interpolates each staged coarse row along axis 2 at its column, then along
// axis 1 to every fine row, and keeps the result of coarse plane m (A) in
// registers, so fine plane 2m reads A and plane 2m + 1 combines A with the
// next coarse plane (B) along axis 0.  A nodal node takes its coarse value
// exactly: weights (1, 0) or (0, 1), never a rounded mix.
//
// One tile (CTA work unit); `tile` plays the role of the block index and
// `smem_raw` is the dynamic shared memory.  Any block of at least g.threads
// threads runs it; a tile returns with its barriers invalidated so that the
// next tile of a persistent CTA can set them up again.  GMAX > 1 allows row
// groups: g.groups groups of g.gthreads threads share the staged planes of a
// tile of g.groups x T1C coarse rows, group q writing fine rows 2 q T1C ..
// 2 q T1C + 2 T1C - 1 of it, so a narrow grid keeps more warps busy.
template <typename T, int NS, int T1C, bool PERSIST = false, int GMAX = 1>
__device__ __forceinline__ void finish_march_tile(const LevelK<T>& lv,
                                                  const T* __restrict__ nodal_src,
                                                  const T* __restrict__ interp_src, T sign,
                                                  T* __restrict__ fine, const FinishGeom& g,
                                                  unsigned int* __restrict__ status, int tile,
                                                  unsigned char*) {
  // The dynamic shared memory of the launch (every tile starts at its base).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NC = NS + 1;  // coarse ring
  constexpr int R1M = 2 * T1C, RCM = T1C + 1;
  __shared__ __align__(8) uint64_t bars[NS];
  __shared__ int s_fshift[2 * NS];  // fine buffers: stage x plane
  __shared__ int s_cshift[NC];      // coarse ring
  __shared__ int s_nshift[NC];      // ring of nodal-source planes (decomposition)

  const int tid = threadIdx.x;
  const int grp = GMAX > 1 ? tid / g.gthreads : 0;          // row group
  const int ltid = GMAX > 1 ? tid - grp * g.gthreads : tid;  // column within the chunk
  const int croff = grp * T1C, froff = 2 * croff;           // its first coarse / fine row
  // The copies are issued by lane 0 of the last warp, which owns the fewest
  // columns (often one), so the issue work stays off the busiest warps.
  const int producer = static_cast<int>(blockDim.x) - 32;
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int b2 = tile % g.nb2;
  const int b1 = (tile / g.nb2) % g.nb1;
  const int b0 = tile / (g.nb2 * g.nb1);
  const int npairs = (n0 + 1) / 2;
  const int K1 = b1 * g.t1, T1 = min(g.t1, c1 - K1);
  const int M0 = b0 * g.t0, M1 = min(M0 + g.t0, npairs);     // plane pairs [M0, M1)
  const int J2lo = b2 * g.tc2, J2hi = min(J2lo + g.tc2, n2);  // fine columns
  const int W2 = J2hi - J2lo;
  const int klo2 = J2lo / 2, khi2 = min(J2hi / 2, c2 - 1);
  const int kw = khi2 - klo2 + 1;
  const int r1lo = 2 * K1, r1hi = min(2 * (K1 + T1), n1);     // owned fine rows [r1lo, r1hi)
  const int R1 = r1hi - r1lo;
  const int k1lo = K1, k1hi = min(K1 + T1, c1 - 1);           // coarse rows needed
  const int R1c = k1hi - k1lo + 1;

  T* fbuf = reinterpret_cast<T*>(smem_raw);                // 2 NS x FBUF
  T* cbuf = fbuf + 2 * NS * static_cast<size_t>(g.FBUF);   // NC x CBUF
  T* nbuf = cbuf + NC * static_cast<size_t>(g.CBUF);       // NC x CBUF when sep
  // Decomposition takes nodal values from a second coarse array; in
  // recomposition they are the interpolant's own coarse values.
  const bool sep = nodal_src != interp_src;

  if (tid == producer) {
    for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const uint64_t flim = (static_cast<uint64_t>(n0) * n1 * n2 * sizeof(T)) & ~15ull;
  const uint64_t clim = (static_cast<uint64_t>(c0) * c1 * c2 * sizeof(T)) & ~15ull;
  // Copies are issued by thread 0 alone.  One region [e0, e0 + len) of
  // `src` into dst: the 16-byte-aligned superset by bulk copy, and the at
  // most 15 bytes past the last whole 16 bytes of the array by plain loads
  // (visible to the CTA after the barrier that ends the wait).  Returns the
  // bulk bytes.
  auto region = [&](const T* src, uint64_t lim, uint64_t e0, int len, T* dst, int* shift_slot,
                    uint64_t* bar, bool count_only) -> unsigned {
    const uint64_t sb = e0 * sizeof(T), eb = sb + static_cast<uint64_t>(len) * sizeof(T);
    const uint64_t ab = sb & ~15ull;
    uint64_t bb = (eb + 15) & ~15ull;
    if (bb > lim) bb = lim;
    const unsigned bytes = bb > ab ? static_cast<unsigned>(bb - ab) : 0u;
    if (count_only) return bytes;
    const int shift = static_cast<int>((sb - ab) / sizeof(T));
    *shift_slot = shift;
    if (bytes) tma_bulk_g2s(dst, reinterpret_cast<const char*>(src) + ab, bytes, bar);
    for (uint64_t x = bb > sb ? bb : sb; x < eb; x += sizeof(T))
      dst[shift + static_cast<int>((x - sb) / sizeof(T))] = PERSIST ? __ldcg(src + x / sizeof(T)) : src[x / sizeof(T)];
    return bytes;
  };
  // Stage for plane pair m: fine planes 2m, 2m + 1, coarse plane m + 1 and,
  // for the first pair, coarse plane m (thread 0 only).
  auto issue = [&](int m, int stage) {
    unsigned bytes = 0;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) mbar_arrive_expect_tx(&bars[stage], bytes);
      for (int w = 0; w < 2; ++w) {
        const int j0 = 2 * m + w;
        if (j0 >= n0) continue;
        const uint64_t e0 = (static_cast<uint64_t>(j0) * n1 + r1lo) * n2 + J2lo;
        const int len = (R1 - 1) * n2 + W2;
        bytes += region(fine, flim, e0, len, fbuf + static_cast<size_t>(2 * stage + w) * g.FBUF,
                        &s_fshift[2 * stage + w], &bars[stage], pass == 0);
      }
      for (int cm = (m == M0 ? m : m + 1); cm <= m + 1; ++cm) {
        if (cm >= c0) continue;
        const uint64_t e0 = (static_cast<uint64_t>(cm) * c1 + k1lo) * c2 + klo2;
        const int len = (R1c - 1) * c2 + kw;
        bytes += region(interp_src, clim, e0, len, cbuf + static_cast<size_t>(cm % NC) * g.CBUF,
                        &s_cshift[cm % NC], &bars[stage], pass == 0);
        if (sep)
          bytes += region(nodal_src, clim, e0, len, nbuf + static_cast<size_t>(cm % NC) * g.CBUF,
                          &s_nshift[cm % NC], &bars[stage], pass == 0);
      }
    }
  };

  // Column data of this thread (axis 2).
  const int j2 = J2lo + ltid;
  const bool colact = GMAX > 1 ? grp < g.groups && froff < R1 && ltid < W2 : tid < W2;
  const bool q2 = colact && is_coef(j2, n2);
  const int kn2 = colact ? nodal_k(j2, n2, c2) : 0;
  const int kl = (q2 ? (j2 >> 1) : kn2) - klo2, kr = q2 ? kl + 1 : kl;
  const T wl2 = q2 ? lv.ax[2].iwl[j2] : T(1), wr2 = q2 ? lv.ax[2].iwr[j2] : T(0);
  const int kcol = kn2 - klo2;  // staged coarse column of a nodal column
  // Row data (axis 1, the same for every thread).  Even rows are nodal with
  // coarse row r / 2; odd row r mixes coarse rows r / 2 and r / 2 + 1, except
  // a last fine row n1 - 1 that is nodal (even n1): weights (0, 1).
  // The weights sit in shared memory (read after the first wait's barrier).
  __shared__ T s_wl1[T1C * GMAX], s_wr1[T1C * GMAX];
  unsigned q1mask = 0u;  // bit r: fine row froff + r is a coefficient row
  if constexpr (GMAX == 1) {
#pragma unroll
    for (int i = 0; i < T1C; ++i) {
      const int j1 = r1lo + 2 * i + 1;
      const bool q = 2 * i + 1 < R1 && is_coef(j1, n1);
      if (tid == i) {
        s_wl1[i] = q ? lv.ax[1].iwl[j1] : T(0);
        s_wr1[i] = q ? lv.ax[1].iwr[j1] : T(1);
      }
      if (q) q1mask |= 1u << (2 * i + 1);
    }
  } else {
    for (int i = tid; i < T1C * GMAX; i += blockDim.x) {
      const int j1 = r1lo + 2 * i + 1;
      const bool q = 2 * i + 1 < R1 && is_coef(j1, n1);
      s_wl1[i] = q ? lv.ax[1].iwl[j1] : T(0);
      s_wr1[i] = q ? lv.ax[1].iwr[j1] : T(1);
    }
#pragma unroll
    for (int i = 0; i < T1C; ++i) {
      const int j1 = r1lo + froff + 2 * i + 1;
      const bool q = froff + 2 * i + 1 < R1 && is_coef(j1, n1);
      if (q) q1mask |= 1u << (2 * i + 1);
    }
  }
  // Interpolant of coarse plane `cm` at this column and every owned fine row.
  auto interp_plane = [&](int cm, T (&out)[R1M]) {
    const T* C = cbuf + static_cast<size_t>(cm % NC) * g.CBUF + s_cshift[cm % NC] + croff * c2;
    T i2[RCM];
#pragma unroll
    for (int i = 0; i < RCM; ++i)
      i2[i] = (croff + i < R1c) ? wl2 * C[i * c2 + kl] + wr2 * C[i * c2 + kr] : T(0);
#pragma unroll
    for (int i = 0; i < T1C; ++i) {
      out[2 * i] = i2[i];
      out[2 * i + 1] = s_wl1[croff + i] * i2[i] + s_wr1[croff + i] * i2[i + 1];
    }
  };

  unsigned phases = 0u;   // bit i: parity to wait for on bars[i]
  unsigned pending = 0u;  // bit i: bars[i] has copies in flight
  for (int i = 0; i < NS - 1 && M0 + i < M1; ++i) {
    if (tid == producer) issue(M0 + i, i);
    pending |= 1u << i;
  }
  T A[R1M], B[R1M];
  for (int m = M0; m < M1; ++m) {
    const int stage = (m - M0) % NS;
    const bool got = mbar_wait(&bars[stage], (phases >> stage) & 1u, kWaitLimitNs);
    if (__syncthreads_or(!got)) {
      // A copy did not land in time: record it, give every stage still in
      // flight a second bounded wait so nothing lands after the CTA exits.
      if (tid == producer) *reinterpret_cast<volatile unsigned*>(status) = 1u;
      for (int i = 0; i < NS; ++i)
        if ((pending >> i) & 1u) mbar_wait(&bars[i], (phases >> i) & 1u, kWaitLimitNs);
      return;
    }
    phases ^= 1u << stage;
    pending &= ~(1u << stage);
    if (m + NS - 1 < M1) {
      // The stage refilled here was last read in the previous pair.
      const int st = (m - M0 + NS - 1) % NS;
      if (tid == producer) {
        fence_proxy_async();
        issue(m + NS - 1, st);
      }
      pending |= 1u << st;
    }
    if (colact) {
      if (m == M0) interp_plane(m, A);
      const bool has_b = m + 1 < c0;
      if (has_b) interp_plane(m + 1, B);
      // Fine plane 2m: nodal along axis 0, coarse plane m.
      {
        const int j0 = 2 * m;
        const T* fb = fbuf + static_cast<size_t>(2 * stage) * g.FBUF + s_fshift[2 * stage] +
                      froff * n2 + ltid;
        T* dst = fine + (static_cast<int64_t>(j0) * n1 + r1lo + froff) * n2 + j2;
        const T* nsrc = nbuf + static_cast<size_t>(m % NC) * g.CBUF + s_nshift[m % NC] + kcol +
                        croff * c2;
#pragma unroll
        for (int r = 0; r < R1M; ++r) {
          if (froff + r < R1) {
            const bool nodal = !q2 && !((q1mask >> r) & 1u);
            // Fully nodal rows sit on coarse row r / 2, or (0, 1) row r / 2 + 1.
            const int kr1 = (r & 1) ? (r >> 1) + 1 : (r >> 1);
            const T v = A[r];
            dst[r * n2] = nodal ? (sep ? nsrc[kr1 * c2] : v) : fb[r * n2] + sign * v;
          }
        }
      }
      // Fine plane 2m + 1: coarse planes m and m + 1, or the nodal last
      // plane of an even axis (coarse plane m + 1 alone).
      const int j0 = 2 * m + 1;
      if (j0 < n0) {
        const bool q0 = is_coef(j0, n0);
        const T wl0 = q0 ? lv.ax[0].iwl[j0] : T(0), wr0 = q0 ? lv.ax[0].iwr[j0] : T(1);
        const T* fb = fbuf + static_cast<size_t>(2 * stage + 1) * g.FBUF + s_fshift[2 * stage + 1] +
                      froff * n2 + ltid;
        T* dst = fine + (static_cast<int64_t>(j0) * n1 + r1lo + froff) * n2 + j2;
        const int mn = (m + 1) % NC;
        const T* nsrc = nbuf + static_cast<size_t>(mn) * g.CBUF + s_nshift[mn] + kcol + croff * c2;
#pragma unroll
        for (int r = 0; r < R1M; ++r) {
          if (froff + r < R1) {
            const bool nodal = !q0 && !q2 && !((q1mask >> r) & 1u);
            const int kr1 = (r & 1) ? (r >> 1) + 1 : (r >> 1);
            const T v = wl0 * A[r] + wr0 * B[r];
            dst[r * n2] = nodal ? (sep ? nsrc[kr1 * c2] : v) : fb[r * n2] + sign * v;
          }
        }
      }
      if (has_b) {
#pragma unroll
        for (int r = 0; r < R1M; ++r) A[r] = B[r];
      }
    }
    __syncthreads();  // this stage's buffers may be refilled
  }
  if (PERSIST && tid == producer)
    for (int i = 0; i < NS; ++i) mbar_inval(&bars[i]);
}

template <typename T>
inline bool finish_geometry(const LevelK<T>& lv, FinishGeom& g, int groups = 1) {
  const int n1 = lv.ax[1].n, n2 = lv.ax[2].n, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  if (n1 == 1) groups = 1;
  g.t1 = (n1 == 1) ? 1 : FinishCfg<T>::T1 * groups;
  if (n1 == 1) g.tc2 = std::min(n2, kFMaxThreads - (kFMaxThreads % 2));
  else if (n2 <= kFMaxThreads) g.tc2 = n2;
  else return false;  // 3D rows wider than one CTA: not contiguous per plane
  if (g.tc2 < n2 && (g.tc2 & 1)) --g.tc2;
  g.gthreads = 32 * ((g.tc2 + 31) / 32);
  g.groups = groups;
  g.threads = g.gthreads * groups;
  const int vec = 16 / static_cast<int>(sizeof(T));
  const int R1 = (n1 == 1) ? 1 : 2 * g.t1;
  g.FBUF = (((R1 - 1) * n2 + g.tc2 + 2 * vec) / vec + 1) * vec;
  const int kwmax = std::min(g.tc2 / 2 + 1, c2);
  const int R1c = std::min(g.t1 + 1, c1);
  g.CBUF = (((R1c - 1) * c2 + kwmax + 2 * vec) / vec + 1) * vec;
  g.nb1 = (c1 + g.t1 - 1) / g.t1;
  g.nb2 = (n2 + g.tc2 - 1) / g.tc2;
  return g.gthreads <= kFMaxThreads;
}


}  // namespace mgb
