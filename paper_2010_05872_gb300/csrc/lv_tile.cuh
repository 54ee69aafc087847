// The marching load-vector tile (what each CTA of the load-vector kernel
// computes), shared by the per-level kernel and the persistent batched
// kernel.  See load_vector.cu for the method.
#pragma once

#include <algorithm>
#include <cstdint>

#include "grid.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace mgb {

constexpr int kLvMaxThreads = 256;  // CTA size limit (a thread owns CPT coarse columns of a row)

struct MarchGeom {
  int t1, tc2, t0;     // coarse rows / columns / planes per CTA
  int nb2, nb1, nb0;   // CTAs along axes 2, 1, 0
  int pitch;           // elements between staged rows (n2 in 3D; the tile width in 2D)
  int BUF;             // elements of one plane buffer (16-byte multiple)
  int threads;         // CTA size
  int groups;          // row groups (see load_vector_march_tile)
  int gthreads;        // threads per row group
};

// Pipeline depth and coarse rows per CTA along axis 1, per element type.
template <typename T>
struct MarchCfg;
template <>
struct MarchCfg<float> {
  // Levels larger than L2: measured at 513^3 on GB300 with one wave of
  // 26-plane marches, (NS, T1) in {(2, 4), (2, 6), (2, 8), (3, 4), (3, 6),
  // (4, 4)}, two plane buffers of 2 T1 + 3 = 11 rows gave the shortest
  // finest-level launch (176 us; 182 with T1 = 6).  Levels that stay in L2
  // march a few planes per CTA, so their shape favours planes in flight
  // (NS_L2, T1_L2).  Two coarse columns per thread (CPT) beat one at 257^3
  // as well (41 against 43-64 us over six shapes).
  static constexpr int NS = 2, T1 = 4, CPT = 2;
  static constexpr int NS_L2 = 3, T1_L2 = 4, CPT_L2 = 2;
};
template <>
struct MarchCfg<double> {
  // FP64 is bound by the FMA rate, so fewer halo rows pay: over (NS, T1) in
  // {(2, 4), (3, 4), (2, 6), (3, 6), (2, 8)} at 513^3, T1 = 6 gave the
  // shortest finest launch (2.29 ms; 2.46 with T1 = 4), two buffers the
  // smaller footprint of the two equal ones.
  static constexpr int NS = 2, T1 = 6, CPT = 2;
  static constexpr int NS_L2 = 3, T1_L2 = 4, CPT_L2 = 2;
};

// One tile (CTA work unit) of the marching load vector; `tile` plays the
// role of the block index.  Any block of at least g.threads threads runs
// it.  GMAX > 1 allows row groups: g.groups groups of g.gthreads threads
// share the staged planes of a tile of g.groups x T1C coarse rows, group q
// taking coarse rows q T1C .. q T1C + T1C - 1 (staged rows 2 q T1C onwards),
// so a narrow grid keeps more warps of the block busy.  REG: all three axes
// have odd lengths, so coarse node k sits at 2k on each and the taps that
// are zero there are skipped (a column's 5-tap R window starts at its
// node - 2, its X taps sit at even offsets, an odd staged row feeds two
// coarse rows, an odd plane feeds two coarse planes through R0 alone).
// PERSIST: the CTA runs further tiles in the same launch, so the tile
// invalidates its barriers at the end (the next tile sets them up again) and
// reads its few plain-loaded elements through L2 (other CTAs of the launch
// may have written them).
template <typename T, bool DEC, int NS, int T1C, bool THREE, bool PERSIST = false, int CPT = 2,
          int GMAX = 1, bool REG = false>
__device__ __forceinline__ void load_vector_march_tile(const LevelK<T>& lv,
                                                       const T* __restrict__ fine,
                                                       T* __restrict__ coarse, T* __restrict__ F,
                                                       const MarchGeom& g, uint64_t fine_count,
                                                       unsigned int* __restrict__ status, int tile,
                                                       unsigned char*) {
  // The dynamic shared memory of the launch (every tile starts at its base).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int S1M = THREE ? 2 * T1C + 3 : 1;  // staged rows of a row group
  constexpr int S1T = THREE ? 2 * T1C * GMAX + 3 : 1;  // staged rows of the largest tile
  constexpr int TM = THREE ? T1C : 1;           // coarse rows per row group
  constexpr int VEC = 16 / sizeof(T);
  constexpr int PADL = 2 * VEC;                 // zeroed elements before a tile
  __shared__ __align__(8) uint64_t bars[NS];
  __shared__ int s_off[NS];   // buffer index of tile element (0, 0)
  __shared__ T s_w1[S1T][3];  // R1 weight of row s for coarse row base(s) + i
  __shared__ T s_y1[S1T][3];  // X1 weight of nodal row s for the same coarse rows
  __shared__ int s_rown[S1T]; // coarse row of a nodal row s, or -1
  __shared__ T s_lg[S1M];     // row sums of the left-over column (see `lrows`)
  __shared__ T s_lh[S1M];

  const int tid = threadIdx.x;
  const int grp = GMAX > 1 ? tid / g.gthreads : 0;          // row group
  const int ltid = GMAX > 1 ? tid - grp * g.gthreads : tid;  // thread within it
  const int roff = THREE ? grp * T1C : 0;                    // its first coarse row
  const int soff = 2 * roff;                                 // its first staged row
  // The copies are issued by lane 0 of the last warp, which owns the fewest
  // columns (often one), so the issue work stays off the busiest warps.
  const int producer = static_cast<int>(blockDim.x) - 32;
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int b2 = tile % g.nb2;
  const int b1 = (tile / g.nb2) % g.nb1;
  const int b0 = tile / (g.nb2 * g.nb1);
  const int K2 = b2 * g.tc2, K1 = b1 * g.t1, K0 = b0 * g.t0;
  const int T2 = min(g.tc2, c2 - K2), T1 = min(g.t1, c1 - K1), T0 = min(g.t0, c0 - K0);
  const int rbase = THREE ? 2 * K1 - 2 : 0;  // fine row of tile row 0
  const int cbase = 2 * K2 - 2;              // fine column of tile column 0
  const int jr_lo = max(rbase, 0), jr_hi = THREE ? min(2 * K1 + 2 * T1, n1 - 1) : 0;
  const int jc_lo = max(cbase, 0), jc_hi = min(2 * (K2 + T2 - 1) + 2, n2 - 1);
  const int jlo = max(2 * K0 - 2, 0), jhi = min(2 * (K0 + T0 - 1) + 2, n0 - 1);
  // Tile index of the first copied element and the copied length.
  const int t_first = (jr_lo - rbase) * g.pitch + (jc_lo - cbase);
  const int t_len = (jr_hi - jr_lo) * n2 + (jc_hi - jc_lo + 1);

  T* vbuf = reinterpret_cast<T*>(smem_raw);  // NS x BUF

  // Zero the buffers (virtual rows and pads must hold finite values) and
  // build the row tables.
  for (int i = tid; i < NS * g.BUF; i += blockDim.x) vbuf[i] = T(0);
  for (int s = tid; s < S1T; s += blockDim.x) {
    const int j1 = rbase + s;
    const bool valid = j1 >= 0 && j1 < n1;
    const bool nod = valid && !is_coef(j1, n1);
    const int kr = nod ? nodal_k(j1, n1, c1) : -1;
    s_rown[s] = kr;
    const int base = (s & 1) ? (s - 3) / 2 : s / 2 - 2;
    for (int i = 0; i < 3; ++i) {
      const int t = base + i, k = K1 + t;
      T w = T(0), y = T(0);
      if (valid && t >= 0 && t < T1) {
        const int off = j1 - cpos(k, n1) + 2;
        if (off >= 0 && off <= 4) w = lv.ax[1].rw[5 * k + off];
        const int d = kr - k + 1;
        if (nod && d >= 0 && d <= 2) y = (DEC ? lv.ax[1].xd : lv.ax[1].xr)[3 * k + d];
      }
      s_w1[s][i] = w;
      s_y1[s][i] = y;
    }
  }
  if (tid == producer) {
    for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }

  // Columns of this thread: coarse kc0 = K2 + CPT tid and the CPT - 1 after
  // it.  Fine taps are read from a window of W columns starting 2 left of
  // kc0's node; column c's 5 taps sit at window dcol[c] .. dcol[c] + 4, with
  // dcol[c] = cpos(kc0 + c) - cpos(kc0) (2c, or 2c - 1 when kc0 + c is the
  // last node of an even axis).
  //
  // An odd column count whose pairs exactly fill whole warps (every level
  // of a 2^k + 1 grid) leaves one column over.  A warp of its own would run
  // the whole row loop for that one lane, so instead the last warp takes it
  // with one lane per staged row (`lrows`, `lwarp`): lane s forms row s's
  // sums of the column and lanes t < T1 combine them into coarse row t.  It
  // keeps the column's weights in rwc[0] / xc[0] and its sums and
  // accumulators in G1[0][0], H1[0][0], acc[0][.][0].
  constexpr int W = 2 * CPT + 3;
  const bool lrows = CPT == 2 && GMAX == 1 && S1M <= 32 && (T2 & 1) && (((T2 - 1) / 2) & 31) == 0;
  const int TP = lrows ? T2 - 1 : T2;  // columns taken in pairs
  const int lane = tid & 31;
  const bool lwarp = lrows && (tid >> 5) == (TP / 2) >> 5;
  const int kL = K2 + T2 - 1;          // the left-over column
  // Coarse rows of the group, and whether it has any (one group: the tile's).
  const int T1g = GMAX > 1 && THREE ? max(0, min(T1C, T1 - roff)) : T1;
  const bool gact = GMAX > 1 ? grp < g.groups && T1g > 0 : true;
  const int kc0 = K2 + CPT * ltid;
  const int ccol = lwarp ? cpos(kL, n2) - cbase
                         : (CPT * ltid < TP ? cpos(kc0, n2) - cbase : 2);  // tile column of kc0's node
  bool actc[CPT];
  int dcol[CPT];
  T rwc[CPT][W], xc[CPT][W];
  {
    const T* X = DEC ? lv.ax[2].xd : lv.ax[2].xr;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int k = lwarp ? kL : kc0 + c;
      actc[c] = lwarp ? c == 0 : gact && CPT * ltid + c < TP;
      dcol[c] = actc[c] && !lwarp ? cpos(k, n2) - cpos(kc0, n2) : 2 * c;
#pragma unroll
      for (int oo = 0; oo < W; ++oo) rwc[c][oo] = xc[c][oo] = T(0);
      if (actc[c]) {
#pragma unroll
        for (int oo = 0; oo < W; ++oo) {
          const int o = oo - dcol[c];
          if (o >= 0 && o < 5) rwc[c][oo] = lv.ax[2].rw[5 * k + o];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int kk = k - 1 + d;
          if (kk >= 0 && kk < c2) {
            const int o = cpos(kk, n2) - cpos(lwarp ? kL : kc0, n2) + 2;
            const T xv = X[3 * k + d];
#pragma unroll
            for (int oo = 0; oo < W; ++oo)
              if (oo == o) xc[c][oo] = xv;
          }
        }
      }
    }
  }
  __syncthreads();

  // Plane loader, thread 0 only: fine plane j into buffer `slot`.
  const uint64_t lim = (fine_count * sizeof(T)) & ~15ull;
  auto issue = [&](int j, int slot) {
    const uint64_t e0 = (static_cast<uint64_t>(j) * n1 + jr_lo) * n2 + jc_lo;
    const uint64_t sb = e0 * sizeof(T), eb = sb + static_cast<uint64_t>(t_len) * sizeof(T);
    const uint64_t ab = sb & ~15ull;
    uint64_t bb = (eb + 15) & ~15ull;
    if (bb > lim) bb = lim;
    const int shift = static_cast<int>((sb - ab) / sizeof(T));
    const int dst_e = ((PADL + t_first - shift + VEC - 1) / VEC) * VEC;
    T* dst = vbuf + static_cast<size_t>(slot) * g.BUF + dst_e;
    s_off[slot] = dst_e + shift - t_first;
    const unsigned bytes = bb > ab ? static_cast<unsigned>(bb - ab) : 0u;
    mbar_arrive_expect_tx(&bars[slot], bytes);
    if (bytes) tma_bulk_g2s(dst, reinterpret_cast<const char*>(fine) + ab, bytes, &bars[slot]);
    for (uint64_t x = bb > sb ? bb : sb; x < eb; x += sizeof(T))
      dst[shift + static_cast<int>((x - sb) / sizeof(T))] =
          PERSIST ? __ldcg(fine + x / sizeof(T)) : fine[x / sizeof(T)];
  };

  T acc[CPT][3][TM];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int t = 0; t < TM; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[c][k][t] = T(0);
  int kdone = K0;
  auto store_done = [&](int upto_plane, bool all) {
    while (kdone < K0 + T0 && (all || cpos(kdone, n0) + 2 <= upto_plane)) {
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        T* dst = F + (static_cast<int64_t>(kdone) * c1 + (K1 + roff + t)) * c2 + kc0;
        if (lwarp && t == 0 && lane < T1)
          F[(static_cast<int64_t>(kdone) * c1 + (K1 + lane)) * c2 + kL] = acc[0][0][0];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          if (!lwarp && actc[c] && t < T1g) dst[c] = acc[c][0][t];
          acc[c][0][t] = acc[c][1][t];
          acc[c][1][t] = acc[c][2][t];
          acc[c][2][t] = T(0);
        }
      }
      ++kdone;
    }
  };

  unsigned phases = 0u;   // bit i: parity to wait for on bars[i]
  unsigned pending = 0u;  // bit i: bars[i] has a copy in flight
  if (tid == producer) fence_proxy_async();  // the zero fill precedes every bulk copy
  for (int i = 0; i < NS - 1 && jlo + i <= jhi; ++i) {
    if (tid == producer) issue(jlo + i, i);
    pending |= 1u << i;
  }
  for (int j = jlo; j <= jhi; ++j) {
    const int slot = (j - jlo) % NS;
    const bool got = mbar_wait(&bars[slot], (phases >> slot) & 1u, kWaitLimitNs);
    if (__syncthreads_or(!got)) {
      // A copy did not land in time: record it, give every stage still in
      // flight a second bounded wait so nothing lands after the CTA exits.
      if (tid == producer) *reinterpret_cast<volatile unsigned*>(status) = 1u;
      for (int i = 0; i < NS; ++i)
        if ((pending >> i) & 1u) mbar_wait(&bars[i], (phases >> i) & 1u, kWaitLimitNs);
      return;
    }
    phases ^= 1u << slot;
    pending &= ~(1u << slot);
    if (j + NS - 1 <= jhi) {
      // The buffer refilled here was last read for plane j - 1.
      const int ns = (j - jlo + NS - 1) % NS;
      if (tid == producer) {
        fence_proxy_async();
        issue(j + NS - 1, ns);
      }
      pending |= 1u << ns;
    }

    // Warps without a column of this tile skip the arithmetic.
    if ((gact && CPT * (ltid & ~31) < TP) || lwarp) {
    const bool pn = !is_coef(j, n0);  // nodal plane
    const int kj = pn ? nodal_k(j, n0, c0) : -1;
    const bool gplane = pn && kj >= K0 && kj < K0 + T0;
    const T* tile = vbuf + static_cast<size_t>(slot) * g.BUF + s_off[slot] + ccol;
    T G1[CPT][TM], H1[CPT][TM];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int t = 0; t < TM; ++t) G1[c][t] = H1[c][t] = T(0);
    if (lwarp) {
      if (lane < S1M) {
        const T* row = tile + lane * g.pitch;
        T fe[5];
#pragma unroll
        for (int o = 0; o < 5; ++o) fe[o] = row[o - 2];
        T gs = T(0), hs = T(0);
#pragma unroll
        for (int o = 0; o < 5; ++o) gs += rwc[0][o] * fe[o];
        const int kr = THREE ? s_rown[lane] : 0;
        if (pn && kr >= 0) {
#pragma unroll
          for (int o = 0; o < 5; ++o) hs += xc[0][o] * fe[o];
          if (gplane && kr >= K1 && kr < K1 + T1)
            coarse[(static_cast<int64_t>(kj) * c1 + kr) * c2 + kL] = fe[2];
        }
        s_lg[lane] = gs;
        s_lh[lane] = hs;
      }
      __syncwarp();
      if (!THREE) {
        G1[0][0] = s_lg[0];
        H1[0][0] = s_lh[0];
      } else if (lane < T1) {
        T gsum = T(0), hsum = T(0);
#pragma unroll
        for (int s = 0; s < S1M; ++s) {
          const int i = lane - ((s & 1) ? (s - 3) / 2 : s / 2 - 2);
          if (i >= 0 && i <= 2) {
            gsum += s_w1[s][i] * s_lg[s];
            hsum += s_y1[s][i] * s_lh[s];
          }
        }
        G1[0][0] = gsum;
        H1[0][0] = hsum;
      }
    } else {
#pragma unroll
    for (int s = 0; s < S1M; ++s) {
      const T* row = tile + (s + soff) * g.pitch;
      T fe[W];  // window: tile columns ccol - 2 .. ccol + W - 3 of row s
      if constexpr (sizeof(T) == 4) {
        // Aligned 8-byte loads cover the window (8-byte words per thread: no
        // bank conflicts); the pair parity is that of the row start, the
        // same for the whole warp.
        constexpr int NQ = (W + 1) / 2;
        const T* p0 = row - 2;
        const bool par = (reinterpret_cast<uintptr_t>(p0) >> 2) & 1u;
        const float2* q = reinterpret_cast<const float2*>(p0 - par);
        float2 v[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) v[i] = q[i];
#pragma unroll
        for (int o = 0; o < W; ++o) {
          const float lo = (o & 1) ? v[o / 2].y : v[o / 2].x;
          const float hi = (o & 1) ? v[o / 2 + 1].x : v[o / 2].y;
          fe[o] = par ? hi : lo;
        }
      } else {
#pragma unroll
        for (int o = 0; o < W; ++o) fe[o] = row[o - 2];
      }
      T gs[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        gs[c] = T(0);
#pragma unroll
        for (int o = REG ? 2 * c : (c ? 2 * c - 1 : 0); o < W && o <= 2 * c + 4; ++o)
          gs[c] += rwc[c][o] * fe[o];
      }
      const int base = (s & 1) ? (s - 3) / 2 : s / 2 - 2;
      const int kr = THREE ? s_rown[s + soff] : 0;
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        if (!THREE) {
          G1[c][0] = gs[c];
        } else {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const int t = base + i;
            if (REG && (s & 1) && i == 2) continue;  // a zero weight
            if (t >= 0 && t < TM) G1[c][t] += s_w1[s + soff][i] * gs[c];
          }
        }
      }
      if (pn && kr >= 0) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          T hs = T(0);
#pragma unroll
          for (int o = 2 * c; o < W && o <= 2 * c + 4; o += REG ? 2 : 1) hs += xc[c][o] * fe[o];
          if (!THREE) {
            H1[c][0] = hs;
          } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const int t = base + i;
              if (t >= 0 && t < TM) H1[c][t] += s_y1[s + soff][i] * hs;
            }
          }
        }
        if (gplane && kr >= K1 + roff && kr < K1 + roff + T1g) {
          T* dst = coarse + (static_cast<int64_t>(kj) * c1 + kr) * c2 + kc0;
#pragma unroll
          for (int c = 0; c < CPT; ++c)
            if (actc[c]) dst[c] = (c == 0 || dcol[c] == 2 * c) ? fe[2 + 2 * c] : fe[1 + 2 * c];
        }
      }
    }
    }
    // Axis 0: plane j feeds the coarse planes kdone .. kdone + 2.
    T wk[3], yk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int kk = kdone + k;
      wk[k] = yk[k] = T(0);
      if (kk < K0 + T0) {
        const int off = j - cpos(kk, n0) + 2;
        if (off >= 0 && off <= 4) wk[k] = __ldg(lv.ax[0].rw + 5 * kk + off);
        const int d = kj - kk + 1;
        if (pn && d >= 0 && d <= 2) yk[k] = __ldg((DEC ? lv.ax[0].xd : lv.ax[0].xr) + 3 * kk + d);
      }
    }
    if (REG && !pn) {
      // An odd plane of an odd axis 0 feeds coarse planes kdone and kdone + 1
      // through R0 alone (wk[2] and every yk are zero).
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int t = 0; t < TM; ++t)
#pragma unroll
          for (int k = 0; k < 2; ++k) acc[c][k][t] += wk[k] * G1[c][t];
    } else {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int t = 0; t < TM; ++t)
#pragma unroll
          for (int k = 0; k < 3; ++k) acc[c][k][t] += wk[k] * G1[c][t] - yk[k] * H1[c][t];
    }
    store_done(j, false);
    }
    __syncthreads();  // every read of this buffer is done
  }
  store_done(jhi, true);
  if (PERSIST && tid == producer)
    for (int i = 0; i < NS; ++i) mbar_inval(&bars[i]);
}

// Tile shape of a level for CPT coarse columns per thread, T1 coarse rows per
// row group, `groups` row groups and NS plane buffers (the per-level kernel's
// MarchCfg and one group by default; the batched kernel passes its own).
template <typename T>
inline bool plan_geometry(const LevelK<T>& lv, MarchGeom& g, int cpt = 2, int t1 = MarchCfg<T>::T1,
                          int ns = MarchCfg<T>::NS, int groups = 1) {
  const int n1 = lv.ax[1].n, n2 = lv.ax[2].n, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int vec = 16 / static_cast<int>(sizeof(T));
  if (n1 > 1) {
    if (c2 > cpt * kLvMaxThreads) return false;  // rows too wide for one CTA
    g.t1 = t1 * groups;
    g.tc2 = c2;
    g.pitch = n2;
    g.BUF = ((4 * vec + (2 * g.t1 + 3) * n2 + 4 + vec - 1) / vec) * vec;
  } else {
    groups = 1;
    g.t1 = 1;
    g.tc2 = c2 <= cpt * kLvMaxThreads ? c2 : cpt * kLvMaxThreads / 2;
    g.pitch = 2 * g.tc2 + 3;
    g.BUF = ((4 * vec + g.pitch + 4 + vec - 1) / vec) * vec;
  }
  g.nb2 = (c2 + g.tc2 - 1) / g.tc2;
  g.nb1 = (c1 + g.t1 - 1) / g.t1;
  g.gthreads = 32 * (((g.tc2 + cpt - 1) / cpt + 31) / 32);
  g.groups = groups;
  g.threads = g.gthreads * groups;
  return g.gthreads <= kLvMaxThreads && sizeof(T) * static_cast<size_t>(ns) * g.BUF <= 200 * 1024;
}


}  // namespace mgb
