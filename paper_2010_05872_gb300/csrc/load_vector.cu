// Marching load-vector kernel for the level-l grids of 2D and 3D fields
// (Section 2 step 4 and Section 5.2: coefficient computation, mass multiply
// and restriction to the coarse load vector, fused).
//
// Work split: a CTA owns a block of T1 coarse rows along axis 1 and all the
// coarse columns of axis 2 (for 2D levels, a chunk of them), and marches along
// axis 0 through a chunk of coarse planes.  The fine rows a CTA needs from one
// plane are contiguous in memory, so each plane enters shared memory by one
// 1D TMA bulk copy (cp.async.bulk, completion on an mbarrier) of the
// enclosing 16-byte-aligned range; the offset of the first element is kept,
// bytes past the end of the array are never requested and the at most 3
// elements there come in by plain loads.  With FP32 the copy of the next pair
// of planes overlaps the arithmetic on the current pair.
//
// A thread owns the fine column pair (2P, 2P+1) and with it the coarse column
// P.  Lanes 2..30 of a warp own consecutive pairs; lanes 0, 1 and 31 repeat
// their neighbours' pairs, so the 5-tap axis-2 restriction takes its taps
// from warp shuffles only.  Each thread walks the rows of a plane with
// everything in registers: for a nodal fine plane p (its axis-0 index is a
// coarse node) the interpolant E(p) of p's fully nodal values over the
// (axis 1, axis 2) plane, w(p) = v(p) - E(p); for the coefficient plane q
// between nodal planes p' < q < p, w(q) = v(q) - (iwl0[q] E(p') + iwr0[q]
// E(p)), with E(p) parked in shared memory by the same thread that reads it
// back.  Recomposition reads w = u_mc directly (zero on the fully nodal
// nodes).  The axis-2 restriction of each row is accumulated into the axis-1
// restriction as the rows stream by, and the axis-0 restriction accumulates
// in registers for the three coarse planes a fine plane can touch; a coarse
// plane is stored to F once its last fine plane has passed.  The nodal values
// of every nodal plane are gathered into the coarse grid.  Waits on the
// mbarriers give up after 2 s, record the failure in `status` and end the CTA.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "kernels.cuh"
#include "tma.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

__device__ __forceinline__ int cpos(int k, int n) { return min(2 * k, n - 1); }
__device__ __forceinline__ bool is_coef(int j, int n) { return (j & 1) && (j != n - 1); }
__device__ __forceinline__ int nodal_k(int j, int n, int nc) { return j == n - 1 ? nc - 1 : (j >> 1); }

constexpr int kMaxThreads = 288;                  // 9 warps x 29 owned pairs >= 257 coarse columns
constexpr int kMaxRows = 15;                      // staged fine rows per plane (2 T1 + 3)
constexpr int kPairsPerWarp = 29;                 // lanes 2..30

template <typename T>
struct V2;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V2<double> {
  using type = double2;
};

struct MarchGeom {
  int S1max, S2max, T2max;  // staged rows, staged columns, coarse columns per CTA
  int BUF;                  // elements of one plane buffer (16-byte multiple)
  int tc2, t1, t0;          // coarse columns / rows / planes per CTA
  int nb2, nb1, nb0;        // CTAs along axes 2, 1, 0
  int threads;              // CTA size
};

template <typename T, bool DEC, int NS, int T1C>
__global__ void __launch_bounds__(kMaxThreads, 1)
load_vector_march_kernel(LevelK<T> lv, const T* __restrict__ fine, T* __restrict__ coarse,
                         T* __restrict__ F, MarchGeom g, uint64_t fine_count,
                         unsigned int* __restrict__ status) {
  using TT = typename V2<T>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NV = 2 * NS;  // plane buffers: NS stages of (coefficient, nodal) planes
  __shared__ __align__(8) uint64_t bars[NS];
  __shared__ int s_shift[NV];
  __shared__ T s_iwl1[kMaxRows], s_iwr1[kMaxRows];  // coefficient rows: interpolation weights
  __shared__ T s_W1[kMaxRows][T1C];                  // axis-1 restriction weight of row r for t1
  __shared__ int s_next[kMaxRows];                   // next nodal row after a nodal row

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n0 = lv.ax[0].n, n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c0 = lv.ax[0].nc, c1 = lv.ax[1].nc, c2 = lv.ax[2].nc;
  const int b2 = blockIdx.x % g.nb2;
  const int b1 = (blockIdx.x / g.nb2) % g.nb1;
  const int b0 = blockIdx.x / (g.nb2 * g.nb1);
  const int K2 = b2 * g.tc2, K1 = b1 * g.t1, K0 = b0 * g.t0;
  const int T2 = min(g.tc2, c2 - K2), T1 = min(g.t1, c1 - K1), T0 = min(g.t0, c0 - K0);
  const int j2lo = max(2 * K2 - 2, 0), j2hi = min(2 * (K2 + T2 - 1) + 2, n2 - 1);
  const int j1lo = max(2 * K1 - 2, 0), j1hi = min(2 * (K1 + T1 - 1) + 2, n1 - 1);
  const int jlo = max(2 * K0 - 2, 0), jhi = min(2 * (K0 + T0 - 1) + 2, n0 - 1);
  const int S2 = j2hi - j2lo + 1, S1 = j1hi - j1lo + 1;

  T* vbuf = reinterpret_cast<T*>(smem_raw);                                  // NV x BUF
  TT* ebuf = reinterpret_cast<TT*>(vbuf + static_cast<size_t>(NV) * g.BUF);  // 2 x S1max x threads

  // Row tables.
  for (int r = tid; r < S1; r += blockDim.x) {
    const int j1 = j1lo + r;
    const bool q = is_coef(j1, n1);
    s_iwl1[r] = q ? lv.ax[1].iwl[j1] : T(0);
    s_iwr1[r] = q ? lv.ax[1].iwr[j1] : T(0);
    s_next[r] = (j1 + 1 == n1 - 1) ? r + 1 : r + 2;
#pragma unroll
    for (int t1 = 0; t1 < T1C; ++t1) {
      T wv = T(0);
      if (t1 < T1) {
        const int off = j1 - cpos(K1 + t1, n1) + 2;
        if (off >= 0 && off <= 4) wv = lv.ax[1].rw[5 * (K1 + t1) + off];
      }
      s_W1[r][t1] = wv;
    }
  }
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }

  // Column pair of this thread.
  const int P = K2 + kPairsPerWarp * warp + lane - 2;
  const bool own = lane >= 2 && lane <= 30 && P >= K2 && P < K2 + T2;
  const int a = 2 * P, b = 2 * P + 1;
  const bool av = P >= 0 && a >= j2lo && a <= j2hi;
  const bool bv = av && b <= j2hi;
  const int al = av ? a - j2lo : 0;  // local column of a (0 for a lane without data)
  const bool bcoef = bv && is_coef(b, n2);  // otherwise b is absent or the last node of an even axis
  const T kca = bcoef ? lv.ax[2].iwl[b] : T(0);
  const T kcb = bcoef ? lv.ax[2].iwr[b] : T(0);
  // Axis-2 restriction weights over the sources (lane-2 b, lane-1 a, lane-1 b,
  // own a, own b, lane+1 a).
  T rw6[6];
#pragma unroll
  for (int o = 0; o < 6; ++o) rw6[o] = T(0);
  const bool special = own && cpos(P, n2) != a;  // last coarse node of an even axis
  if (own) {
    const T* rw = lv.ax[2].rw + 5 * P;
    if (!special) {
#pragma unroll
      for (int o = 0; o < 5; ++o) rw6[o + 1] = rw[o];
    } else {  // last coarse node of an even axis, at fine b of pair P - 1
      rw6[0] = rw[0];
      rw6[1] = rw[1];
      rw6[2] = rw[2];
    }
  }
  __syncthreads();

  // Plane loader: planes q (may be -1) and p into the buffers of `slot`.
  const uint64_t lim = (fine_count * sizeof(T)) & ~15ull;
  const int plane_elems = S1 * S2;
  auto issue = [&](int q, int p, int slot) {
    const int bq = 2 * slot;
    uint64_t ab[2], bb[2], sb[2], eb[2];
    unsigned bytes = 0;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int plane = w ? p : q;
      if (plane < 0) { ab[w] = bb[w] = sb[w] = eb[w] = 0; continue; }
      const uint64_t e0 = (static_cast<uint64_t>(plane) * n1 + j1lo) * n2 + j2lo;
      sb[w] = e0 * sizeof(T);
      eb[w] = sb[w] + static_cast<uint64_t>(plane_elems) * sizeof(T);
      ab[w] = sb[w] & ~15ull;
      bb[w] = (eb[w] + 15) & ~15ull;
      if (bb[w] > lim) bb[w] = lim;
      if (bb[w] > ab[w]) bytes += static_cast<unsigned>(bb[w] - ab[w]);
    }
    if (tid == 0) {
      mbar_arrive_expect_tx(&bars[slot], bytes);
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int plane = w ? p : q;
        if (plane < 0) continue;
        T* dst = vbuf + static_cast<size_t>(bq + w) * g.BUF;
        s_shift[bq + w] = static_cast<int>((sb[w] - ab[w]) / sizeof(T));
        if (bb[w] > ab[w])
          tma_bulk_g2s(dst, reinterpret_cast<const char*>(fine) + ab[w],
                       static_cast<unsigned>(bb[w] - ab[w]), &bars[slot]);
      }
    }
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int plane = w ? p : q;
      if (plane < 0) continue;
      // Elements after the last whole 16-byte chunk of the array.
      const uint64_t tail0 = bb[w] > sb[w] ? bb[w] : sb[w];
      T* dst = vbuf + static_cast<size_t>(bq + w) * g.BUF;
      const int shift = static_cast<int>((sb[w] - ab[w]) / sizeof(T));
      for (uint64_t x = tail0 + tid * sizeof(T); x < eb[w]; x += blockDim.x * sizeof(T)) {
        const uint64_t off = (x - sb[w]) / sizeof(T);
        dst[shift + static_cast<int>(off)] = fine[x / sizeof(T)];
      }
    }
  };

  // v at columns a, b and a + 2 of staged row r of a plane (two aligned
  // pair loads).
  auto load_row = [&](const T* pb, int r, T& va, T& vb, T& va2) {
    const int base = r * S2 + al;
    const int odd = (reinterpret_cast<uintptr_t>(pb + base) / sizeof(T)) & 1;
    const TT* p2 = reinterpret_cast<const TT*>(pb + base - odd);
    const TT x = p2[0], y = p2[1];
    va = odd ? x.y : x.x;
    vb = odd ? y.x : x.y;
    va2 = odd ? y.y : y.x;
  };

  T g2[T1C];
  T acc[3][T1C];
#pragma unroll
  for (int t = 0; t < T1C; ++t) {
    g2[t] = T(0);
    acc[0][t] = acc[1][t] = acc[2][t] = T(0);
  }
  int kdone = K0;

  // One row of w: axis-2 restriction (shuffles) into the axis-1 sums.
  auto row_out = [&](int r, T wa, T wb) {
    const T u2b = __shfl_up_sync(0xffffffffu, wb, 2);
    const T u1a = __shfl_up_sync(0xffffffffu, wa, 1);
    const T u1b = __shfl_up_sync(0xffffffffu, wb, 1);
    const T d1a = __shfl_down_sync(0xffffffffu, wa, 1);
    const T g1 = rw6[0] * u2b + rw6[1] * u1a + rw6[2] * u1b + rw6[3] * wa + rw6[4] * wb +
                 rw6[5] * d1a;
#pragma unroll
    for (int t = 0; t < T1C; ++t) g2[t] += s_W1[r][t] * g1;
  };

  // Axis-0 restriction of a finished fine plane j into the accumulators.
  auto plane_done = [&](int j) {
    T wk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int kk = kdone + k;
      wk[k] = T(0);
      if (kk < K0 + T0) {
        const int off = j - cpos(kk, n0) + 2;
        if (off >= 0 && off <= 4) wk[k] = __ldg(lv.ax[0].rw + 5 * kk + off);
      }
    }
#pragma unroll
    for (int t = 0; t < T1C; ++t) {
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k][t] += wk[k] * g2[t];
      g2[t] = T(0);
    }
  };

  auto store_done = [&](int upto_plane, bool all) {
    while (kdone < K0 + T0 && (all || cpos(kdone, n0) + 2 <= upto_plane)) {
#pragma unroll
      for (int t = 0; t < T1C; ++t) {
        if (own && t < T1)
          F[(static_cast<int64_t>(kdone) * c1 + (K1 + t)) * c2 + P] = acc[0][t];
        acc[0][t] = acc[1][t];
        acc[1][t] = acc[2][t];
        acc[2][t] = T(0);
      }
      ++kdone;
    }
  };

  // Steps of the march: (q, p) = (coefficient plane or -1, nodal plane).
  // NS stages cycle; while step s is computed, the copies of steps up to
  // s + NS - 1 are in flight.
  auto next_nodal = [&](int p) { return (p + 1 == n0 - 1) ? p + 1 : p + 2; };
  unsigned phases = 0u;   // bit i: parity to wait for on bars[i]
  unsigned pending = 1u;  // bit i: bars[i] has copies in flight
  int es = 0;             // E slot of the current nodal plane
  int iss_p = jlo;        // nodal plane of the last step issued
  issue(-1, jlo, 0);
  for (int i = 1; i < NS - 1 && iss_p < jhi; ++i) {
    const int np = next_nodal(iss_p);
    issue(np == iss_p + 2 ? iss_p + 1 : -1, np, i);
    pending |= 1u << i;
    iss_p = np;
  }
  int step_q = -1, step_p = jlo;
  for (int st = 0;; ++st) {
    const int slot = st % NS;
    const unsigned par = (phases >> slot) & 1u;
    const bool got = mbar_wait(&bars[slot], par, kWaitLimitNs);
    if (__syncthreads_or(!got)) {
      // A copy did not land in time: record it, give every stage still in
      // flight a second bounded wait so nothing lands after the CTA exits.
      if (tid == 0) *reinterpret_cast<volatile unsigned*>(status) = 1u;
      for (int i = 0; i < NS; ++i)
        if ((pending >> i) & 1u) mbar_wait(&bars[i], (phases >> i) & 1u, kWaitLimitNs);
      return;
    }
    phases ^= 1u << slot;
    pending &= ~(1u << slot);
    if (iss_p < jhi) {
      // The stage refilled here was last read in the previous step.
      const int np = next_nodal(iss_p);
      const int ns = (st + NS - 1) % NS;
      if (tid == 0) fence_proxy_async();
      issue(np == iss_p + 2 ? iss_p + 1 : -1, np, ns);
      pending |= 1u << ns;
      iss_p = np;
    }
    const int bq = 2 * slot, bp = bq + 1;
    const T* vp = vbuf + static_cast<size_t>(bp) * g.BUF + s_shift[bp];
    const T* vq = vbuf + static_cast<size_t>(bq) * g.BUF + s_shift[bq];
    TT* Ep = ebuf + static_cast<size_t>(es) * g.S1max * blockDim.x + tid;
    const TT* Eq = ebuf + static_cast<size_t>(es ^ 1) * g.S1max * blockDim.x + tid;

    // Nodal plane p: walk its nodal rows; a coefficient row sits between
    // two nodal rows exactly when they are 2 apart.
    {
      const int kc0 = nodal_k(step_p, n0, c0);
      const bool gplane = kc0 >= K0 && kc0 < K0 + T0;
      T epa = T(0), epb = T(0);
      int rprev = -1;
      for (int rn = 0; rn < S1; rn = s_next[rn]) {
        T va, vb, va2;
        load_row(vp, rn, va, vb, va2);
        const T era = va;
        const T erb = bcoef ? kca * va + kcb * va2 : (bv ? vb : T(0));
        if (rn - rprev == 2) {
          const int rc = rn - 1;
          T ca, cb, cx;
          load_row(vp, rc, ca, cb, cx);
          T wa, wb;
          if (DEC) {
            const T Ea = s_iwl1[rc] * epa + s_iwr1[rc] * era;
            const T Eb = s_iwl1[rc] * epb + s_iwr1[rc] * erb;
            Ep[rc * blockDim.x] = TT{Ea, Eb};
            wa = av ? ca - Ea : T(0);
            wb = bv ? cb - Eb : T(0);
          } else {
            wa = av ? ca : T(0);
            wb = bv ? cb : T(0);
          }
          row_out(rc, wa, wb);
        }
        T wa, wb;
        if (DEC) {
          Ep[rn * blockDim.x] = TT{era, erb};
          wa = T(0);
          wb = bv ? vb - erb : T(0);
        } else {
          wa = T(0);
          wb = bcoef ? vb : T(0);
        }
        row_out(rn, wa, wb);
        if (gplane) {
          const int k1 = nodal_k(j1lo + rn, n1, c1);
          if (k1 >= K1 && k1 < K1 + T1) {
            // The last node of an even axis is column b of the pair before.
            const T vb_up = __shfl_up_sync(0xffffffffu, vb, 1);
            if (own) coarse[(static_cast<int64_t>(kc0) * c1 + k1) * c2 + P] = special ? vb_up : va;
          }
        }
        epa = era;
        epb = erb;
        rprev = rn;
      }
      plane_done(step_p);
    }
    // Coefficient plane q between the previous nodal plane and p.
    if (step_q >= 0) {
      const T wl0 = __ldg(lv.ax[0].iwl + step_q), wr0 = __ldg(lv.ax[0].iwr + step_q);
      for (int r = 0; r < S1; ++r) {
        T va, vb, va2;
        load_row(vq, r, va, vb, va2);
        T wa, wb;
        if (DEC) {
          const TT e0 = Eq[r * blockDim.x], e1 = Ep[r * blockDim.x];
          wa = av ? va - (wl0 * e0.x + wr0 * e1.x) : T(0);
          wb = bv ? vb - (wl0 * e0.y + wr0 * e1.y) : T(0);
        } else {
          wa = av ? va : T(0);
          wb = bv ? vb : T(0);
        }
        row_out(r, wa, wb);
      }
      plane_done(step_q);
    }
    store_done(step_p, false);
    if (step_p >= jhi) break;
    __syncthreads();  // every read of this step's buffers is done
    const int np = next_nodal(step_p);
    step_q = (np == step_p + 2) ? step_p + 1 : -1;
    step_p = np;
    es ^= 1;
  }
  store_done(jhi, true);
}

template <typename T>
struct MarchCfg;
template <>
struct MarchCfg<float> {
  static constexpr int NS = 3, T1 = 4;
};
template <>
struct MarchCfg<double> {
  static constexpr int NS = 2, T1 = 2;
};

template <typename T>
bool plan_geometry(const LevelK<T>& lv, MarchGeom& g) {
  using C = MarchCfg<T>;
  const int n1 = lv.ax[1].n, n2 = lv.ax[2].n;
  const int c2 = lv.ax[2].nc, c1 = lv.ax[1].nc;
  g.t1 = (n1 == 1) ? 1 : C::T1;
  if (n1 == 1) {
    g.tc2 = (n2 <= 514) ? c2 : 256;
  } else {
    if (c2 > kPairsPerWarp * (kMaxThreads / 32)) return false;  // rows too wide for one CTA
    g.tc2 = c2;
  }
  g.T2max = g.tc2;
  g.S1max = (n1 == 1) ? 1 : std::min(2 * g.t1 + 3, n1);
  g.S2max = std::min(2 * g.tc2 + 3, n2);
  const int vec = 16 / static_cast<int>(sizeof(T));
  g.BUF = ((g.S1max * g.S2max + 3 * vec + 4 + vec - 1) / vec) * vec;
  g.nb2 = (c2 + g.tc2 - 1) / g.tc2;
  g.nb1 = (c1 + g.t1 - 1) / g.t1;
  g.threads = 32 * ((g.tc2 + kPairsPerWarp - 1) / kPairsPerWarp);
  return g.threads <= kMaxThreads && g.S1max <= kMaxRows;
}

template <typename T>
size_t smem_bytes(const MarchGeom& g, bool dec) {
  using C = MarchCfg<T>;
  return sizeof(T) * static_cast<size_t>(2 * C::NS) * g.BUF +
         (dec ? 2 * sizeof(T) * 2 * static_cast<size_t>(g.S1max) * g.threads : 0);
}

}  // namespace

template <typename T>
bool load_vector_march_supported(const LevelK<T>& lv_in) {
  // 2D and 3D levels large enough to fill the GPU (1D and tiny levels use
  // the generic tiled kernel).
  const int64_t nf = int64_t(lv_in.ax[0].n) * lv_in.ax[1].n * lv_in.ax[2].n;
  if (lv_in.ax[0].n == 1 && lv_in.ax[1].n == 1) return false;
  if (nf < (int64_t(1) << 17)) return false;
  LevelK<T> lv = lv_in;
  if (lv.ax[0].n == 1) std::swap(lv.ax[0], lv.ax[1]);
  MarchGeom g{};
  return plan_geometry(lv, g);
}

template <typename T>
cudaError_t launch_load_vector_march(const LevelK<T>& lv_in, bool dec, const T* fine, T* coarse,
                                     T* F, unsigned int* status, cudaStream_t s) {
  using C = MarchCfg<T>;
  // A 2D level (1, n1, n2) marches along its rows: view it as (n1, 1, n2).
  LevelK<T> lv = lv_in;
  if (lv.ax[0].n == 1) std::swap(lv.ax[0], lv.ax[1]);
  const int c0 = lv.ax[0].nc;
  MarchGeom g{};
  if (!plan_geometry(lv, g)) return cudaErrorInvalidConfiguration;
  const size_t smem = smem_bytes<T>(g, dec);
  using KernelFn = void (*)(LevelK<T>, const T*, T*, T*, MarchGeom, uint64_t, unsigned int*);
  KernelFn kernel = load_vector_march_kernel<T, false, C::NS, C::T1>;
  if (dec) kernel = load_vector_march_kernel<T, true, C::NS, C::T1>;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, g.threads, smem);
  per_sm = std::max(per_sm, 1);
  // Planes per CTA: aim at whole waves over the 152 SMs, with at least 8
  // coarse planes per CTA so the halo planes stay a small overhead.
  const int cols = g.nb2 * g.nb1;
  const int slots = 152 * per_sm;
  int best_t0 = c0, best_score = 1 << 30;
  for (int waves = 1; waves <= 16; ++waves) {
    const int chunks = std::max(1, (slots * waves + cols - 1) / cols);
    const int t0 = std::min(std::max(8, (c0 + chunks - 1) / chunks), c0);
    const int ctas = ((c0 + t0 - 1) / t0) * cols;
    const int used = (ctas + slots - 1) / slots;
    const int score = used * slots - ctas + 4 * waves * per_sm;  // idle slots; prefer fewer CTAs
    if (score < best_score) { best_score = score; best_t0 = t0; }
  }
  g.t0 = best_t0;
  g.nb0 = (c0 + g.t0 - 1) / g.t0;
  const uint64_t count = uint64_t(lv.ax[0].n) * lv.ax[1].n * lv.ax[2].n;
  const unsigned grid = static_cast<unsigned>(g.nb0 * g.nb1 * g.nb2);
  kernel<<<grid, g.threads, smem, s>>>(lv, fine, coarse, F, g, count, status);
  return cudaGetLastError();
}

template bool load_vector_march_supported<float>(const LevelK<float>&);
template bool load_vector_march_supported<double>(const LevelK<double>&);
template cudaError_t launch_load_vector_march<float>(const LevelK<float>&, bool, const float*,
                                                     float*, float*, unsigned int*, cudaStream_t);
template cudaError_t launch_load_vector_march<double>(const LevelK<double>&, bool, const double*,
                                                      double*, double*, unsigned int*,
                                                      cudaStream_t);

}  // namespace mgb
