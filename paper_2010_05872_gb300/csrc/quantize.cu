// sm_103a kernels of level-wise quantization (Section 4.1; the quantization
// step of Algorithm 1), dequantization and the value range that scales a
// relative bound.
//
// Both quantizer directions are defined in FP64 (label = round(x / q) with
// ties away from zero; value = label * q rounded to the element type).  FP64
// arithmetic is slow on this part, so each direction has an exact fast path
// that reproduces the FP64 result bit for bit and falls back to FP64 only
// where it cannot prove agreement:
//  * quantize: the quotient is estimated in FP32 (x * fl32(1/q)); its error
//    is below |y| 2^-22.3, so whenever the estimate is farther than
//    |y| 2^-21 + 2^-126 from the nearest half-integer, the FP64 quotient
//    rounds to the same label.  Otherwise the IEEE FP64 division decides.
//  * dequantize (FP32): for |label| < 2^24 the exact product of |label| and
//    q's 53-bit significand comes from two 32 x 32 -> 64 integer multiplies
//    and is rounded to nearest even at 53 bits (the FP64 multiply) and then
//    at 24 bits (the conversion); other labels, results outside the normal
//    FP32 range and FP64 output use one FP64 multiply with the int64 -> FP64
//    conversion built from the bits.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "pdl.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kFlagNonfinite = 1u;
constexpr unsigned kFlagOverflow = 2u;

// Nearest integer with ties away from zero.  y - trunc(y) is exact in binary
// floating point, so comparing it with 0.5 decides the rounding exactly.
__device__ __forceinline__ long long round_half_away(double y) {
  const double t = trunc(y);
  const double fr = y - t;
  long long k = static_cast<long long>(t);
  if (fr >= 0.5) k += 1;
  else if (fr <= -0.5) k -= 1;
  return k;
}

template <typename T>
__device__ __forceinline__ long long quantize_one(T x, double q, float rq, unsigned& bad) {
  const float x32 = static_cast<float>(x);
  const float y = __fmul_rn(x32, rq);
  const float ay = fabsf(y);
  const float t = truncf(y);
  const float fr = __fsub_rn(y, t);
  const float afr = fabsf(fr);
  const float dist = fabsf(afr - 0.5f);
  const bool x_ok = (x32 == 0.0f) || (fabsf(x32) >= FLT_MIN);
  if (x_ok && ay < 1048576.0f && dist > ay * 4.76837158203125e-07f + FLT_MIN) {  // 2^20, 2^-21
    int k = static_cast<int>(t);
    if (afr >= 0.5f) k += (y > 0.0f) ? 1 : -1;
    return k;
  }
  const double xd = static_cast<double>(x);
  if (!isfinite(xd)) {
    bad |= kFlagNonfinite;
    return 0;
  }
  const double yd = xd / q;
  if (fabs(yd) >= 4611686018427387904.0) {  // 2^62
    bad |= kFlagOverflow;
    return 0;
  }
  return round_half_away(yd);
}

// fl32(fl64(k q)) from integer arithmetic for 0 < |k| < 2^24 and q > 0 normal:
// the exact product |k| m_q (m_q the 53-bit significand of q) is formed from
// two 32 x 32 -> 64 multiplies, rounded to nearest even at 53 bits (the FP64
// multiply) and again at 24 bits (the conversion to FP32).  Returns false when
// the result is outside the normal FP32 range.
__device__ __forceinline__ bool mul_f32_exact(long long k, unsigned long long qbits, float& out) {
  const unsigned K = static_cast<unsigned>(k < 0 ? -k : k);
  const unsigned long long mq = (qbits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int eq = static_cast<int>((qbits >> 52) & 0x7FF) - 1075;  // q = mq 2^eq
  const unsigned long long plo = static_cast<unsigned long long>(K) * static_cast<unsigned>(mq);
  const unsigned long long phi = static_cast<unsigned long long>(K) * static_cast<unsigned>(mq >> 32);
  const unsigned lo32 = static_cast<unsigned>(plo);
  const unsigned long long mid = (plo >> 32) + phi;  // product = mid 2^32 + lo32, mid >= 2^20
  const int bm = 64 - __clzll(static_cast<long long>(mid));
  int s = bm - 21;  // bits below the 53 kept ones, 0 .. 24
  unsigned long long m53;
  if (s == 0) {
    m53 = (mid << 32) | lo32;
  } else {
    m53 = (mid << (32 - s)) | (lo32 >> s);
    const unsigned rem = lo32 & ((1u << s) - 1u), half = 1u << (s - 1);
    if (rem > half || (rem == half && (m53 & 1ull))) {
      ++m53;
      if (m53 == (1ull << 53)) { m53 >>= 1; ++s; }
    }
  }
  int E = eq + s + 52;  // exponent of the FP64 product
  if (E < -126 || E > 127) return false;
  unsigned m24 = static_cast<unsigned>(m53 >> 29);
  const unsigned rem2 = static_cast<unsigned>(m53) & 0x1FFFFFFFu, half2 = 0x10000000u;
  if (rem2 > half2 || (rem2 == half2 && (m24 & 1u))) {
    ++m24;
    if (m24 == (1u << 24)) { m24 >>= 1; ++E; }
  }
  if (E > 127) return false;
  out = __uint_as_float((k < 0 ? 0x80000000u : 0u) | (static_cast<unsigned>(E + 127) << 23) |
                        (m24 & 0x7FFFFFu));
  return true;
}

// Exact int64 -> FP64 for 0 < |k| < 2^53, built from the bits.
__device__ __forceinline__ double i64_to_f64(long long k) {
  const unsigned long long K = k < 0 ? static_cast<unsigned long long>(-k) : static_cast<unsigned long long>(k);
  const int nb = 64 - __clzll(static_cast<long long>(K));  // 1 .. 53
  const unsigned long long mant = K << (53 - nb);           // leading bit at 52
  const unsigned long long bits = (k < 0 ? (1ull << 63) : 0ull) |
                                  (static_cast<unsigned long long>(1022 + nb) << 52) |
                                  (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double(static_cast<long long>(bits));
}

// FP64 -> FP32 with round to nearest even, done on the bits, for results in
// the normal FP32 range; returns false otherwise.
__device__ __forceinline__ bool f64_to_f32(double y, float& out) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(y));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const int e = static_cast<int>((hi >> 20) & 0x7FF) - 1023;
  if (e < -126 || e > 127) return false;
  unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // 23 fraction bits
  const unsigned rem = lo & 0x1FFFFFFFu, half = 0x10000000u;
  if (rem > half || (rem == half && (m & 1u))) ++m;
  unsigned eb = static_cast<unsigned>(e + 127);
  if (m == 0x800000u) {
    m = 0;
    if (++eb >= 255u) return false;
  }
  out = __uint_as_float((hi & 0x80000000u) | (eb << 23) | m);
  return true;
}

// The FP64 route of dequantization, kept out of line so that the common
// integer route carries no FP64 instruction.
__device__ __noinline__ float dequantize_f64_route(long long k, double q) {
  const long long ak = k < 0 ? -k : k;
  if (ak >= (1ll << 53)) return static_cast<float>(static_cast<double>(k) * q);
  const double y = i64_to_f64(k) * q;
  float r;
  return f64_to_f32(y, r) ? r : static_cast<float>(y);
}

// FP32 route of fl32(fl64(k q)) for 0 < |k| < 2^24, with qf = fl32(q) and
// dqf = fl32(q - qf): K qf = p + e exactly (FMA remainder), t = K dqf + e
// (one rounding), r = fl32(p + t) and delta = p + t - r exactly (Fast2Sum).
// |K q - (p + t)| < 2^-46 |r|, so when delta is farther than 2^-40 |r| from
// the midpoint towards the neighbouring float, K q rounds to r both in one
// step and through FP64 (whose rounding moves it by at most 2^-53 |r|).
// Returns false near a midpoint or outside [2^-100, FLT_MAX].
__device__ __forceinline__ bool deq_f32_fast(long long k, float qf, float dqf, float& out) {
  const float K = static_cast<float>(static_cast<int>(k < 0 ? -k : k));  // exact: |k| < 2^24
  const float p = __fmul_rn(K, qf);
  const float e = __fmaf_rn(K, qf, -p);
  const float t = __fmaf_rn(K, dqf, e);
  const float r = __fadd_rn(p, t);
  const float delta = __fsub_rn(t, __fsub_rn(r, p));
  const unsigned rb = __float_as_uint(r);
  const float nb = __uint_as_float(delta >= 0.0f ? rb + 1u : rb - 1u);
  const float h = __fmul_rn(fabsf(__fsub_rn(nb, r)), 0.5f);
  const float ar = fabsf(r);
  if (!(fabsf(delta) < h - ar * 9.094947017729282e-13f) || !(ar >= 7.888609052210118e-31f) ||
      !(ar <= FLT_MAX))  // 2^-40, 2^-100
    return false;
  out = k < 0 ? -r : r;
  return true;
}

// label * q in FP64, rounded to the element type.  FP32: the FP32 route,
// then the exact integer route, then one FP64 multiply.
__device__ __forceinline__ float dequantize_one(long long k, double q, float qf, float dqf, float*) {
  if (k == 0) return 0.0f;
  const long long ak = k < 0 ? -k : k;
  float r;
  if (ak < (1ll << 24) && deq_f32_fast(k, qf, dqf, r)) return r;
  if (ak < (1ll << 24) && mul_f32_exact(k, static_cast<unsigned long long>(__double_as_longlong(q)), r))
    return r;
  return dequantize_f64_route(k, q);
}

__device__ __forceinline__ double dequantize_one(long long k, double q, float, float, double*) {
  if (k == 0) return 0.0;
  const long long ak = k < 0 ? -k : k;
  if (ak >= (1ll << 53)) return static_cast<double>(k) * q;
  return i64_to_f64(k) * q;
}

struct SmemTable {
  double q[48];
  float rq[48];
  float qf[48];
  float dqf[48];
};

// The level table in shared memory: the host's, or (rt.range set) the same
// table formed from the device range, one thread per level, with the
// operations of the host's level_tolerances and make_level_table.
__device__ __forceinline__ void load_table(const LevelTable& tab, const RelTol& rt, SmemTable& s) {
  if (rt.range == nullptr) {
    for (int i = threadIdx.x; i < 48; i += blockDim.x) {
      s.q[i] = tab.q[i];
      s.rq[i] = tab.rq[i];
      s.qf[i] = tab.qf[i];
      s.dqf[i] = tab.dqf[i];
    }
  } else if (threadIdx.x < 48) {
    const int l = threadIdx.x;
    const double tau = __dmul_rn(rt.rel, __dsub_rn(rt.range[1], rt.range[0]));
    const double t0 = __ddiv_rn(__dmul_rn(__dsub_rn(1.0, rt.kappa), tau),
                                __dmul_rn(__dsub_rn(1.0, rt.kpow), rt.C));
    if (l == 0 && !(tau > 0.0 && isfinite(tau) && t0 > 0.0 && isfinite(t0)) && rt.flags)
      atomicOr(rt.flags, 4u);
    double q = 1.0;
    float rq = __int_as_float(0x7fc00000), qf = 1.0f, dqf = 0.0f;
    if (l <= rt.L) {
      double t = t0;  // tau of level max(l, stop)
      for (int k = rt.stop + 1; k <= l; ++k) t = __dmul_rn(rt.kappa, t);
      q = __dmul_rn(2.0, t);
      const float rf = __double2float_rn(__ddiv_rn(1.0, q));
      rq = (isfinite(rf) && rf >= 1.17549435e-38f) ? rf : __int_as_float(0x7fc00000);
      const float qf0 = __double2float_rn(q);
      const bool qok = isfinite(qf0) && qf0 >= 1.17549435e-38f;
      qf = qok ? qf0 : __int_as_float(0x7fc00000);
      dqf = qok ? __double2float_rn(__dsub_rn(q, static_cast<double>(qf0))) : 0.0f;
    }
    s.q[l] = q;
    s.rq[l] = rq;
    s.qf[l] = qf;
    s.dqf[l] = dqf;
  }
  __syncthreads();
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float v[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void store(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double v[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double v[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
};

// Row tiles: a CTA takes kQRows consecutive rows of the field and a chunk of
// columns, one thread per column.  The level of node (row, column) is
// max(level of the row, level of the column, stopping level); the column's
// level stays in a register and the row's is uniform, so the tolerance comes
// from a shared-memory table.  All kQRows loads of a thread are issued first.
constexpr int kQRows = 8;
constexpr int kQCols = 640;

template <typename T>
__global__ void __launch_bounds__(kQCols)
quantize_kernel(const T* __restrict__ coeffs, int64_t* __restrict__ labels,
                const uint8_t* __restrict__ lev01, const uint8_t* __restrict__ lev2, int64_t n2,
                int64_t nrows, int stop, LevelTable tab, unsigned int* __restrict__ flags,
                RelTol rt) {
  grid_dep_enter();
  __shared__ SmemTable st;
  load_table(tab, rt, st);
  const int64_t ngroups = (nrows + kQRows - 1) / kQRows;
  const int64_t nchunks = (n2 + blockDim.x - 1) / blockDim.x;
  unsigned bad = 0;
  for (int64_t b = blockIdx.x; b < ngroups * nchunks; b += gridDim.x) {
    const int64_t rg = b / nchunks, cx = b - rg * nchunks;
    const int64_t j2 = cx * blockDim.x + threadIdx.x;
    if (j2 >= n2) continue;
    const int64_t r0 = rg * kQRows;
    const int lc = max(static_cast<int>(__ldg(lev2 + j2)), stop);
    T x[kQRows];
#pragma unroll
    for (int u = 0; u < kQRows; ++u)
      if (r0 + u < nrows) x[u] = coeffs[(r0 + u) * n2 + j2];
#pragma unroll
    for (int u = 0; u < kQRows; ++u) {
      if (r0 + u < nrows) {
        const int l = max(static_cast<int>(__ldg(lev01 + r0 + u)), lc);
        labels[(r0 + u) * n2 + j2] = quantize_one(x[u], st.q[l], st.rq[l], bad);
      }
    }
  }
  if (bad) atomicOr(flags, bad);
}

template <typename T>
__global__ void __launch_bounds__(kQCols)
dequantize_kernel(const int64_t* __restrict__ labels, T* __restrict__ coeffs,
                  const uint8_t* __restrict__ lev01, const uint8_t* __restrict__ lev2, int64_t n2,
                  int64_t nrows, int stop, LevelTable tab, RelTol rt) {
  grid_dep_enter();
  __shared__ SmemTable st;
  load_table(tab, rt, st);
  const int64_t ngroups = (nrows + kQRows - 1) / kQRows;
  const int64_t nchunks = (n2 + blockDim.x - 1) / blockDim.x;
  for (int64_t b = blockIdx.x; b < ngroups * nchunks; b += gridDim.x) {
    const int64_t rg = b / nchunks, cx = b - rg * nchunks;
    const int64_t j2 = cx * blockDim.x + threadIdx.x;
    if (j2 >= n2) continue;
    const int64_t r0 = rg * kQRows;
    const int lc = max(static_cast<int>(__ldg(lev2 + j2)), stop);
    long long k[kQRows];
#pragma unroll
    for (int u = 0; u < kQRows; ++u)
      if (r0 + u < nrows) k[u] = labels[(r0 + u) * n2 + j2];
#pragma unroll
    for (int u = 0; u < kQRows; ++u) {
      if (r0 + u < nrows) {
        const int l = max(static_cast<int>(__ldg(lev01 + r0 + u)), lc);
        coeffs[(r0 + u) * n2 + j2] =
            dequantize_one(k[u], st.q[l], st.qf[l], st.dqf[l], static_cast<T*>(nullptr));
      }
    }
  }
}

// Flat forms for aligned arrays: a thread takes vectors of 4 consecutive
// elements (16-byte loads and stores), QU vectors in flight, over a
// persistent grid of TH-thread blocks.  Shapes measured at 513^3 FP32 on
// GB300 over QU x TH in {1, 2, 3, 4, 8} x {128, 256, 512, 1024}: quantize
// 3 x 512 (258 us, 0.92 of the copy peak), dequantize 1 x 1024 (265 us).  The row of element e is umulhi(e, M) with
// M = ceil(2^64 / n2), exact for every e of the array (checked on the host);
// the 4 elements of a vector span at most two rows (n2 >= 4).
constexpr int kQUq = 3, kQThreadsQ = 512;    // quantize
constexpr int kQUd = 1, kQThreadsD = 1024;   // dequantize

__device__ __forceinline__ void vec_levels(uint64_t e, uint64_t magic, uint32_t n2,
                                           const uint8_t* __restrict__ lev01,
                                           const uint8_t* __restrict__ lev2, int stop, int lv[4]) {
  const uint64_t row = __umul64hi(e, magic);
  const uint32_t col = static_cast<uint32_t>(e - row * n2);
  const int la = max(static_cast<int>(__ldg(lev01 + row)), stop);
  const int lb = (col + 3 >= n2) ? max(static_cast<int>(__ldg(lev01 + row + 1)), stop) : la;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uint32_t c = col + u;
    const bool wrap = c >= n2;
    if (wrap) c -= n2;
    lv[u] = max(static_cast<int>(__ldg(lev2 + c)), wrap ? lb : la);
  }
}

template <typename T>
__global__ void __launch_bounds__(kQThreadsQ)
quantize_flat_kernel(const T* __restrict__ coeffs, int64_t* __restrict__ labels,
                     const uint8_t* __restrict__ lev01, const uint8_t* __restrict__ lev2,
                     uint64_t nvec, uint32_t n2, uint64_t magic, int stop, LevelTable tab,
                     unsigned int* __restrict__ flags, RelTol rt) {
  grid_dep_enter();
  __shared__ SmemTable st;
  load_table(tab, rt, st);
  unsigned bad = 0;
  constexpr int QU = kQUq, TH = kQThreadsQ;
  const uint64_t step = static_cast<uint64_t>(gridDim.x) * TH * QU;
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * TH * QU + threadIdx.x;
       base < nvec; base += step) {
    T x[QU][4];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const uint64_t v = base + static_cast<uint64_t>(u) * TH;
      if (v < nvec) Vec4<T>::load(coeffs + 4 * v, x[u]);
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const uint64_t v = base + static_cast<uint64_t>(u) * TH;
      if (v < nvec) {
        int lv[4];
        vec_levels(4 * v, magic, n2, lev01, lev2, stop, lv);
        long long k[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) k[i] = quantize_one(x[u][i], st.q[lv[i]], st.rq[lv[i]], bad);
        longlong2* out = reinterpret_cast<longlong2*>(labels + 4 * v);
        out[0] = make_longlong2(k[0], k[1]);
        out[1] = make_longlong2(k[2], k[3]);
      }
    }
  }
  if (bad) atomicOr(flags, bad);
}

template <typename T>
__global__ void __launch_bounds__(kQThreadsD)
dequantize_flat_kernel(const int64_t* __restrict__ labels, T* __restrict__ coeffs,
                       const uint8_t* __restrict__ lev01, const uint8_t* __restrict__ lev2,
                       uint64_t nvec, uint32_t n2, uint64_t magic, int stop, LevelTable tab,
                       RelTol rt) {
  grid_dep_enter();
  __shared__ SmemTable st;
  load_table(tab, rt, st);
  constexpr int QU = kQUd, TH = kQThreadsD;
  const uint64_t step = static_cast<uint64_t>(gridDim.x) * TH * QU;
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * TH * QU + threadIdx.x;
       base < nvec; base += step) {
    longlong2 k[QU][2];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const uint64_t v = base + static_cast<uint64_t>(u) * TH;
      if (v < nvec) {
        const longlong2* in = reinterpret_cast<const longlong2*>(labels + 4 * v);
        k[u][0] = in[0];
        k[u][1] = in[1];
      }
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const uint64_t v = base + static_cast<uint64_t>(u) * TH;
      if (v < nvec) {
        int lv[4];
        vec_levels(4 * v, magic, n2, lev01, lev2, stop, lv);
        const long long kk[4] = {k[u][0].x, k[u][0].y, k[u][1].x, k[u][1].y};
        T y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          y[i] = dequantize_one(kk[i], st.q[lv[i]], st.qf[lv[i]], st.dqf[lv[i]],
                                static_cast<T*>(nullptr));
        Vec4<T>::store(coeffs + 4 * v, y);
      }
    }
  }
}

// Block-wide min/max in the element type (exact), then FP64 partials;
// non-finite elements are flagged and left out.
template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }
template <typename T>
struct Lim;
template <>
struct Lim<float> { static __device__ __forceinline__ float max() { return FLT_MAX; } };
template <>
struct Lim<double> { static __device__ __forceinline__ double max() { return DBL_MAX; } };

// Value range: a grid of kRangeBlocks x kThreads threads, kRangeLoads
// 16-byte loads in flight per thread (measured at 513^3 FP32 on GB300 over
// {2, 4, 8} loads x {608, 1216, 2432} blocks: 8 x 608, 91 us).
constexpr int kRangeLoads = 8;
constexpr int kRangeBlocks = 608;

template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads)
minmax_partial_kernel(const T* __restrict__ data, uint64_t count, double* __restrict__ partial,
                      unsigned int* __restrict__ flags) {
  grid_dep_enter();
  __shared__ T smin[kThreads], smax[kThreads];
  T mn = Lim<T>::max(), mx = -Lim<T>::max();
  bool bad = false;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (VEC) {
    // kRangeLoads 16-byte loads of a thread in flight at a time.
    const uint64_t ngroups = count / 4;
    uint64_t g = tid;
    for (; g + (kRangeLoads - 1) * stride < ngroups; g += kRangeLoads * stride) {
      T v[kRangeLoads][4];
#pragma unroll
      for (int i = 0; i < kRangeLoads; ++i) Vec4<T>::load(data + (g + i * stride) * 4, v[i]);
#pragma unroll
      for (int i = 0; i < kRangeLoads; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          bad |= !finite_val(v[i][u]);
          mn = fmin(mn, v[i][u]);
          mx = fmax(mx, v[i][u]);
        }
    }
    for (; g < ngroups; g += stride) {
      T v[4];
      Vec4<T>::load(data + g * 4, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bad |= !finite_val(v[u]);
        mn = fmin(mn, v[u]);
        mx = fmax(mx, v[u]);
      }
    }
    done = ngroups * 4;
  }
  for (uint64_t e = done + tid; e < count; e += stride) {
    const T v = data[e];
    bad |= !finite_val(v);
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  if (bad) atomicOr(flags, kFlagNonfinite);
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = static_cast<double>(smin[0]);
    partial[2 * blockIdx.x + 1] = static_cast<double>(smax[0]);
  }
}

__global__ void __launch_bounds__(kThreads)
minmax_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ result) {
  grid_dep_enter();
  __shared__ double smin[kThreads], smax[kThreads];
  double mn = DBL_MAX, mx = -DBL_MAX;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    mn = fmin(mn, partial[2 * i]);
    mx = fmax(mx, partial[2 * i + 1]);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = smin[0];
    result[1] = smax[0];
  }
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


}  // namespace

// Row-tile kernels run as a persistent grid: as many CTAs as fit on the
// 152 SMs at once, each looping over row groups, so no CTA is launched for
// a few KB of work.
template <typename K>
unsigned row_blocks(K kernel, int64_t nrows, int64_t n2, int threads) {
  const int64_t work = ((nrows + kQRows - 1) / kQRows) * ((n2 + threads - 1) / threads);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  const int64_t cap = 152 * static_cast<int64_t>(std::max(per_sm, 1));
  return static_cast<unsigned>(std::max<int64_t>(1, std::min(work, cap)));
}

// M = ceil(2^64 / n2) gives row = umulhi(e, M) exactly while e (M n2 - 2^64)
// < 2^64 for every element index e < count.
bool flat_magic(uint64_t count, int64_t n2, uint64_t& magic) {
  if (n2 < 4 || n2 > (int64_t(1) << 31)) return false;
  const unsigned __int128 two64 = static_cast<unsigned __int128>(1) << 64;
  const unsigned __int128 m = (two64 + static_cast<uint64_t>(n2) - 1) / static_cast<uint64_t>(n2);
  if (m >> 64) return false;
  const unsigned __int128 eps = m * static_cast<uint64_t>(n2) - two64;
  if (eps != 0 && static_cast<unsigned __int128>(count) * eps >= two64) return false;
  magic = static_cast<uint64_t>(m);
  return true;
}

template <typename K>
unsigned flat_blocks(K kernel, uint64_t nvec, int threads, int qu) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  const uint64_t need = (nvec + uint64_t(threads) * qu - 1) / (uint64_t(threads) * qu);
  const uint64_t cap = 152ull * static_cast<uint64_t>(std::max(per_sm, 1));
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min(need, cap)));
}

int row_threads(int64_t n2) {
  const int64_t t = 32 * ((std::min<int64_t>(n2, kQCols) + 31) / 32);
  return static_cast<int>(t < 64 ? 64 : t);
}

template <typename T>
cudaError_t launch_quantize(const T* coeffs, int64_t* labels, const uint8_t* lev01,
                            const uint8_t* lev2, int64_t rows, int64_t n2, int stop_level,
                            const LevelTable& tab, unsigned int* flags, cudaStream_t s,
                            const RelTol* rtp) {
  const RelTol rt = rtp ? *rtp : RelTol{};
  const uint64_t count = static_cast<uint64_t>(rows) * n2;
  TraceScope ts(kKQuantize, -1, double(count) * (sizeof(T) + 8), s);
  uint64_t magic = 0;
  if (aligned16(coeffs) && aligned16(labels) && flat_magic(count, n2, magic)) {
    const uint64_t nvec = count / 4;
    if (nvec > 0)
      launch_pdl(quantize_flat_kernel<T>,
                 dim3(flat_blocks(quantize_flat_kernel<T>, nvec, kQThreadsQ, kQUq)),
                 dim3(kQThreadsQ), 0, s, coeffs, labels, lev01, lev2, nvec,
                 static_cast<uint32_t>(n2), magic, stop_level, tab, flags, rt);
    if (count % 4 == 0) return cudaGetLastError();
    // The last count % 4 elements: one row-tile pass over the last row
    // would redo work, so the row-tile kernel takes the whole last row.
    const int64_t r_last = rows - 1;
    ts.more_kernels(1);
    launch_pdl(quantize_kernel<T>, dim3(1), dim3(row_threads(n2)), 0, s, coeffs + r_last * n2,
               labels + r_last * n2, lev01 + r_last, lev2, n2, 1, stop_level, tab, flags, rt);
    return cudaGetLastError();
  }
  const int threads = row_threads(n2);
  launch_pdl(quantize_kernel<T>, dim3(row_blocks(quantize_kernel<T>, rows, n2, threads)),
             dim3(threads), 0, s, coeffs, labels, lev01, lev2, n2, rows, stop_level, tab, flags, rt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dequantize(const int64_t* labels, T* coeffs, const uint8_t* lev01,
                              const uint8_t* lev2, int64_t rows, int64_t n2, int stop_level,
                              const LevelTable& tab, cudaStream_t s, const RelTol* rtp) {
  const RelTol rt = rtp ? *rtp : RelTol{};
  const uint64_t count = static_cast<uint64_t>(rows) * n2;
  TraceScope ts(kKDequantize, -1, double(count) * (sizeof(T) + 8), s);
  uint64_t magic = 0;
  if (aligned16(coeffs) && aligned16(labels) && flat_magic(count, n2, magic)) {
    const uint64_t nvec = count / 4;
    if (nvec > 0)
      launch_pdl(dequantize_flat_kernel<T>,
                 dim3(flat_blocks(dequantize_flat_kernel<T>, nvec, kQThreadsD, kQUd)),
                 dim3(kQThreadsD), 0, s, labels, coeffs, lev01, lev2, nvec,
                 static_cast<uint32_t>(n2), magic, stop_level, tab, rt);
    if (count % 4 == 0) return cudaGetLastError();
    const int64_t r_last = rows - 1;
    ts.more_kernels(1);
    launch_pdl(dequantize_kernel<T>, dim3(1), dim3(row_threads(n2)), 0, s, labels + r_last * n2,
               coeffs + r_last * n2, lev01 + r_last, lev2, n2, 1, stop_level, tab, rt);
    return cudaGetLastError();
  }
  const int threads = row_threads(n2);
  launch_pdl(dequantize_kernel<T>, dim3(row_blocks(dequantize_kernel<T>, rows, n2, threads)),
             dim3(threads), 0, s, labels, coeffs, lev01, lev2, n2, rows, stop_level, tab, rt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_minmax(const T* data, int64_t count, double* partial, unsigned int* flags,
                          double* result, cudaStream_t s) {
  int64_t blocks = (count / 4 + kThreads - 1) / kThreads;
  if (blocks > kRangeBlocks) blocks = kRangeBlocks;
  if (blocks < 1) blocks = 1;
  TraceScope ts(kKMinmax, -1, double(count) * sizeof(T), s);
  if (aligned16(data))
    launch_pdl(minmax_partial_kernel<T, true>, dim3(static_cast<unsigned>(blocks)), dim3(kThreads),
               0, s, data, static_cast<uint64_t>(count), partial, flags);
  else
    launch_pdl(minmax_partial_kernel<T, false>, dim3(static_cast<unsigned>(blocks)), dim3(kThreads),
               0, s, data, static_cast<uint64_t>(count), partial, flags);
  ts.more_kernels(1);
  launch_pdl(minmax_final_kernel, dim3(1), dim3(kThreads), 0, s, partial, static_cast<int>(blocks),
             result);
  return cudaGetLastError();
}

#define MGB_INST(T)                                                                             \
  template cudaError_t launch_quantize<T>(const T*, int64_t*, const uint8_t*, const uint8_t*,  \
                                          int64_t, int64_t, int, const LevelTable&,             \
                                          unsigned int*, cudaStream_t, const RelTol*);          \
  template cudaError_t launch_dequantize<T>(const int64_t*, T*, const uint8_t*, const uint8_t*, \
                                            int64_t, int64_t, int, const LevelTable&,           \
                                            cudaStream_t, const RelTol*);                       \
  template cudaError_t launch_minmax<T>(const T*, int64_t, double*, unsigned int*, double*,    \
                                        cudaStream_t);
MGB_INST(float)
MGB_INST(double)
#undef MGB_INST

}  // namespace mgb
