// Canonical Huffman coding of the labels (the lossless encoder of Algorithm
// 1 line 23, which the paper does not name; Huffman's code reaches the
// order-0 entropy that Section 4.1's cost estimate uses within one bit per
// label), the labels' order-0 entropy, and the cost model of Section 4.1.
//
// Stream layout (little-endian): uint64 N | uint32 K = 32817 | uint32
// longest code length | K bytes of code lengths (0 = unused symbol) | zero
// padding to 8 bytes | per chunk of 1024 labels a uint32 payload word count
// | zero padding to 8 bytes | per chunk its 64-bit words.  A label's zigzag code z is symbol z
// when z < 2^15; a larger z of bit length b is symbol 32768 + b - 16
// followed by its b - 1 low bits (the leading 1 implied), as DEFLATE codes
// lengths with extra bits.  Each symbol's canonical code is written most
// significant bit first at increasing bit positions from the least
// significant bit of the chunk's first word, its extra bits after it, least
// significant first.
//
// Code lengths come from Huffman's construction with a fixed order (leaves
// sorted by (count, symbol), merged nodes queued in creation order, a leaf
// taken on a tie), on the host from the device histogram; a code longer
// than 31 bits makes every used count c become max(1, c / 2) and the code
// is rebuilt.  Canonical codes: symbols ordered by (length, symbol) take
// consecutive values, shifted left at each length step.
//
// Encoding: a histogram pass (per-CTA shared-memory bins for the small
// symbols), the code on the host, a warp per chunk for its size, a scan,
// and a warp per chunk that assembles the chunk's words in shared memory.
// Decoding: a thread per chunk reads its bits through an 11-bit lookup
// table of the short codes and the canonical first-code table otherwise.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "mgard_gb.h"
#include "pdl.cuh"
#include "plan.hpp"

namespace mgb {
namespace {

constexpr int kHuffDirect = 32768;    // zigzag codes below this are their own symbol
constexpr int kHuffK = kHuffDirect + 49;  // then one symbol per bit length 16 .. 64
constexpr int kHuffChunk = 1024;
constexpr int kHuffMaxLen = 31;
constexpr int kSmemBins = 8192;   // symbols counted in shared memory per CTA
constexpr int kPeekBits = 11;     // decoder lookup table of the short codes
constexpr int kHeaderFixed = 16;  // N, K, longest length
constexpr int kEncWarps = 8;
constexpr int kChunkWords = (kHuffChunk * (kHuffMaxLen + 63) + 63) / 64;  // 1504

__device__ __forceinline__ uint64_t zig(int64_t k) {
  return (static_cast<uint64_t>(k) << 1) ^ static_cast<uint64_t>(k >> 63);
}
__device__ __forceinline__ int64_t unzig(uint64_t z) {
  return static_cast<int64_t>(z >> 1) ^ -static_cast<int64_t>(z & 1);
}
// Symbol of a zigzag code, and the number of its extra bits.
__device__ __forceinline__ uint32_t symbol_of(uint64_t z, uint32_t& nx) {
  if (z < uint64_t(kHuffDirect)) {
    nx = 0;
    return static_cast<uint32_t>(z);
  }
  const uint32_t b = 64u - static_cast<uint32_t>(__clzll(static_cast<long long>(z)));
  nx = b - 1;
  return uint32_t(kHuffDirect) + b - 16;
}

inline unsigned grid_for(int64_t n, int per) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(152 * 8, (n + per - 1) / per)));
}

// ------------------------------------------------------------------ kernels

__global__ void __launch_bounds__(256)
huff_hist_kernel(const int64_t* __restrict__ labels, int64_t n, unsigned long long* __restrict__ hist) {
  grid_dep_enter();
  __shared__ unsigned int bins[kSmemBins];
  for (int i = threadIdx.x; i < kSmemBins; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    uint32_t nx;
    const uint32_t s = symbol_of(zig(labels[t]), nx);
    if (s < uint32_t(kSmemBins)) atomicAdd(&bins[s], 1u);
    else atomicAdd(&hist[s], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSmemBins; i += blockDim.x)
    if (bins[i]) atomicAdd(&hist[i], static_cast<unsigned long long>(bins[i]));
}

// The zigzag codes of 2^15 and above, compacted in any order (the entropy
// counts their distinct values).
__global__ void __launch_bounds__(256)
huff_large_codes_kernel(const int64_t* __restrict__ labels, int64_t n, uint64_t* __restrict__ out,
                    unsigned long long* __restrict__ count, unsigned long long cap) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t z = zig(labels[t]);
    if (z >= uint64_t(kHuffDirect)) {
      const unsigned long long i = atomicAdd(count, 1ull);
      if (i < cap) out[i] = z;
    }
  }
}

// Per chunk: payload words, also written to the stream's chunk table.
__global__ void __launch_bounds__(256)
huff_sizes_kernel(const int64_t* __restrict__ labels, int64_t n, int64_t nchunks,
                  const uint64_t* __restrict__ enc, uint64_t* __restrict__ words,
                  uint32_t* __restrict__ table, unsigned long long* __restrict__ maxw) {
  grid_dep_enter();
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t c = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += nw) {
    const int64_t base = c * kHuffChunk;
    const int nc = static_cast<int>(min(int64_t(kHuffChunk), n - base));
    uint64_t bits = 0;
    for (int i = lane; i < nc; i += 32) {
      uint32_t nx;
      const uint32_t s = symbol_of(zig(labels[base + i]), nx);
      bits += (enc[s] >> 32) + nx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
    if (lane == 0) {
      const uint64_t w = (bits + 63) / 64;
      words[c] = w;
      table[c] = static_cast<uint32_t>(w);
      atomicMax(maxw, static_cast<unsigned long long>(w));
    }
  }
}

// Exclusive prefix sum in place in one CTA; total[0] gets the sum.
constexpr int kScanT = 1024;
__global__ void __launch_bounds__(kScanT)
huff_scan_kernel(uint64_t* __restrict__ v, int64_t n, uint64_t* __restrict__ total) {
  grid_dep_enter();
  __shared__ uint64_t s[kScanT];
  const int t = threadIdx.x;
  const int64_t per = (n + kScanT - 1) / kScanT;
  const int64_t lo = min(n, t * per), hi = min(n, lo + per);
  uint64_t run = 0;
  for (int64_t i = lo; i < hi; ++i) run += v[i];
  s[t] = run;
  __syncthreads();
  for (int off = 1; off < kScanT; off <<= 1) {
    const uint64_t add = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  uint64_t acc = s[t] - run;
  for (int64_t i = lo; i < hi; ++i) {
    const uint64_t w = v[i];
    v[i] = acc;
    acc += w;
  }
  if (t == kScanT - 1) total[0] = s[t];
}

// A warp per chunk: bit positions by a warp scan of the labels' bit counts
// (code + extra bits), the chunk's words assembled in shared memory, then
// stored.
// Each warp's words sit in dynamic shared memory at a pitch of the
// largest chunk's word count.
__global__ void __launch_bounds__(32 * kEncWarps)
huff_encode_kernel(const int64_t* __restrict__ labels, int64_t n, int64_t nchunks,
                   const uint64_t* __restrict__ enc, const uint64_t* __restrict__ woff,
                   uint64_t* __restrict__ payload, int pitch) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned long long sw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long* w = sw + static_cast<size_t>(wid) * pitch;
  const int64_t nw = int64_t(gridDim.x) * kEncWarps;
  for (int64_t c = int64_t(blockIdx.x) * kEncWarps + wid; c < nchunks; c += nw) {
    for (int i = lane; i < pitch; i += 32) w[i] = 0ull;
    __syncwarp();
    const int64_t base = c * kHuffChunk;
    const int nc = static_cast<int>(min(int64_t(kHuffChunk), n - base));
    uint64_t pos = 0;
    for (int i0 = 0; i0 < nc; i0 += 32) {
      const int i = i0 + lane;
      uint32_t len = 0, code = 0, nx = 0;
      uint64_t z = 0;
      if (i < nc) {
        z = zig(labels[base + i]);
        const uint32_t s = symbol_of(z, nx);
        const uint64_t e = enc[s];
        len = static_cast<uint32_t>(e >> 32);
        code = static_cast<uint32_t>(e);
      }
      const uint32_t tl = len + nx;
      uint32_t incl = tl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint64_t b = pos + incl - tl;
      if (len) {
        // Bit j of the code (from its most significant end) goes to b + j:
        // the reversed code, shifted into place.
        const uint64_t rc = static_cast<uint64_t>(__brev(code) >> (32 - len));
        const uint32_t word = static_cast<uint32_t>(b >> 6), sh = static_cast<uint32_t>(b & 63);
        atomicOr(&w[word], static_cast<unsigned long long>(rc << sh));
        if (sh + len > 64) atomicOr(&w[word + 1], static_cast<unsigned long long>(rc >> (64 - sh)));
      }
      if (nx) {
        const uint64_t x = z & ((uint64_t(1) << nx) - 1);  // the low b - 1 bits
        const uint64_t p = b + len;
        const uint32_t word = static_cast<uint32_t>(p >> 6), sh = static_cast<uint32_t>(p & 63);
        atomicOr(&w[word], static_cast<unsigned long long>(x << sh));
        if (sh + nx > 64) atomicOr(&w[word + 1], static_cast<unsigned long long>(x >> (64 - sh)));
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const uint64_t nwords = (pos + 63) / 64;
    uint64_t* dst = payload + woff[c];
    for (uint64_t i = lane; i < nwords; i += 32) dst[i] = w[i];
    __syncwarp();
  }
}

// Decoder tables.
struct DecTables {
  uint32_t first[kHuffMaxLen + 2];   // first canonical code of each length
  uint32_t count[kHuffMaxLen + 2];   // codes of each length
  uint32_t offset[kHuffMaxLen + 2];  // index of the length's first symbol in `sorted`
  int maxlen;
};

// The 64 bits of a chunk from bit `pos` on (zeros past the chunk).
__device__ __forceinline__ uint64_t bits_at(const uint64_t* __restrict__ src, uint64_t nwords,
                                            uint64_t pos) {
  const uint64_t wi = pos >> 6;
  const uint32_t sh = static_cast<uint32_t>(pos & 63);
  uint64_t buf = wi < nwords ? src[wi] >> sh : 0ull;
  if (sh && wi + 1 < nwords) buf |= src[wi + 1] << (64 - sh);
  return buf;
}

__global__ void __launch_bounds__(128)
huff_decode_kernel(const uint64_t* __restrict__ payload, const uint64_t* __restrict__ woff,
                   const uint32_t* __restrict__ peek, const uint16_t* __restrict__ sorted,
                   DecTables dt, int64_t n, int64_t nchunks, int64_t* __restrict__ labels,
                   unsigned int* __restrict__ bad) {
  grid_dep_enter();
  __shared__ uint32_t speek[1 << kPeekBits];
  for (int i = threadIdx.x; i < (1 << kPeekBits); i += blockDim.x) speek[i] = peek[i];
  __syncthreads();
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nchunks;
       c += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t* src = payload + woff[c];
    const uint64_t nwords = woff[c + 1] - woff[c];
    const uint64_t nbits = 64 * nwords;
    const int64_t base = c * kHuffChunk;
    const int nc = static_cast<int>(min(int64_t(kHuffChunk), n - base));
    uint64_t pos = 0;
    bool ok = true;
    for (int i = 0; i < nc; ++i) {
      // Reading order: bit 0 of the fetched bits first, i.e. the code's most
      // significant bit; reversed, the first bits read sit at the top.
      const uint32_t head = __brev(static_cast<uint32_t>(bits_at(src, nwords, pos)));
      uint32_t sym = 0, len = 0;
      const uint32_t pk = speek[head >> (32 - kPeekBits)];
      if (pk) {
        sym = pk >> 8;
        len = pk & 0xFFu;
      } else {
        for (int L = kPeekBits + 1; L <= dt.maxlen; ++L) {
          const uint32_t code = head >> (32 - L);
          if (code - dt.first[L] < dt.count[L]) {
            sym = sorted[dt.offset[L] + (code - dt.first[L])];
            len = static_cast<uint32_t>(L);
            break;
          }
        }
      }
      if (len == 0 || pos + len > nbits) {
        ok = false;
        break;
      }
      pos += len;
      uint64_t z = sym;
      if (sym >= uint32_t(kHuffDirect)) {
        const uint32_t nx = sym - uint32_t(kHuffDirect) + 15;  // bit length - 1
        if (pos + nx > nbits) {
          ok = false;
          break;
        }
        z = (uint64_t(1) << nx) | (bits_at(src, nwords, pos) & ((uint64_t(1) << nx) - 1));
        pos += nx;
      }
      labels[base + i] = unzig(z);
    }
    if (!ok) atomicOr(bad, 1u);
  }
}

// ------------------------------------------------------------------ host

// Huffman code lengths with the fixed order and the 31-bit limit above.
void huff_lengths(std::vector<uint64_t> counts, std::vector<uint8_t>& len) {
  const int K = static_cast<int>(counts.size());
  len.assign(K, 0);
  for (;;) {
    std::vector<std::pair<uint64_t, int>> used;
    for (int s = 0; s < K; ++s)
      if (counts[s]) used.emplace_back(counts[s], s);
    std::fill(len.begin(), len.end(), 0);
    if (used.empty()) return;
    if (used.size() == 1) {
      len[used[0].second] = 1;
      return;
    }
    std::sort(used.begin(), used.end());
    const int m = static_cast<int>(used.size());
    // Nodes 0..m-1 are the sorted leaves, m.. the merged nodes.
    std::vector<uint64_t> w(2 * m - 1);
    std::vector<int> parent(2 * m - 1, -1);
    for (int i = 0; i < m; ++i) w[i] = used[i].first;
    int li = 0, mi = m, next = m;
    auto take = [&]() {
      if (mi >= next || (li < m && w[li] <= w[mi])) return li++;
      return mi++;
    };
    while ((m - li) + (next - mi) > 1) {
      const int a = take();
      const int b = take();
      w[next] = w[a] + w[b];
      parent[a] = parent[b] = next;
      ++next;
    }
    std::vector<int> depth(2 * m - 1, 0);
    for (int v = next - 2; v >= 0; --v) depth[v] = depth[parent[v]] + 1;
    int longest = 0;
    for (int i = 0; i < m; ++i) {
      len[used[i].second] = static_cast<uint8_t>(std::min(depth[i], 255));
      longest = std::max(longest, depth[i]);
    }
    if (longest <= kHuffMaxLen) return;
    for (auto& c : counts)
      if (c) c = std::max<uint64_t>(1, c / 2);
  }
}

// Canonical codes and the decoder's tables from the lengths.  Returns false
// if the lengths over-fill the code space (Kraft sum above 1).
bool huff_codes(const std::vector<uint8_t>& len, std::vector<uint64_t>& enc, DecTables& dt,
                std::vector<uint16_t>& sorted, std::vector<uint32_t>& peek) {
  const int K = static_cast<int>(len.size());
  std::vector<uint32_t> cnt(kHuffMaxLen + 2, 0);
  int maxlen = 0;
  for (int s = 0; s < K; ++s) {
    if (len[s] > kHuffMaxLen) return false;
    if (len[s]) {
      ++cnt[len[s]];
      maxlen = std::max<int>(maxlen, len[s]);
    }
  }
  // Kraft: sum 2^-L <= 1, in units of 2^-maxlen.
  uint64_t kraft = 0;
  for (int L = 1; L <= maxlen; ++L) kraft += uint64_t(cnt[L]) << (maxlen - L);
  if (maxlen && kraft > (uint64_t(1) << maxlen)) return false;
  std::memset(&dt, 0, sizeof dt);
  dt.maxlen = maxlen;
  uint32_t code = 0, off = 0;
  for (int L = 1; L <= kHuffMaxLen; ++L) {
    code = L == 1 ? 0 : (code + cnt[L - 1]) << 1;
    dt.first[L] = code;
    dt.count[L] = cnt[L];
    dt.offset[L] = off;
    off += cnt[L];
  }
  sorted.assign(off, 0);
  std::vector<uint32_t> fill(kHuffMaxLen + 2, 0);
  enc.assign(K, 0);
  // One pass in symbol order: within a length, codes go to the symbols in
  // increasing order.
  for (int s = 0; s < K; ++s) {
    const int L = len[s];
    if (L == 0) continue;
    const uint32_t c = dt.first[L] + fill[L];
    sorted[dt.offset[L] + fill[L]] = static_cast<uint16_t>(s);
    ++fill[L];
    enc[s] = (uint64_t(L) << 32) | c;
  }
  peek.assign(1u << kPeekBits, 0);
  for (int s = 0; s < K; ++s) {
    const int L = len[s];
    if (L == 0 || L > kPeekBits) continue;
    const uint32_t c = static_cast<uint32_t>(enc[s]);
    const uint32_t lo = c << (kPeekBits - L), span = 1u << (kPeekBits - L);
    for (uint32_t i = 0; i < span; ++i) peek[lo + i] = (uint32_t(s) << 8) | uint32_t(L);
  }
  return true;
}

// Offset of the chunk table (after the code lengths, 8-byte aligned) and
// of the payload.
constexpr size_t kTableOff = (kHeaderFixed + kHuffK + 7) / 8 * 8;
size_t header_bytes(int64_t n) {
  const int64_t nchunks = (n + kHuffChunk - 1) / kHuffChunk;
  return (kTableOff + 4 * static_cast<size_t>(nchunks) + 7) / 8 * 8;
}

// Device scratch of one call, freed on the stream at the end.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), s) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

#define HUFF_TRY(x)                               \
  do {                                            \
    if ((x) != cudaSuccess) return MGARD_ERR_CUDA; \
  } while (0)

int histogram(const int64_t* labels, int64_t n, Scratch& sc, std::vector<uint64_t>& h) {
  unsigned long long* hist = sc.get<unsigned long long>(kHuffK);
  if (!hist) return MGARD_ERR_CUDA;
  HUFF_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kHuffK, sc.s));
  if (n > 0)
    HUFF_TRY(launch_pdl(huff_hist_kernel, dim3(grid_for(n, 256 * 16)), dim3(256), 0, sc.s, labels, n, hist));
  h.assign(kHuffK, 0);
  HUFF_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(uint64_t) * kHuffK, cudaMemcpyDeviceToHost, sc.s));
  HUFF_TRY(cudaStreamSynchronize(sc.s));
  return MGARD_OK;
}

int encode(int64_t n, const int64_t* labels, uint8_t* out, size_t capacity, size_t* bytes_out,
           cudaStream_t s) {
  const size_t hdr = header_bytes(n);
  if (capacity < hdr) return MGARD_ERR_WORKSPACE;
  Scratch sc(s);
  std::vector<uint64_t> h;
  int rc = histogram(labels, n, sc, h);
  if (rc != MGARD_OK) return rc;
  std::vector<uint8_t> len;
  huff_lengths(h, len);
  std::vector<uint64_t> enc;
  std::vector<uint16_t> sorted;
  std::vector<uint32_t> peek;
  DecTables dt;
  if (!huff_codes(len, enc, dt, sorted, peek)) return MGARD_ERR_CUDA;  // cannot happen
  const int64_t nchunks = (n + kHuffChunk - 1) / kHuffChunk;
  std::vector<uint8_t> head(kTableOff, 0);
  const uint64_t N = static_cast<uint64_t>(n);
  const uint32_t K = kHuffK, ml = static_cast<uint32_t>(dt.maxlen);
  std::memcpy(head.data(), &N, 8);
  std::memcpy(head.data() + 8, &K, 4);
  std::memcpy(head.data() + 12, &ml, 4);
  std::memcpy(head.data() + kHeaderFixed, len.data(), kHuffK);
  uint64_t* d_enc = sc.get<uint64_t>(kHuffK);
  uint64_t* words = sc.get<uint64_t>(nchunks);
  uint64_t* tot = sc.get<uint64_t>(2);  // total words, largest chunk
  if (!d_enc || !words || !tot) return MGARD_ERR_CUDA;
  HUFF_TRY(cudaMemcpyAsync(d_enc, enc.data(), sizeof(uint64_t) * kHuffK, cudaMemcpyHostToDevice, s));
  HUFF_TRY(cudaMemcpyAsync(out, head.data(), head.size(), cudaMemcpyHostToDevice, s));
  const size_t pad0 = kTableOff + 4 * static_cast<size_t>(nchunks);
  if (hdr > pad0) HUFF_TRY(cudaMemsetAsync(out + pad0, 0, hdr - pad0, s));
  uint64_t totals[2] = {0, 0};
  if (nchunks > 0) {
    HUFF_TRY(cudaMemsetAsync(tot + 1, 0, sizeof(uint64_t), s));
    HUFF_TRY(launch_pdl(huff_sizes_kernel, dim3(grid_for(nchunks, 8)), dim3(256), 0, s, labels, n,
                        nchunks, static_cast<const uint64_t*>(d_enc), words,
                        reinterpret_cast<uint32_t*>(out + kTableOff),
                        reinterpret_cast<unsigned long long*>(tot + 1)));
    HUFF_TRY(launch_pdl(huff_scan_kernel, dim3(1), dim3(kScanT), 0, s, words, nchunks, tot));
    HUFF_TRY(cudaMemcpyAsync(totals, tot, sizeof totals, cudaMemcpyDeviceToHost, s));
    HUFF_TRY(cudaStreamSynchronize(s));
  }
  const size_t bytes = hdr + 8 * totals[0];
  if (bytes > capacity) return MGARD_ERR_WORKSPACE;
  if (nchunks > 0) {
    const int pitch = static_cast<int>(std::max<uint64_t>(1, totals[1]));  // <= kChunkWords
    const size_t smem = sizeof(uint64_t) * kEncWarps * static_cast<size_t>(pitch);
    HUFF_TRY(allow_dynamic_smem(huff_encode_kernel, smem));
    HUFF_TRY(launch_pdl(huff_encode_kernel, dim3(grid_for(nchunks, kEncWarps)), dim3(32 * kEncWarps),
                        smem, s, labels, n, nchunks, static_cast<const uint64_t*>(d_enc),
                        static_cast<const uint64_t*>(words), reinterpret_cast<uint64_t*>(out + hdr),
                        pitch));
  }
  HUFF_TRY(cudaGetLastError());
  *bytes_out = bytes;
  return MGARD_OK;
}

int decode(const uint8_t* in, size_t bytes, int64_t n, int64_t* labels, cudaStream_t s) {
  const size_t hdr = header_bytes(n);
  if (bytes < hdr) return MGARD_ERR_ARG;
  const int64_t nchunks = (n + kHuffChunk - 1) / kHuffChunk;
  std::vector<uint8_t> head(hdr);
  HUFF_TRY(cudaMemcpyAsync(head.data(), in, hdr, cudaMemcpyDeviceToHost, s));
  HUFF_TRY(cudaStreamSynchronize(s));
  uint64_t N = 0;
  uint32_t K = 0, ml = 0;
  std::memcpy(&N, head.data(), 8);
  std::memcpy(&K, head.data() + 8, 4);
  std::memcpy(&ml, head.data() + 12, 4);
  if (N != static_cast<uint64_t>(n) || K != uint32_t(kHuffK) || ml > uint32_t(kHuffMaxLen))
    return MGARD_ERR_ARG;
  std::vector<uint8_t> len(head.begin() + kHeaderFixed, head.begin() + kHeaderFixed + kHuffK);
  std::vector<uint64_t> enc;
  std::vector<uint16_t> sorted;
  std::vector<uint32_t> peek;
  DecTables dt;
  if (!huff_codes(len, enc, dt, sorted, peek) || dt.maxlen != static_cast<int>(ml)) return MGARD_ERR_ARG;
  // Chunk offsets on the host from the chunk table; the sizes must add up.
  std::vector<uint64_t> woff(nchunks + 1, 0);
  for (int64_t c = 0; c < nchunks; ++c) {
    uint32_t w = 0;
    std::memcpy(&w, head.data() + kTableOff + 4 * c, 4);
    if (w > uint32_t(kChunkWords)) return MGARD_ERR_ARG;
    woff[c + 1] = woff[c] + w;
  }
  if (bytes != hdr + 8 * woff[nchunks]) return MGARD_ERR_ARG;
  if (nchunks == 0) return MGARD_OK;
  Scratch sc(s);
  uint64_t* d_woff = sc.get<uint64_t>(nchunks + 1);
  uint32_t* d_peek = sc.get<uint32_t>(peek.size());
  uint16_t* d_sorted = sc.get<uint16_t>(sorted.size());
  unsigned int* d_bad = sc.get<unsigned int>(1);
  if (!d_woff || !d_peek || !d_sorted || !d_bad) return MGARD_ERR_CUDA;
  HUFF_TRY(cudaMemcpyAsync(d_woff, woff.data(), 8 * woff.size(), cudaMemcpyHostToDevice, s));
  HUFF_TRY(cudaMemcpyAsync(d_peek, peek.data(), 4 * peek.size(), cudaMemcpyHostToDevice, s));
  if (!sorted.empty())
    HUFF_TRY(cudaMemcpyAsync(d_sorted, sorted.data(), 2 * sorted.size(), cudaMemcpyHostToDevice, s));
  HUFF_TRY(cudaMemsetAsync(d_bad, 0, sizeof(unsigned), s));
  HUFF_TRY(launch_pdl(huff_decode_kernel, dim3(grid_for(nchunks, 128)), dim3(128), 0, s,
                      reinterpret_cast<const uint64_t*>(in + hdr), static_cast<const uint64_t*>(d_woff),
                      static_cast<const uint32_t*>(d_peek), static_cast<const uint16_t*>(d_sorted), dt, n,
                      nchunks, labels, d_bad));
  unsigned bad = 0;
  HUFF_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, s));
  HUFF_TRY(cudaStreamSynchronize(s));
  return bad ? MGARD_ERR_ARG : MGARD_OK;
}

int entropy(int64_t n, const int64_t* labels, double* out, cudaStream_t s) {
  if (n == 0) {
    *out = 0.0;
    return MGARD_OK;
  }
  Scratch sc(s);
  std::vector<uint64_t> h;
  int rc = histogram(labels, n, sc, h);
  if (rc != MGARD_OK) return rc;
  // Codes below 2^15 are counted by the histogram; the larger ones are
  // gathered and their distinct values counted on the host.
  uint64_t nlarge = 0;
  for (int sym = kHuffDirect; sym < kHuffK; ++sym) nlarge += h[sym];
  std::vector<uint64_t> counts(h.begin(), h.begin() + kHuffDirect);
  if (nlarge) {
    uint64_t* d_big = sc.get<uint64_t>(nlarge);
    unsigned long long* d_cnt = sc.get<unsigned long long>(1);
    if (!d_big || !d_cnt) return MGARD_ERR_CUDA;
    HUFF_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s));
    HUFF_TRY(launch_pdl(huff_large_codes_kernel, dim3(grid_for(n, 256 * 16)), dim3(256), 0, s, labels, n,
                        d_big, d_cnt, static_cast<unsigned long long>(nlarge)));
    std::vector<uint64_t> big(nlarge);
    HUFF_TRY(cudaMemcpyAsync(big.data(), d_big, 8 * nlarge, cudaMemcpyDeviceToHost, s));
    HUFF_TRY(cudaStreamSynchronize(s));
    std::sort(big.begin(), big.end());
    for (size_t i = 0; i < big.size();) {
      size_t j = i;
      while (j < big.size() && big[j] == big[i]) ++j;
      counts.push_back(j - i);
      i = j;
    }
  }
  // -sum p log2 p in a fixed order (codes ascending).
  const double N = static_cast<double>(n);
  double H = 0.0;
  for (uint64_t c : counts)
    if (c) {
      const double p = static_cast<double>(c) / N;
      H -= p * std::log2(p);
    }
  *out = H;
  return MGARD_OK;
}

}  // namespace
}  // namespace mgb

using namespace mgb;

extern "C" {

int mgard_huffman_bound(int64_t count, size_t* bytes) {
  if (count < 0 || bytes == nullptr) return MGARD_ERR_ARG;
  const int64_t nchunks = (count + kHuffChunk - 1) / kHuffChunk;
  // At most 31 code bits and 63 extra bits per label, rounded up per chunk.
  *bytes = header_bytes(count) + 8 * static_cast<size_t>(nchunks) +
           static_cast<size_t>((count * (kHuffMaxLen + 63) + 7) / 8);
  return MGARD_OK;
}

int mgard_huffman_encode(int64_t count, const int64_t* labels, void* out, size_t capacity,
                         size_t* bytes_out, void* stream) {
  if (count < 0 || bytes_out == nullptr || out == nullptr || reinterpret_cast<uintptr_t>(out) % 8 ||
      (count > 0 && (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8)))
    return MGARD_ERR_ARG;
  return encode(count, labels, static_cast<uint8_t*>(out), capacity, bytes_out,
                static_cast<cudaStream_t>(stream));
}

int mgard_huffman_decode(const void* in, size_t bytes, int64_t count, int64_t* labels, void* stream) {
  if (count < 0 || in == nullptr || reinterpret_cast<uintptr_t>(in) % 8 ||
      (count > 0 && (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8)))
    return MGARD_ERR_ARG;
  return decode(static_cast<const uint8_t*>(in), bytes, count, labels, static_cast<cudaStream_t>(stream));
}

int mgard_label_entropy(int64_t count, const int64_t* labels, double* bits_per_label, void* stream) {
  if (count < 0 || bits_per_label == nullptr ||
      (count > 0 && (labels == nullptr || reinterpret_cast<uintptr_t>(labels) % 8)))
    return MGARD_ERR_ARG;
  return entropy(count, labels, bits_per_label, static_cast<cudaStream_t>(stream));
}

int mgard_huffman_lengths(int nsym, const uint64_t* counts, uint8_t* lengths) {
  if (nsym < 0 || nsym > kHuffK || (nsym > 0 && (counts == nullptr || lengths == nullptr)))
    return MGARD_ERR_ARG;
  std::vector<uint8_t> len;
  huff_lengths(std::vector<uint64_t>(counts, counts + nsym), len);
  std::memcpy(lengths, len.data(), len.size());
  return MGARD_OK;
}

int mgard_cost_model(int ndim, const int64_t* dims, int stop_level, const double* tau_levels,
                     double range, double* bits) {
  if (tau_levels == nullptr || bits == nullptr || !(range > 0.0) || !std::isfinite(range))
    return MGARD_ERR_ARG;
  int L = 0;
  const int rc = count_levels(ndim, dims, &L);
  if (rc != MGARD_OK) return rc;
  if (stop_level < 0 || stop_level > L) return MGARD_ERR_LEVEL;
  for (int l = stop_level; l <= L; ++l)
    if (!(tau_levels[l] > 0.0) || !std::isfinite(tau_levels[l])) return MGARD_ERR_ARG;
  // Level shapes: every axis n -> n / 2 + 1 per level.
  std::vector<double> nodes(L + 1);
  std::vector<int64_t> cur(dims, dims + ndim);
  for (int l = L; l >= 0; --l) {
    double c = 1.0;
    for (int64_t v : cur) c *= static_cast<double>(v);
    nodes[l] = c;
    for (auto& v : cur) v = v / 2 + 1;
  }
  double cost = 0.0;
  for (int l = stop_level; l <= L; ++l) {
    const double cnt = l == stop_level ? nodes[l] : nodes[l] - nodes[l - 1];
    cost += cnt * std::log2(range / (2.0 * tau_levels[l]));
  }
  *bits = cost;
  return MGARD_OK;
}

}  // extern "C"
