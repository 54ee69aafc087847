// The labels' lossless stage (the last step of Algorithm 1): a chunked zigzag
// bit-packing coder, so that compressed labels, not 8-byte integers, cross
// between host and device.
//
// Stream layout (little-endian): uint64 N | one width byte per chunk of
// kPackChunk labels | zero padding to 8 bytes | per chunk, ceil(n_c w / 64)
// 64-bit words holding the chunk's zigzag codes (0, -1, 1, -2, .. -> 0, 1,
// 2, 3, ..) in w bits each, least significant bit first; w is the bit length
// of the chunk's largest code (0: all labels 0, no words).
//
// Encoding: one warp per chunk finds the width; one CTA scans the chunks'
// word counts into offsets; one warp per chunk writes its words (lane j
// assembles word j from the at most 64 / w + 1 codes that overlap it).
// Decoding: the same scan from the widths, then one thread per label.
#include <algorithm>
#include <cstdint>

#include "pdl.cuh"
#include "kernels.cuh"
#include "trace.hpp"

namespace mgb {
namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint64_t zigzag(int64_t k) {
  return (static_cast<uint64_t>(k) << 1) ^ static_cast<uint64_t>(k >> 63);
}
__device__ __forceinline__ int64_t unzigzag(uint64_t z) {
  return static_cast<int64_t>(z >> 1) ^ -static_cast<int64_t>(z & 1);
}
__device__ __forceinline__ uint64_t low_mask(int w) { return w >= 64 ? ~0ull : ((1ull << w) - 1); }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__global__ void __launch_bounds__(256)
pack_widths_kernel(const int64_t* __restrict__ labels, int64_t n, int64_t nchunks,
                   uint8_t* __restrict__ widths, uint64_t* __restrict__ words) {
  grid_dep_enter();
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t c = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks;
       c += warps) {
    const int64_t base = c * kPackChunk;
    const int nc = static_cast<int>(min64(kPackChunk, n - base));
    uint64_t zmax = 0;
    for (int i = lane; i < nc; i += 32) zmax = max(zmax, zigzag(labels[base + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zmax = max(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    if (lane == 0) {
      const int w = zmax ? 64 - __clzll(static_cast<long long>(zmax)) : 0;
      widths[c] = static_cast<uint8_t>(w);
      words[c] = (static_cast<uint64_t>(nc) * w + 63) / 64;
    }
  }
}

// Word counts of the chunks from their widths (decoding side).
__global__ void __launch_bounds__(256)
unpack_words_kernel(const uint8_t* __restrict__ widths, int64_t n, int64_t nchunks,
                    uint64_t* __restrict__ words) {
  grid_dep_enter();
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < nchunks;
       c += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t nc = static_cast<uint64_t>(min64(kPackChunk, n - c * kPackChunk));
    words[c] = (nc * widths[c] + 63) / 64;
  }
}

// Exclusive prefix sum of words[0..nchunks) in place, in one CTA (each
// thread a contiguous run, then a scan of the run totals); total[0] gets
// the sum.
__global__ void __launch_bounds__(kScanThreads)
scan_words_kernel(uint64_t* __restrict__ words, int64_t nchunks, uint64_t* __restrict__ total) {
  grid_dep_enter();
  __shared__ uint64_t s[kScanThreads];
  const int t = threadIdx.x;
  const int64_t per = (nchunks + kScanThreads - 1) / kScanThreads;
  const int64_t lo = min64(nchunks, t * per), hi = min64(nchunks, lo + per);
  uint64_t run = 0;
  for (int64_t c = lo; c < hi; ++c) run += words[c];
  s[t] = run;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const uint64_t add = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  uint64_t acc = s[t] - run;  // exclusive
  for (int64_t c = lo; c < hi; ++c) {
    const uint64_t w = words[c];
    words[c] = acc;
    acc += w;
  }
  if (t == kScanThreads - 1) total[0] = s[t];
}

__global__ void __launch_bounds__(256)
pack_payload_kernel(const int64_t* __restrict__ labels, int64_t n, int64_t nchunks,
                    const uint8_t* __restrict__ widths, const uint64_t* __restrict__ offsets,
                    uint64_t* __restrict__ payload) {
  grid_dep_enter();
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t c = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks;
       c += warps) {
    const int w = widths[c];
    if (w == 0) continue;
    const int64_t base = c * kPackChunk;
    const int nc = static_cast<int>(min64(kPackChunk, n - base));
    const int64_t nwords = (static_cast<int64_t>(nc) * w + 63) / 64;
    const uint64_t mask = low_mask(w);
    uint64_t* dst = payload + offsets[c];
    for (int64_t j = lane; j < nwords; j += 32) {
      const int64_t lo = 64 * j;
      const int i0 = static_cast<int>(lo / w);
      const int i1 = static_cast<int>(min64(nc - 1, (lo + 63) / w));
      uint64_t word = 0;
      for (int i = i0; i <= i1; ++i) {
        const uint64_t z = zigzag(labels[base + i]) & mask;
        const int64_t b = static_cast<int64_t>(i) * w;
        word |= b >= lo ? z << (b - lo) : z >> (lo - b);
      }
      dst[j] = word;
    }
  }
}

__global__ void __launch_bounds__(256)
unpack_payload_kernel(const uint64_t* __restrict__ payload, const uint8_t* __restrict__ widths,
                      const uint64_t* __restrict__ offsets, int64_t n, int64_t* __restrict__ labels) {
  grid_dep_enter();
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = t / kPackChunk;
    const int i = static_cast<int>(t - c * kPackChunk);
    const int w = widths[c];
    uint64_t z = 0;
    if (w) {
      const int64_t b = static_cast<int64_t>(i) * w;
      const uint64_t* src = payload + offsets[c] + (b >> 6);
      const int sh = static_cast<int>(b & 63);
      z = src[0] >> sh;
      if (sh + w > 64) z |= src[1] << (64 - sh);
      z &= low_mask(w);
    }
    labels[t] = unzigzag(z);
  }
}

__global__ void write_count_kernel(uint64_t* __restrict__ head, int64_t n) {
  grid_dep_enter();
  head[0] = static_cast<uint64_t>(n);
}

unsigned warp_grid(int64_t nchunks) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(8 * 152 * 8, (nchunks + 7) / 8)));
}

}  // namespace

size_t pack_header_bytes(int64_t n) {
  const int64_t nchunks = (n + kPackChunk - 1) / kPackChunk;
  return static_cast<size_t>((8 + nchunks + 7) / 8 * 8);
}

cudaError_t launch_pack_labels(const int64_t* labels, int64_t n, uint8_t* out, uint64_t* words,
                               uint64_t* total_words, cudaStream_t s) {
  const int64_t nchunks = (n + kPackChunk - 1) / kPackChunk;
  const size_t hdr = pack_header_bytes(n);
  TraceScope ts(kKPack, -1, 8.0 * double(n), s);
  ts.more_kernels(nchunks > 0 ? 3 : 0);
  launch_pdl(write_count_kernel, dim3(1), dim3(1), 0, s, reinterpret_cast<uint64_t*>(out), n);
  if (hdr > 8) cudaMemsetAsync(out + 8, 0, hdr - 8, s);
  if (nchunks == 0) return cudaMemsetAsync(total_words, 0, sizeof(uint64_t), s);
  launch_pdl(pack_widths_kernel, dim3(warp_grid(nchunks)), dim3(256), 0, s, labels, n, nchunks,
             out + 8, words);
  launch_pdl(scan_words_kernel, dim3(1), dim3(kScanThreads), 0, s, words, nchunks, total_words);
  launch_pdl(pack_payload_kernel, dim3(warp_grid(nchunks)), dim3(256), 0, s, labels, n, nchunks,
             static_cast<const uint8_t*>(out + 8), static_cast<const uint64_t*>(words),
             reinterpret_cast<uint64_t*>(out + hdr));
  return cudaGetLastError();
}

cudaError_t launch_unpack_labels(const uint8_t* in, int64_t n, uint64_t* words, uint64_t* total_words,
                                 int64_t* labels, cudaStream_t s) {
  const int64_t nchunks = (n + kPackChunk - 1) / kPackChunk;
  if (nchunks == 0) return cudaSuccess;
  const size_t hdr = pack_header_bytes(n);
  TraceScope ts(kKUnpack, -1, 8.0 * double(n), s);
  ts.more_kernels(2);
  const unsigned g = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(8 * 152, (nchunks + 255) / 256)));
  launch_pdl(unpack_words_kernel, dim3(g), dim3(256), 0, s, in + 8, n, nchunks, words);
  launch_pdl(scan_words_kernel, dim3(1), dim3(kScanThreads), 0, s, words, nchunks, total_words);
  const unsigned gl = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(16 * 152 * 8, (n + 255) / 256)));
  launch_pdl(unpack_payload_kernel, dim3(gl), dim3(256), 0, s,
             reinterpret_cast<const uint64_t*>(in + hdr), in + 8,
             static_cast<const uint64_t*>(words), n, labels);
  return cudaGetLastError();
}

}  // namespace mgb
