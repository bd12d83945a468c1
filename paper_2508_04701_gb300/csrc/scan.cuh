// Exclusive scan of m 32-bit counts in place over several blocks (three launches: the sums of
// segments of kScanSeg entries, their scan in one block, then each segment scanned from its
// base).  The total goes to *total (nullable, device).  Scratch: scan_part_entries(m) 64-bit
// partial sums.
#pragma once
#include "tables.cuh"

namespace sirius {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanSeg = 4096;  // entries per block: 4 per thread

inline int64_t scan_part_entries(int64_t m) { return (m + kScanSeg - 1) / kScanSeg; }

__global__ void __launch_bounds__(kScanThreads)
scan_partials_kernel(const uint32_t* a, int64_t m, unsigned long long* part) {
  __shared__ unsigned long long s[kScanThreads / 32];
  unsigned long long acc = 0;
  const int64_t base = (int64_t)blockIdx.x * kScanSeg;
  for (int64_t i = base + threadIdx.x; i < base + kScanSeg && i < m; i += blockDim.x) acc += a[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanThreads)
scan_top_kernel(unsigned long long* part, int64_t nb, unsigned long long* total) {
  __shared__ unsigned long long s[kScanThreads];
  unsigned long long carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int64_t i = b0 + threadIdx.x;
    const unsigned long long v = i < nb ? part[i] : 0ull;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
      const unsigned long long x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
      __syncthreads();
      s[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) part[i] = carry + s[threadIdx.x] - v;  // exclusive
    const unsigned long long blk = s[kScanThreads - 1];
    __syncthreads();
    carry += blk;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(uint32_t* a, int64_t m, const unsigned long long* part) {
  __shared__ unsigned long long s[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * 4;
  uint32_t v[4];
  unsigned long long loc = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < m ? a[base + j] : 0u;
    loc += v[j];
  }
  s[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const unsigned long long x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  unsigned long long run = part[blockIdx.x] + s[threadIdx.x] - loc;
  for (int j = 0; j < 4; ++j) {
    if (base + j < m) a[base + j] = (uint32_t)run;  // prefixes stay below 2^32 (they count rows)
    run += v[j];
  }
}

inline sirius_status exclusive_scan_u32(uint32_t* a, int64_t m, unsigned long long* part,
                                        unsigned long long* total, cudaStream_t s) {
  const int64_t nb = scan_part_entries(m > 0 ? m : 1);
  scan_partials_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(a, m, part);
  SIRIUS_LAUNCH_CHECK();
  scan_top_kernel<<<1, kScanThreads, 0, s>>>(part, nb, total);
  SIRIUS_LAUNCH_CHECK();
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(a, m, part);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

}  // namespace
}  // namespace sirius
