// CUDA twin of the seeded input generator (paper_2508_04701_gb300/datagen.py): SplitMix64
// streams, bounded integers by multiply-high, Zipf ranks by binary search of a host-built CDF.
// Input recipe only -- no filter / join / group-by arithmetic.  Built as its own library,
// libsirius_datagen.so.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t elem(uint64_t base, int64_t i) {
  return mix64(base + (uint64_t)(i + 1) * kGamma);
}
__device__ __forceinline__ uint64_t bounded(uint64_t r, uint64_t n) { return __umul64hi(r, n); }

__global__ void stream_u64(uint64_t base, int64_t i0, int64_t n, uint64_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = elem(base, i0 + i);
}
__global__ void bounded_i32(uint64_t base, int64_t i0, int64_t n, uint64_t bound, int32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)bounded(elem(base, i0 + i), bound);
}
__global__ void bounded_i64(uint64_t base, int64_t i0, int64_t n, uint64_t bound, int64_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)bounded(elem(base, i0 + i), bound);
}
// rank0 = first k with cdf[k] > u (cdf[m-1] == 1 > u); out = src[rank0]
__global__ void zipf_gather(uint64_t base, int64_t i0, int64_t n, const double* cdf, int64_t m,
                            const int32_t* src, int32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(elem(base, i0 + i) >> 11) * 0x1.0p-53;
    int64_t lo = 0, hi = m - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    out[i] = src[lo];
  }
}
__global__ void composite_bounded(uint64_t base, int64_t i0, int64_t n, uint64_t bound, uint64_t salt,
                                  int32_t* lo, int32_t* hi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = mix64(bounded(elem(base, i0 + i), bound) ^ salt);
    lo[i] = (int32_t)(uint32_t)k;
    hi[i] = (int32_t)(uint32_t)(k >> 32);
  }
}
__global__ void composite_of(const int64_t* v, int64_t n, uint64_t salt, int32_t* lo, int32_t* hi) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = mix64((uint64_t)v[i] ^ salt);
    lo[i] = (int32_t)(uint32_t)k;
    hi[i] = (int32_t)(uint32_t)(k >> 32);
  }
}

int grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

extern "C" {
int dg_stream_u64(uint64_t base, int64_t i0, int64_t n, void* out, void* s) {
  stream_u64<<<grid(n), 256, 0, (cudaStream_t)s>>>(base, i0, n, (uint64_t*)out);
  return (int)cudaGetLastError();
}
int dg_bounded_i32(uint64_t base, int64_t i0, int64_t n, uint64_t bound, void* out, void* s) {
  bounded_i32<<<grid(n), 256, 0, (cudaStream_t)s>>>(base, i0, n, bound, (int32_t*)out);
  return (int)cudaGetLastError();
}
int dg_bounded_i64(uint64_t base, int64_t i0, int64_t n, uint64_t bound, void* out, void* s) {
  bounded_i64<<<grid(n), 256, 0, (cudaStream_t)s>>>(base, i0, n, bound, (int64_t*)out);
  return (int)cudaGetLastError();
}
int dg_zipf_gather_i32(uint64_t base, int64_t i0, int64_t n, void* cdf, int64_t m, void* src, void* out, void* s) {
  zipf_gather<<<grid(n), 256, 0, (cudaStream_t)s>>>(base, i0, n, (const double*)cdf, m, (const int32_t*)src,
                                                   (int32_t*)out);
  return (int)cudaGetLastError();
}
int dg_composite_bounded(uint64_t base, int64_t i0, int64_t n, uint64_t bound, uint64_t salt, void* lo, void* hi,
                         void* s) {
  composite_bounded<<<grid(n), 256, 0, (cudaStream_t)s>>>(base, i0, n, bound, salt, (int32_t*)lo, (int32_t*)hi);
  return (int)cudaGetLastError();
}
int dg_composite_of(void* v, int64_t n, uint64_t salt, void* lo, void* hi, void* s) {
  composite_of<<<grid(n), 256, 0, (cudaStream_t)s>>>((const int64_t*)v, n, salt, (int32_t*)lo, (int32_t*)hi);
  return (int)cudaGetLastError();
}
}
