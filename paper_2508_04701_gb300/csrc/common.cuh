// Shared device/host helpers of libsirius (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>
#include <atomic>
#include <stdint.h>
#include <string.h>

#include "../../include/sirius.h"

namespace sirius {

// ------------------------------------------------------------------ host-side error state
void set_error(const char* fmt, ...);
void clear_error();
void count_launch(int k = 1);
void set_launch_counting(bool on);  // off while a CUDA graph is captured: replays count instead
int sm_count();

// Phase timing (see sirius_profile_start): records a CUDA event pair around a scope when on.
struct PhaseTimer {
  int phase;
  cudaStream_t stream;
  void* a = nullptr;
  PhaseTimer(cudaStream_t s, int p);
  ~PhaseTimer();
};

#define SIRIUS_CUDA_TRY(expr)                                                             \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) {                                                              \
      ::sirius::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),       \
                          __FILE__, __LINE__);                                            \
      return SIRIUS_ERR_CUDA;                                                             \
    }                                                                                     \
  } while (0)

#define SIRIUS_LAUNCH_CHECK()                                                             \
  do {                                                                                    \
    ::sirius::count_launch();                                                             \
    cudaError_t _e = cudaGetLastError();                                                  \
    if (_e != cudaSuccess) {                                                              \
      ::sirius::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e),    \
                          __FILE__, __LINE__);                                            \
      return SIRIUS_ERR_CUDA;                                                             \
    }                                                                                     \
  } while (0)

#define SIRIUS_REQUIRE(cond, ...)                                                         \
  do {                                                                                    \
    if (!(cond)) {                                                                        \
      ::sirius::set_error(__VA_ARGS__);                                                   \
      return SIRIUS_ERR_INVALID;                                                          \
    }                                                                                     \
  } while (0)

constexpr int64_t kMaxRows = 0xFFFFFFFELL;  // row ids are uint32; 0xFFFFFFFF marks "empty"
constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;
constexpr uint64_t kEmpty64 = 0xFFFFFFFFFFFFFFFFull;
constexpr int64_t kEmptyKey = INT64_MIN;     // empty slot of a group table

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Raises a kernel's dynamic shared-memory limit once per device (one bit per device ordinal in
// `done`; two threads racing on a device's first call both set it, which is harmless).
template <typename K>
inline cudaError_t ensure_smem_limit(K kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Scratch handed to a call: either the caller's buffer or one allocated stream-ordered.
struct Scratch {
  char* base = nullptr;
  size_t bytes = 0;
  bool owned = false;
  cudaStream_t stream = nullptr;
  size_t used = 0;
  sirius_status acquire(void* d_scratch, size_t have, size_t need, cudaStream_t s);
  void* take(size_t n) {  // 256-byte aligned bump allocation inside the scratch
    size_t off = align_up(used, 256);
    used = off + n;
    return base + off;
  }
  ~Scratch();
};

// Device status word: the first error wins.
struct DevHeader {
  int32_t status;
  uint32_t has_dups;
  uint64_t count;        // filter: selected rows; probe: pairs; group-by: G
  uint64_t distinct;     // group-table slots claimed
  uint64_t counter;      // tile ticket (filter look-back)
  uint64_t pad[4];
};
static_assert(sizeof(DevHeader) <= 256, "header fits its 256-byte slot");

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ hashing
// Finalizers of MurmurHash3 (Austin Appleby, public domain): full avalanche on 32/64 bits.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}
// Map a 32-bit hash onto [0, cap) by a multiply-high (Lemire's range reduction).
__host__ __device__ __forceinline__ uint32_t reduce_range(uint32_t h, uint32_t cap) {
  return (uint32_t)(((uint64_t)h * (uint64_t)cap) >> 32);
}
// Home slots start a 32-byte bucket (one DRAM sector): four 8-byte slots or two 16-byte slots.
// Probing stays plain linear probing from the home slot; a probe just reads a whole bucket per
// load.  Join-table capacities are multiples of 4.
__host__ __device__ __forceinline__ uint32_t home_slot32(uint32_t key, uint32_t cap) {
  return reduce_range(fmix32(key), cap >> 2) << 2;
}
__host__ __device__ __forceinline__ uint32_t home_slot64(uint64_t key, uint32_t cap) {
  return reduce_range((uint32_t)(fmix64(key) >> 32), cap >> 1) << 1;
}

// 32-byte read-only load (a whole bucket); the address must be 32-byte aligned.
__device__ __forceinline__ void ldg_bucket(const void* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
// The same load through L2 only (no L1 or read-only cache): for tables written earlier in the
// same launch by other blocks, which the non-coherent path may not see.
__device__ __forceinline__ void ldcg_bucket(const void* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
  asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
__host__ __device__ __forceinline__ uint64_t pack_key64(int32_t hi, int32_t lo) {
  return ((uint64_t)(uint32_t)hi << 32) | (uint64_t)(uint32_t)lo;
}
__host__ __device__ __forceinline__ int64_t group_key(int32_t grp, const int8_t* flag, int64_t row) {
  return flag ? (int64_t)grp * 256 + (int64_t)(uint8_t)flag[row] : (int64_t)grp;
}

// ------------------------------------------------------------------ predicates
__device__ __forceinline__ bool cmp_op(int32_t v, int32_t lit, int op) {
  switch (op) {
    case SIRIUS_LT: return v < lit;
    case SIRIUS_LE: return v <= lit;
    case SIRIUS_GT: return v > lit;
    case SIRIUS_GE: return v >= lit;
    case SIRIUS_EQ: return v == lit;
    default: return v != lit;
  }
}

// ------------------------------------------------------------------ memory helpers
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  return cuda::atomic_ref<uint64_t, cuda::thread_scope_device>(*const_cast<uint64_t*>(p))
      .load(cuda::memory_order_relaxed);
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  cuda::atomic_ref<uint64_t, cuda::thread_scope_device>(*p).store(v, cuda::memory_order_relaxed);
}

// 128-bit compare-and-swap (sm_90+): returns the previous 16 bytes at p.
__device__ __forceinline__ void cas128(unsigned long long* p, unsigned long long cmp_lo,
                                       unsigned long long cmp_hi, unsigned long long new_lo,
                                       unsigned long long new_hi, unsigned long long& old_lo,
                                       unsigned long long& old_hi) {
  asm volatile(
      "{\n\t.reg .b128 c, n, o;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 n, {%4, %5};\n\t"
      "atom.global.cas.b128 o, [%6], c, n;\n\t"
      "mov.b128 {%0, %1}, o;\n\t}"
      : "=l"(old_lo), "=l"(old_hi)
      : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
      : "memory");
}

// ------------------------------------------------------------------ async copies (sm_90+)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy accesses to shared memory before later async-proxy
// (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// One-dimensional TMA bulk copy global -> this CTA's shared memory; completion is counted in
// bytes on `bar`.  Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bounded wait for phase `parity` of `bar`; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_tries) {
  for (int i = 0; i < max_tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 16-byte asynchronous copy global -> shared through L2 only (Ampere-style cp.async).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Minimum / maximum of a 64-bit value over the full warp (every lane gets the result).
__device__ __forceinline__ long long warp_min_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  return v;
}
__device__ __forceinline__ long long warp_max_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Warp-aggregated append: every lane with `want` gets a distinct index from *counter.
__device__ __forceinline__ uint64_t warp_append(unsigned long long* counter, bool want) {
  unsigned mask = __ballot_sync(0xffffffffu, want);
  int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  int leader = mask ? __ffs(mask) - 1 : 0;
  if (mask && lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + __popc(mask & lanemask_lt());
}

}  // namespace sirius
