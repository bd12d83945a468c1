// A1 / A3 / A4: hash join build and probe, and late materialisation by row id
// (Sec. 3.2.2 join and materialisation operators; Sec. 4.2: joins dominate query time).
//
// Table layout in caller memory: a 256-byte header (has_dups flag, status) followed by
// `capacity` slots.  4-byte keys: one uint64 slot = key (low word) | payload << 32.
// 8-byte keys: a 16-byte slot {uint64 key, uint32 payload, uint32 pad}.  A slot is empty when
// its payload is 0xFFFFFFFF, which no row id takes (row counts stay below 2^32 - 1), so every
// key value -- including all-ones -- can be stored.  Inserts walk linearly from the key's home
// slot and claim the first empty slot with a single compare-and-swap of the whole slot; a walk
// that passes a slot holding the same key records a duplicate.  Two inserts of equal keys walk
// the same sequence, so the later one always passes the earlier one's slot: the flag is exact.
#include "tables.cuh"

namespace sirius {
namespace {

constexpr int kThreads = 256;

__global__ void join_build32_kernel(const int32_t* __restrict__ keys, int64_t m,
                                    uint64_t* __restrict__ slots, uint32_t cap, JoinHeader* hdr) {
  bool dup = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = (uint32_t)keys[j];
    const uint64_t desired = (uint64_t)key | ((uint64_t)(uint32_t)j << 32);
    if (!join_insert32(slots, cap, key, desired, dup)) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) hdr->has_dups = 1;
}

__global__ void join_build64_kernel(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                    int64_t m, ulonglong2* __restrict__ slots, uint32_t cap,
                                    JoinHeader* hdr) {
  bool dup = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = pack_key64(hi[j], lo[j]);
    if (!join_insert64(slots, cap, key, (uint32_t)j, dup)) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) hdr->has_dups = 1;
}

// Probe: one probe row per lane per round; a round ends when every lane of the warp has
// finished its walk.  Matches are appended with one atomic per warp and step.
template <bool kWide>
__global__ void __launch_bounds__(kThreads)
join_probe_kernel(const void* __restrict__ slots_v, uint32_t cap, const JoinHeader* __restrict__ hdr,
                  const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                  const uint32_t* __restrict__ sel, int64_t n, uint32_t* __restrict__ out_probe,
                  uint32_t* __restrict__ out_build, int64_t out_cap,
                  unsigned long long* __restrict__ counter) {
  const bool dups = hdr->has_dups != 0;
  const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)(kThreads / 32) + (threadIdx.x >> 5); w * 32 < n; w += warps) {
    const int64_t i = w * 32 + lane;
    bool walking = i < n;
    uint32_t row = 0, s = 0;
    uint64_t key = 0;
    if (walking) {
      row = sel ? sel[i] : (uint32_t)i;
      key = kWide ? pack_key64(hi[row], lo[row]) : (uint64_t)(uint32_t)lo[row];
      s = kWide ? home_slot64(key, cap) : home_slot32((uint32_t)key, cap);
    }
    uint32_t steps = 0;
    while (__any_sync(0xffffffffu, walking)) {
      bool match = false;
      uint32_t payload = kEmpty32;
      if (walking) {
        uint64_t skey;
        if (kWide) {
          const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(slots_v) + s);
          skey = v.x;
          payload = (uint32_t)v.y;
        } else {
          const uint64_t v = __ldg(reinterpret_cast<const uint64_t*>(slots_v) + s);
          skey = (uint32_t)v;
          payload = (uint32_t)(v >> 32);
        }
        if (payload == kEmpty32 || ++steps > cap) {
          walking = false;
        } else {
          match = skey == key;
          if (match && !dups) walking = false;
          s = (s + 1 == cap) ? 0 : s + 1;
        }
      }
      const uint64_t pos = warp_append(counter, match);
      if (match && (int64_t)pos < out_cap) {
        out_probe[pos] = row;
        out_build[pos] = payload;
      }
    }
  }
}

template <typename T>
__global__ void gather_kernel(const T* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n,
                              T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void gather_group_key_kernel(const int32_t* __restrict__ grp, const int8_t* __restrict__ flag,
                                        const uint32_t* __restrict__ idx, int64_t n,
                                        int64_t* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = idx[i];
    dst[i] = group_key(grp[r], flag, r);
  }
}

}  // namespace

int grid_for(int64_t n, int threads) {
  const int64_t want = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

sirius_status join_build(const int32_t* lo, const int32_t* hi, int64_t m, void* mem, int64_t capacity,
                         cudaStream_t s, bool clear) {
  JoinHeader* hdr = (JoinHeader*)mem;
  void* slots = (char*)mem + 256;
  const size_t slot_bytes = hi ? 16 : 8;
  if (clear) SIRIUS_CUDA_TRY(cudaMemsetAsync(mem, 0, 256, s));
  if (clear) SIRIUS_CUDA_TRY(cudaMemsetAsync(slots, 0xFF, (size_t)capacity * slot_bytes, s));
  if (m == 0) return SIRIUS_OK;
  const int g = grid_for(m, kThreads);
  PhaseTimer pt(s, SIRIUS_PHASE_JOIN_BUILD);
  if (hi)
    join_build64_kernel<<<g, kThreads, 0, s>>>(lo, hi, m, (ulonglong2*)slots, (uint32_t)capacity, hdr);
  else
    join_build32_kernel<<<g, kThreads, 0, s>>>(lo, m, (uint64_t*)slots, (uint32_t)capacity, hdr);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

}  // namespace sirius

using namespace sirius;

extern "C" int64_t sirius_join_table_capacity(int64_t m, double load_factor) {
  if (m < 0) return 0;
  if (!(load_factor > 0.0) || load_factor > 0.95) load_factor = 0.5;
  int64_t c = (int64_t)((double)m / load_factor) + 1;
  if (c <= m) c = m + 1;
  if (c < 16) c = 16;
  return (c + 3) & ~(int64_t)3;  // whole 32-byte buckets
}

extern "C" size_t sirius_join_table_bytes(int64_t capacity, int32_t key_width) {
  if (capacity <= 0 || (key_width != 4 && key_width != 8)) return 0;
  return 256 + (size_t)capacity * (key_width == 8 ? 16 : 8);
}

extern "C" sirius_status sirius_hash_join_build(const int32_t* d_keys, const int32_t* d_keys_hi,
                                                int64_t m, sirius_join_table* table,
                                                int32_t* h_has_dups, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(table && table->d_mem, "join build: NULL table");
  SIRIUS_REQUIRE(table->key_width == (d_keys_hi ? 8 : 4),
                 "join build: key_width %d does not match the key columns", table->key_width);
  SIRIUS_REQUIRE(m >= 0 && m <= kMaxRows && m < table->capacity && table->capacity < (1ll << 32),
                 "join build: m=%lld needs capacity > m (< 2^32), have %lld", (long long)m,
                 (long long)table->capacity);
  SIRIUS_REQUIRE(table->capacity % 4 == 0, "join build: capacity must be a multiple of 4");
  SIRIUS_REQUIRE(m == 0 || d_keys, "join build: NULL keys");
  SIRIUS_REQUIRE(((uintptr_t)table->d_mem & 255) == 0, "join build: table memory must be 256-byte aligned");
  sirius_status st = join_build(d_keys, d_keys_hi, m, table->d_mem, table->capacity, s, true);
  if (st != SIRIUS_OK) return st;
  if (h_has_dups) {
    JoinHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, table->d_mem, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_has_dups = h.has_dups ? 1 : 0;
    if (h.status) {
      set_error("join build: device status %d", h.status);
      return (sirius_status)h.status;
    }
  }
  return SIRIUS_OK;
}

extern "C" sirius_status sirius_hash_join_probe(const sirius_join_table* table, const int32_t* d_keys,
                                                const int32_t* d_keys_hi, const uint32_t* d_sel,
                                                int64_t n, uint32_t* d_out_probe,
                                                uint32_t* d_out_build, int64_t out_cap,
                                                int64_t* d_out_count, int64_t* h_out_count,
                                                sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(table && table->d_mem, "join probe: NULL table");
  SIRIUS_REQUIRE(table->key_width == (d_keys_hi ? 8 : 4), "join probe: key width mismatch");
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "join probe: n=%lld out of range", (long long)n);
  SIRIUS_REQUIRE(out_cap >= 0 && (out_cap == 0 || (d_out_probe && d_out_build)),
                 "join probe: NULL outputs");
  SIRIUS_REQUIRE(n == 0 || d_keys, "join probe: NULL keys");
  SIRIUS_REQUIRE(d_out_count || h_out_count, "join probe: no place for the pair count");
  // the pair counter lives in the table header's spare word (reset here, stream-ordered)
  JoinHeader* hdr = (JoinHeader*)table->d_mem;
  unsigned long long* counter = (unsigned long long*)&hdr->pairs;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(counter, 0, 8, s));
  if (n > 0) {
    const int g = grid_for((n + 31) / 32 * 32, kThreads);
    const void* slots = (const char*)table->d_mem + 256;
    PhaseTimer pt(s, SIRIUS_PHASE_JOIN_PROBE);
    if (d_keys_hi)
      join_probe_kernel<true><<<g, kThreads, 0, s>>>(slots, (uint32_t)table->capacity, hdr, d_keys,
                                                     d_keys_hi, d_sel, n, d_out_probe, d_out_build,
                                                     out_cap, counter);
    else
      join_probe_kernel<false><<<g, kThreads, 0, s>>>(slots, (uint32_t)table->capacity, hdr, d_keys,
                                                      nullptr, d_sel, n, d_out_probe, d_out_build,
                                                      out_cap, counter);
    SIRIUS_LAUNCH_CHECK();
  }
  if (d_out_count)
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(d_out_count, counter, 8, cudaMemcpyDeviceToDevice, s));
  if (h_out_count) {
    unsigned long long c = 0;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&c, counter, 8, cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_out_count = (int64_t)c;
    if ((int64_t)c > out_cap) {
      set_error("join probe: %llu pairs exceed out_cap %lld", c, (long long)out_cap);
      return SIRIUS_ERR_CAPACITY;
    }
  }
  return SIRIUS_OK;
}

template <typename T>
static sirius_status gather_any(const T* src, const uint32_t* idx, int64_t n, T* dst, cudaStream_t s) {
  clear_error();
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "gather: n out of range");
  SIRIUS_REQUIRE(n == 0 || (src && idx && dst), "gather: NULL pointer");
  if (n == 0) return SIRIUS_OK;
  PhaseTimer pt(s, SIRIUS_PHASE_GATHER);
  gather_kernel<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(src, idx, n, dst);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

extern "C" sirius_status sirius_gather_i32(const int32_t* d_src, const uint32_t* d_idx, int64_t n,
                                           int32_t* d_dst, sirius_stream stream) {
  return gather_any<int32_t>(d_src, d_idx, n, d_dst, (cudaStream_t)stream);
}

extern "C" sirius_status sirius_gather_i64(const int64_t* d_src, const uint32_t* d_idx, int64_t n,
                                           int64_t* d_dst, sirius_stream stream) {
  return gather_any<int64_t>(d_src, d_idx, n, d_dst, (cudaStream_t)stream);
}

extern "C" sirius_status sirius_gather_group_key(const int32_t* d_grp, const int8_t* d_flag,
                                                 const uint32_t* d_idx, int64_t n, int64_t* d_dst,
                                                 sirius_stream stream) {
  clear_error();
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "gather_group_key: n out of range");
  SIRIUS_REQUIRE(n == 0 || (d_grp && d_idx && d_dst), "gather_group_key: NULL pointer");
  if (n == 0) return SIRIUS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  gather_group_key_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(d_grp, d_flag, d_idx, n, d_dst);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}
