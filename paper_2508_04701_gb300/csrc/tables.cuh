// Open-addressing hash tables of libsirius: the join table (key -> payload, a multimap) and the
// group table (distinct key -> slot of its aggregates).  Device-side insert routines shared by
// the stand-alone operators and the fused pipeline.
#pragma once

#include "common.cuh"

namespace sirius {

// 256-byte header in front of a join table's slots.
struct JoinHeader {
  uint32_t has_dups;   // some key was inserted twice
  int32_t status;      // first device error of the build
  uint64_t pairs;      // pair counter of the stand-alone probe
  uint64_t pad[30];
};
static_assert(sizeof(JoinHeader) == 256, "join header is 256 bytes");

// Insert (key -> payload) into a table of 8-byte slots {key low word, payload high word}.
// The slot word is read with one aligned 64-bit load; a stale "empty" is settled by the CAS,
// and an occupied slot never becomes empty again during a build.
__device__ __forceinline__ bool join_insert32(uint64_t* slots, uint32_t cap, uint32_t key,
                                              uint64_t desired, bool& dup) {
  uint32_t s = home_slot32(key, cap);
  for (uint32_t step = 0; step < cap; ++step) {
    uint64_t cur = ld_relaxed_u64(&slots[s]);
    if (cur == kEmpty64) {
      cur = atomicCAS((unsigned long long*)&slots[s], kEmpty64, desired);
      if (cur == kEmpty64) return true;
    }
    if ((uint32_t)cur == key) dup = true;
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

// Insert into a table of 16-byte slots {uint64 key, uint32 payload, uint32 pad = ~0}.  Every
// visited slot is read through the 128-bit CAS itself, so key and payload are seen together.
__device__ __forceinline__ bool join_insert64(ulonglong2* slots, uint32_t cap, uint64_t key,
                                              uint32_t payload, bool& dup) {
  uint32_t s = home_slot64(key, cap);
  const unsigned long long nhi = 0xFFFFFFFF00000000ull | payload;
  for (uint32_t step = 0; step < cap; ++step) {
    unsigned long long olo, ohi;
    cas128((unsigned long long*)&slots[s], kEmpty64, kEmpty64, key, nhi, olo, ohi);
    if (olo == kEmpty64 && ohi == kEmpty64) return true;
    if (olo == key) dup = true;
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

// Group table: keys[cap] (int64; kEmptyKey marks an empty slot) plus one extra slot `cap`
// reserved for the key equal to kEmptyKey itself.  Returns the key's slot, inserting it if
// new, or -1 when the table is full (more than `limit` distinct keys).
__device__ __forceinline__ int64_t group_find_or_insert(int64_t* keys, uint32_t cap, int64_t key,
                                                        unsigned long long* distinct,
                                                        unsigned long long limit) {
  if (key == kEmptyKey) return cap;
  uint32_t s = home_slot64((uint64_t)key, cap);
  for (uint32_t step = 0; step < cap; ++step) {
    // A walk this long only happens near or past the limit.  Past it -- once an insert has
    // failed, which takes the count above the limit -- the call fails (TABLE_FULL) and its
    // output is unspecified, so the walk stops: otherwise inserts would go on claiming slots
    // until none is left and every further new key would walk the whole table.  A table
    // holding exactly `limit` keys is still valid (an eighth of its slots are empty), and a
    // lookup there may walk far: it must not stop.
    if ((step & 63) == 63 && ld_relaxed_u64((const uint64_t*)distinct) > limit) return -1;
    int64_t cur = (int64_t)ld_relaxed_u64((const uint64_t*)&keys[s]);
    if (cur == key) return s;
    if (cur == kEmptyKey) {
      cur = (int64_t)atomicCAS((unsigned long long*)&keys[s], (unsigned long long)kEmptyKey,
                               (unsigned long long)key);
      if (cur == kEmptyKey) {
        if (atomicAdd(distinct, 1ull) >= limit) return -1;
        return s;
      }
      if (cur == key) return s;
    }
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return -1;
}

// Blocked Bloom filter over join keys: one 64-bit word per key (index from the high half of a
// 64-bit hash, masked to the power-of-two word count) with three bits set in it (from the low
// bits of the same hash), so a test is one 8-byte read and an insert one atomic OR.  No false
// negatives: every inserted key tests true.
__device__ __forceinline__ void bloom_word(uint64_t key, uint32_t mask, uint32_t& w, uint64_t& bits) {
  const uint64_t h = fmix64(key ^ 0x9E3779B97F4A7C15ull);
  w = (uint32_t)(h >> 32) & mask;
  bits = (1ull << (h & 63)) | (1ull << ((h >> 6) & 63)) | (1ull << ((h >> 12) & 63));
}
__device__ __forceinline__ void bloom_insert(uint64_t* f, uint32_t mask, uint64_t key) {
  uint32_t w;
  uint64_t bits;
  bloom_word(key, mask, w, bits);
  atomicOr(reinterpret_cast<unsigned long long*>(&f[w]), (unsigned long long)bits);
}
// Read-only during the probe pass: through the non-coherent path (kFresh: through L2 only,
// for a filter built earlier in the same launch).
template <bool kFresh = false>
__device__ __forceinline__ bool bloom_test(const uint64_t* f, uint32_t mask, uint64_t key) {
  uint32_t w;
  uint64_t bits;
  bloom_word(key, mask, w, bits);
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(f) + w;
  return ((kFresh ? __ldcg(p) : __ldg(p)) & bits) == bits;
}

// Capacity of a group table for an expected number of distinct keys: a power of two with
// load at most one half; `limit` = the most distinct keys accepted (7/8 of the slots).
inline int64_t group_capacity_for(int64_t hint) {
  if (hint < 1) hint = 1;
  int64_t c = 16;
  while (c < 2 * hint) c <<= 1;
  return c;
}
inline unsigned long long group_limit_for(int64_t cap) { return (unsigned long long)(cap - cap / 8); }

// Aggregates of one group slot.
struct __align__(32) Agg {
  unsigned long long sum;    // two's-complement sum (exact while the true sum fits int64)
  unsigned long long count;
  long long min;
  long long max;
};

// Global aggregation: four fire-and-forget reductions (no result is read back, so they
// compile to RED operations executed at L2).  Reading the {MIN, MAX} pair first and reducing
// MIN / MAX only when the value can change them (exact, since a stale extreme is never tighter
// than the current one) saves a request per row once extremes settle, but measured slower in
// the fused probe pass: the read is a round trip on the row's path and its registers cost the
// kernel half its resident warps.
__device__ __forceinline__ void agg_update_global(Agg* a, int64_t v, uint32_t aggs) {
  if (aggs & SIRIUS_AGG_SUM) atomicAdd(&a->sum, (unsigned long long)v);
  atomicAdd(&a->count, 1ull);
  if (aggs & SIRIUS_AGG_MIN) atomicMin(&a->min, (long long)v);
  if (aggs & SIRIUS_AGG_MAX) atomicMax(&a->max, (long long)v);
}

// The same four reductions with an L2 policy that keeps the aggregate lines resident while the
// fact columns stream past them (createpolicy evict_last).
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void agg_update_global_keep(Agg* a, int64_t v, uint32_t aggs, uint64_t pol) {
  if (aggs & SIRIUS_AGG_SUM)
    asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(&a->sum), "l"(v), "l"(pol) : "memory");
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(&a->count), "l"(1ull), "l"(pol) : "memory");
  if (aggs & SIRIUS_AGG_MIN)
    asm volatile("red.global.min.L2::cache_hint.s64 [%0], %1, %2;" ::"l"(&a->min), "l"(v), "l"(pol) : "memory");
  if (aggs & SIRIUS_AGG_MAX)
    asm volatile("red.global.max.L2::cache_hint.s64 [%0], %1, %2;" ::"l"(&a->max), "l"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void agg_merge_global(Agg* a, unsigned long long sum, unsigned long long cnt,
                                                 long long mn, long long mx, uint32_t aggs) {
  if (aggs & SIRIUS_AGG_SUM) atomicAdd(&a->sum, sum);
  atomicAdd(&a->count, cnt);
  if (aggs & SIRIUS_AGG_MIN) atomicMin(&a->min, mn);
  if (aggs & SIRIUS_AGG_MAX) atomicMax(&a->max, mx);
}

__device__ __forceinline__ void agg_identity(Agg* a) {
  a->sum = 0;
  a->count = 0;
  a->min = INT64_MAX;
  a->max = INT64_MIN;
}

// Host-side helpers shared by the operator entry points.
sirius_status join_build(const int32_t* lo, const int32_t* hi, int64_t m, void* mem,
                         int64_t capacity, cudaStream_t s, bool clear);
int grid_for(int64_t n, int threads);

}  // namespace sirius
