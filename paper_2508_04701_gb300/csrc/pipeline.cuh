// Internal interface of the fused pipeline, shared by the single-query, host-streamed and
// batched paths: memory layouts, the probe pass's per-row device routines, host phases.
#pragma once

#include <type_traits>

#include "tables.cuh"

namespace sirius {

enum { kAggAuto = 0, kAggSmem = 1, kAggGlobal = 2, kAggPart = 3, kAggHot = 4, kAggRouted = 5 };
constexpr int64_t kSmemAggMaxBytes = 96 * 1024;  // shared-memory aggregates up to 3510 slots

// Build side ("dim index"): [DimHeader | JoinHeader + join slots | group keys[gcap + 1]].
// It depends on the dim table only, so it can stay resident and serve many probes.
struct DimHeader {
  int32_t status;                // first device error of the build (TABLE_FULL)
  uint32_t direct;               // 1: build keys dense and unique, the direct array is in use
  unsigned long long distinct;   // group slots claimed
  int32_t key_min, key_max;      // range of the one-column build keys
  uint32_t direct_failed;        // a duplicate key turned the direct array down: hash table used
  uint32_t bloom;                // 1: the hash table is in use and the Bloom filter holds its keys
  long long gkey_min, gkey_max;  // range of the group keys (the direct group-slot decision)
  unsigned long long pad[26];
};
static_assert(sizeof(DimHeader) == 256, "dim header is 256 bytes");

// Per-query run state: [PipeHeader | Agg[gcap + 1]].
struct PipeHeader {
  int32_t status;                // final status of the query (dim status, then CAPACITY)
  uint32_t blocks_done;          // finalize blocks that have finished
  unsigned long long groups;     // G
  unsigned long long pad[30];
};
static_assert(sizeof(PipeHeader) == 256, "pipeline header is 256 bytes");

// Dense one-column build keys (a range of at most 2m values, no duplicates) are joined through
// a direct-address array -- dslot[key - key_min] = group slot -- instead of the hash table (the
// "perfect hash" join of dense integer keys): 4 bytes per key value instead of 16 per key at
// load factor one half, so the structure of a 15M-row dim stays in L2.  The decision is taken
// on the device during the build; the hash table is built only when it is needed.
struct DimLayout {
  int key_width = 4;
  int64_t jcap = 0, gcap = 0;
  int64_t dcap = 0;    // direct-array entries (0: hash table only)
  int bloom_log2 = 0;  // Bloom filter of 2^bloom_log2 64-bit words after the direct array (0: none)
  size_t off_join = 256, off_gkeys = 0, off_direct = 0, off_bloom = 0, total = 0;
};

// Run state: [PipeHeader | Agg[gslots] | (partitioned mode) tuple slots, tuple values, prefixes].
struct RunLayout {
  int64_t gslots = 0;
  int mode = kAggGlobal;  // aggregation mode chosen for this run
  int parts = 0;          // partitioned mode: partitions and pass-1 tiles
  int64_t ntiles = 0;
  size_t off_aggs = 256, off_tgs = 0, off_tval = 0, off_prefix = 0, total = 0;
  size_t off_bounds = 0;  // extreme bounds of a split probe pass (0: none)
  // routed mode: blocks of the launch the exchange is sized for, owners (2^logP), slots per
  // owner, run capacity; exchange values, local slots, run lengths
  int route_blocks = 0, route_logP = 0;
  uint32_t route_R = 0, route_C = 0;
  size_t off_rval = 0, off_rls = 0, off_rfill = 0;
};

struct DimView {
  DimHeader* dhdr;
  JoinHeader* jhdr;
  void* jslots;
  int64_t* gkeys;
  uint32_t* dslot;
  uint64_t* bloom;      // nullptr: no Bloom filter
  uint32_t bloom_mask;  // words - 1
  uint32_t jcap;
  uint32_t gcap;
  int64_t dcap;
  int key_width;
};

struct ExtremeBounds;

struct RunView {
  PipeHeader* phdr;
  Agg* aggs;
  uint32_t* tgs;
  int64_t* tval;
  int32_t* prefix;
  int mode;
  int parts;
  int64_t ntiles;
  int64_t* rval;      // routed mode: exchange buffers (nullptr otherwise)
  uint16_t* rls;
  uint32_t* rfill;
  int route_blocks, route_logP;
  uint32_t route_R, route_C;
  ExtremeBounds* bounds;  // nullptr: the run has no room for a split probe pass
};

struct PipeOut {
  int64_t* keys;
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t cap;
  int64_t* d_groups;
  int32_t* d_status;
};

// Semi-join dims of a star query (further dims joined as filters).  Each has its own region:
// [SemiHeader | bitmap words | JoinHeader + hash-set slots].  After a pass over the keys of its
// qualifying rows, the build takes the bitmap over [key_min, key_max] when the keys are one
// column and span at most 32 bits per dim row (membership = one bit), else the hash set (the
// join table's layout with payload 0; membership = a bucket walk).
constexpr int kMaxSemi = SIRIUS_MAX_SEMIJOINS;

struct SemiHeader {
  int32_t key_min, key_max;  // range of the qualifying one-column keys
  uint32_t bitmap;           // 1: membership by the bitmap
  int32_t pad0;
  unsigned long long pad[30];
};
static_assert(sizeof(SemiHeader) == 256, "semi-join header is 256 bytes");

struct SemiLayout {
  int key_width = 4;
  int64_t words = 0;  // bitmap words (32 bits each): m + 2
  int64_t jcap = 0;   // hash-set slots
  size_t off_bits = 256, off_join = 0, total = 0;
};

// One semi-join dim as the probe pass and its build see it.
struct SemiView {
  const int32_t* fk;     // fact key column, or its low word
  const int32_t* fk_hi;  // nullptr, or the high word
  SemiHeader* hdr;
  uint32_t* bits;
  JoinHeader* jhdr;
  void* jslots;
  uint32_t jcap;
  int64_t words;
  int key_width;
};

// Extreme bounds for the second phase of a split probe pass (taken after the first phase over
// the group table): every slot whose bit is set had joined rows, its MAX at least max_floor and
// its MIN at most min_ceil -- and both only move outwards, so a later row of such a slot whose
// value is below max_floor cannot change the slot's MAX, nor one above min_ceil its MIN.
constexpr uint32_t kBoundSlots = 1u << 17;          // group slots the bitmap covers
constexpr uint32_t kBoundWords = kBoundSlots / 32;  // 16 KB
struct __align__(16) ExtremeBounds {
  // both taken with atomicMin from all-ones (one memset clears them): the order-preserving
  // encoding (value ^ sign bit) of max_floor, and its complement for min_ceil
  unsigned long long max_floor_enc;
  unsigned long long min_ceil_inv;
  unsigned long long pad[2];
  uint32_t seen[kBoundWords];    // bit s: slot s had joined rows when the bounds were taken
};
__host__ __device__ __forceinline__ unsigned long long bound_encode(long long v) {
  return (unsigned long long)v ^ 0x8000000000000000ull;
}
__host__ __device__ __forceinline__ long long bound_decode(unsigned long long e) {
  return (long long)(e ^ 0x8000000000000000ull);
}
// The decoded bounds of the running block (set at the start of a second-phase launch).
__shared__ long long s_bound_floor, s_bound_ceil;

// Everything the probe pass reads for one query.
struct ProbeArgs {
  const int32_t* fk;
  const int32_t* fk_hi;
  const int32_t* pred;
  const int64_t* val;
  int64_t n;
  int32_t op;
  int32_t lit;
  uint32_t aggs;
  uint32_t jcap;
  const void* jslots;
  const JoinHeader* jhdr;
  const DimHeader* dhdr;
  const uint32_t* dslot;
  Agg* tab;
  uint32_t gslots;
  const uint64_t* bloom;  // nullptr: no Bloom filter
  uint32_t bloom_mask;
  const ExtremeBounds* bounds = nullptr;  // second phase of a split probe pass (hot / global modes)
};

// The semi-join dims of a star query: a kernel parameter of its own, read only by the kSemi
// instantiations of the probe pass (so the others carry no trace of it).
struct SemiArgs {
  int32_t nsemi;
  SemiView semi[kMaxSemi];
};

// How the probe pass tests one semi-join dim: its columns and structures, and the outcome of
// the build read once from its header.
struct SemiLookup {
  bool bitmap;
  bool wide;
  int32_t kmin;
  uint32_t range;  // key_max - key_min + 1, 0 when no dim row qualifies
  uint32_t jcap;
  const int32_t* fk;
  const int32_t* fk_hi;
  const uint32_t* bits;
  const void* jslots;
};
struct SemiLookups {
  int n;
  SemiLookup s[kMaxSemi];
};

__device__ __forceinline__ void read_semi_lookup(const SemiArgs& sa, SemiLookups& SL) {
  SL.n = sa.nsemi;
#pragma unroll
  for (int i = 0; i < kMaxSemi; ++i) {
    SL.s[i] = SemiLookup{false, false, 0, 0u, 0u, nullptr, nullptr, nullptr, nullptr};
    if (i < sa.nsemi) {
      const SemiView& v = sa.semi[i];
      const int64_t range = (int64_t)v.hdr->key_max - (int64_t)v.hdr->key_min + 1;
      SL.s[i].bitmap = v.hdr->bitmap != 0;
      SL.s[i].wide = v.key_width == 8;
      SL.s[i].kmin = v.hdr->key_min;
      SL.s[i].range = range > 0 ? (uint32_t)range : 0u;
      SL.s[i].jcap = v.jcap;
      SL.s[i].fk = v.fk;
      SL.s[i].fk_hi = v.fk_hi;
      SL.s[i].bits = v.bits;
      SL.s[i].jslots = v.jslots;
    }
  }
}

// How the probe pass finds a key's group slot, read once from the dim header.
struct Lookup {
  bool direct;     // direct array in use
  bool dups;       // hash table holds duplicate keys (walks go past the first match)
  bool bloom;      // hash table in use and a Bloom filter of its keys to test first
  int32_t kmin;
  uint32_t range;  // key_max - key_min + 1 (direct mode)
};

// kFresh: the build ran earlier in the same launch, so the headers are read through volatile
// loads (L2), never from a line this SM's L1 may hold from before the build finished.
template <bool kFresh = false>
__device__ __forceinline__ Lookup read_lookup(const ProbeArgs& a) {
  using DH = std::conditional_t<kFresh, const volatile DimHeader, const DimHeader>;
  using JH = std::conditional_t<kFresh, const volatile JoinHeader, const JoinHeader>;
  DH* dh = a.dhdr;
  JH* jh = a.jhdr;
  Lookup L;
  L.direct = dh->direct != 0 && dh->direct_failed == 0;
  L.dups = jh->has_dups != 0;
  L.bloom = a.bloom != nullptr && !L.direct && dh->bloom != 0;
  L.kmin = dh->key_min;
  L.range = (uint32_t)((int64_t)dh->key_max - (int64_t)L.kmin + 1);
  return L;
}

// ------------------------------------------------------------------ probe pass, per row
// One join-table slot as (key, payload); payload kEmpty32 = empty.  The table is read-only
// during the probe pass, so slots go through the non-coherent read-only path.
template <bool kWide>
__device__ __forceinline__ void load_slot(const void* slots, uint32_t s, uint64_t& key, uint32_t& payload) {
  if (kWide) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(slots) + s);
    key = v.x;
    payload = (uint32_t)v.y;
  } else {
    const uint64_t v = __ldg(reinterpret_cast<const uint64_t*>(slots) + s);
    key = (uint32_t)v;
    payload = (uint32_t)(v >> 32);
  }
}

// Per-block aggregates in shared memory (the shared-memory and hot-group modes), stored as
// arrays -- SUM, MIN, MAX (64-bit), COUNT (32-bit) and, for the hot-group cache, a tag per
// entry -- rather than as 32-byte records: a warp's updates of random slots then spread over
// the 32 banks, where the record layout puts every record's SUM on the same four banks.
// COUNT is 32-bit because a block counts at most the rows it processes between two merges,
// fewer than 2^32 (the library's row-count limit).
struct SmemAggs {
  unsigned long long* sum = nullptr;
  long long* mn = nullptr;
  long long* mx = nullptr;
  uint32_t* cnt = nullptr;
  uint32_t* tag = nullptr;  // hot-group cache only
};
__host__ __device__ constexpr size_t smem_aggs_bytes(uint32_t slots, bool tags) {
  return (size_t)slots * (tags ? 32 : 28);
}
__device__ __forceinline__ SmemAggs smem_aggs(unsigned char* base, uint32_t slots) {
  SmemAggs t;
  t.sum = reinterpret_cast<unsigned long long*>(base);
  t.mn = reinterpret_cast<long long*>(base + (size_t)slots * 8);
  t.mx = reinterpret_cast<long long*>(base + (size_t)slots * 16);
  t.cnt = reinterpret_cast<uint32_t*>(base + (size_t)slots * 24);
  t.tag = reinterpret_cast<uint32_t*>(base + (size_t)slots * 28);
  return t;
}
__device__ __forceinline__ void smem_identity(const SmemAggs& t, uint32_t i) {
  t.sum[i] = 0;
  t.mn[i] = INT64_MAX;
  t.mx[i] = INT64_MIN;
  t.cnt[i] = 0;
}
__device__ __forceinline__ void agg_update_smem(const SmemAggs& t, uint32_t i, int64_t v, uint32_t aggs) {
  if (aggs & SIRIUS_AGG_SUM) atomicAdd(&t.sum[i], (unsigned long long)v);
  atomicAdd(&t.cnt[i], 1u);
  if ((aggs & SIRIUS_AGG_MIN) && v < t.mn[i]) atomicMin(&t.mn[i], (long long)v);
  if ((aggs & SIRIUS_AGG_MAX) && v > t.mx[i]) atomicMax(&t.mx[i], (long long)v);
}
// Merge entry i into a global aggregate (nothing when it counted no row).
__device__ __forceinline__ void smem_merge(const SmemAggs& t, uint32_t i, Agg* dst, uint32_t aggs) {
  const uint32_t c = t.cnt[i];
  if (c) agg_merge_global(dst, t.sum[i], c, t.mn[i], t.mx[i], aggs);
}

// Hot-group cache (kAggHot): kHotEntries direct-mapped entries per block, each claimed once by
// the first group slot that maps to it (tag[e], kEmpty32 = free).  Under a skewed key
// distribution the frequent groups claim entries early and then aggregate on chip; other
// rows go to the global table.
constexpr int kHotBits = 11;
constexpr int kHotEntries = 1 << kHotBits;
constexpr size_t kHotSmemBytes = smem_aggs_bytes(kHotEntries, true);

// The global reductions of one joined row in the second phase of a split probe pass: MIN and
// MAX are skipped where the bounds show that the value cannot move them.
constexpr size_t kBoundsSmemBytes = sizeof(ExtremeBounds);
template <int kMode>
__device__ __forceinline__ void agg_update_global_bounded(const ProbeArgs& a, uint32_t gs, int64_t v) {
  uint32_t aggs = a.aggs;
  // the bounds' copy in shared memory follows the hot-group cache; the bitmap and the decoded
  // extremes are read where used (no registers held for them)
  extern __shared__ __align__(32) unsigned char probe_dyn_smem[];
  const volatile uint32_t* seen = reinterpret_cast<const volatile ExtremeBounds*>(
                                      probe_dyn_smem + (kMode == kAggHot ? kHotSmemBytes : 0))->seen;
  if (gs < kBoundSlots && ((seen[gs >> 5] >> (gs & 31)) & 1u)) {
    if (v < *(volatile long long*)&s_bound_floor) aggs &= ~(uint32_t)SIRIUS_AGG_MAX;
    if (v > *(volatile long long*)&s_bound_ceil) aggs &= ~(uint32_t)SIRIUS_AGG_MIN;
  }
  agg_update_global(&a.tab[gs], v, aggs);
}

// The extreme bounds after the first phase of a split pass (the fused probe, the group-by): one
// thread per group slot below kBoundSlots (a bit per slot that has joined rows, by ballot), the
// smallest MAX and the largest MIN over those slots by block reductions and one atomicMin per
// block on their encodings (set to all-ones before the launch).
static __global__ void __launch_bounds__(256)
extreme_bounds_kernel(const Agg* __restrict__ tab, uint32_t gslots, ExtremeBounds* b) {
  __shared__ unsigned long long s_floor, s_ceil;  // encoded MAX floor, complemented MIN ceiling
  if (threadIdx.x == 0) {
    s_floor = ~0ull;
    s_ceil = ~0ull;
  }
  __syncthreads();
  const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;  // < kBoundSlots (grid covers it exactly)
  unsigned long long fl = ~0ull, ce = ~0ull;
  bool seen = false;
  if (slot < gslots) {
    const Agg g = tab[slot];
    seen = g.count != 0;
    if (seen) {
      fl = bound_encode(g.max);
      ce = ~bound_encode(g.min);
    }
  }
  const unsigned bits = __ballot_sync(0xffffffffu, seen);
  if ((threadIdx.x & 31) == 0) b->seen[slot >> 5] = bits;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long f2 = __shfl_xor_sync(0xffffffffu, fl, o), c2 = __shfl_xor_sync(0xffffffffu, ce, o);
    fl = f2 < fl ? f2 : fl;
    ce = c2 < ce ? c2 : ce;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&s_floor, fl);
    atomicMin(&s_ceil, ce);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMin(&b->max_floor_enc, s_floor);
    atomicMin(&b->min_ceil_inv, s_ceil);
  }
}

// kKeep: the global reductions carry an L2 evict_last hint (measured faster for star queries,
// whose filter structures and aggregates compete with the streamed columns for L2; slower for
// the others, which therefore go without it).
template <int kMode, bool kKeep = false, bool kBounded = false>
__device__ __forceinline__ void aggregate(const ProbeArgs& a, const SmemAggs& T, uint32_t gs, int64_t v) {
  if (kMode == kAggSmem) {
    agg_update_smem(T, gs, v, a.aggs);
  } else if (kMode == kAggHot) {
    const uint32_t e = (gs * 2654435761u) >> (32 - kHotBits);
    uint32_t t = *(volatile uint32_t*)&T.tag[e];
    if (t == kEmpty32) {
      t = atomicCAS(&T.tag[e], kEmpty32, gs);
      if (t == kEmpty32) t = gs;
    }
    if (t == gs) agg_update_smem(T, e, v, a.aggs);
    else if (kKeep) agg_update_global_keep(&a.tab[gs], v, a.aggs, l2_keep_policy());
    else if (kBounded) agg_update_global_bounded<kAggHot>(a, gs, v);
    else agg_update_global(&a.tab[gs], v, a.aggs);
  } else if (kKeep) {
    agg_update_global_keep(&a.tab[gs], v, a.aggs, l2_keep_policy());
  } else if (kBounded && kMode == kAggGlobal) {
    agg_update_global_bounded<kAggGlobal>(a, gs, v);
  } else {
    agg_update_global(&a.tab[gs], v, a.aggs);
  }
}

// One 32-byte bucket starting at slot s: four 8-byte slots, or two 16-byte slots.  kFresh:
// the table was written earlier in the same launch, so the load goes through L2 only.
template <bool kWide, bool kFresh = false>
__device__ __forceinline__ void load_bucket(const void* slots, uint32_t s, uint64_t (&w)[4]) {
  const char* p = reinterpret_cast<const char*>(slots) + (size_t)s * (kWide ? 16 : 8);
  if (kFresh) ldcg_bucket(p, w[0], w[1], w[2], w[3]);
  else ldg_bucket(p, w[0], w[1], w[2], w[3]);
}

// A read-only 4-byte load that asks L2 to keep the line (the direct array stays resident while
// the fact columns stream past it).
__device__ __forceinline__ uint32_t ldg_keep(const uint32_t* p) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(l2_keep_policy()));
  return v;
}

// Probe up to four rows (bit r of `bits` set = row r selected) and hand every (row, group slot,
// value) match to emit(r, slot, value).  The home bucket of every selected row is loaded before
// any row is examined, so four sector misses are in flight together; a walk continues bucket by
// bucket only past full buckets.  kFresh: the join structures were built earlier in the same
// launch (read through L2 only).  Without duplicate build keys a row matches at most once.
// kRows < 4: the hash-table walk covers rows 0 .. kRows-1 only (fewer buckets held at once).
template <bool kWide, bool kFresh, int kRows = 4, bool kKeep = false, class Emit>
__device__ __forceinline__ void probe_rows_emit(const ProbeArgs& a, const Lookup& L, uint32_t bits,
                                                const uint64_t (&key)[4], const int64_t (&v)[4], Emit&& emit) {
  if (!kWide && L.direct) {
    // dense keys: one 4-byte read of the direct array per selected row, all four in flight
    uint32_t gs[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t k = (uint32_t)key[r] - (uint32_t)L.kmin;
      gs[r] = (((bits >> r) & 1u) && k < L.range) ? (kFresh ? __ldcg(a.dslot + k) : (kKeep ? ldg_keep(a.dslot + k) : __ldg(a.dslot + k)))
                                                   : kEmpty32;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (gs[r] != kEmpty32) emit(r, gs[r], v[r]);
    return;
  }
  if (L.bloom) {
    // keys the filter rules out skip their bucket read (all four tests in flight together)
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (((bits >> r) & 1u) && !bloom_test<kFresh>(a.bloom, a.bloom_mask, key[r])) bits &= ~(1u << r);
    if (!bits) return;
  }
  const bool dups = L.dups;
  constexpr int kPer = kWide ? 2 : 4;  // slots per bucket
  uint32_t s[kRows];
  uint64_t w[kRows][4];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    if ((bits >> r) & 1u) {
      s[r] = kWide ? home_slot64(key[r], a.jcap) : home_slot32((uint32_t)key[r], a.jcap);
      load_bucket<kWide, kFresh>(a.jslots, s[r], w[r]);
    }
  }
  // Each bucket is scanned branch-free into a mask of matching slots before its first empty slot;
  // the matches are then emitted from one site per row (the first one only without duplicate
  // keys), which keeps the unrolled code -- and the instruction cache -- small.
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    if (!((bits >> r) & 1u)) continue;
    uint32_t slot = s[r];
    for (uint32_t step = 0; step < a.jcap; step += kPer) {
      uint32_t mm = 0, em = 0;
      uint32_t pay[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const uint64_t k = kWide ? w[r][2 * j] : (uint64_t)(uint32_t)w[r][j];
        pay[j] = kWide ? (uint32_t)w[r][2 * j + 1] : (uint32_t)(w[r][j] >> 32);
        em |= (uint32_t)(pay[j] == kEmpty32) << j;
        mm |= (uint32_t)(pay[j] != kEmpty32 && k == key[r]) << j;
      }
      if (em) mm &= (em & (0u - em)) - 1;  // only slots before the first empty one
      if (!dups) mm &= 0u - mm;             // unique keys: the first match only
      const bool done = em != 0 || (!dups && mm != 0);
      while (mm) {
        const int j = __ffs(mm) - 1;
        uint32_t p = pay[0];
#pragma unroll
        for (int t = 1; t < kPer; ++t) p = j == t ? pay[t] : p;
        emit(r, p, v[r]);
        mm &= mm - 1;
      }
      if (done) break;
      slot += kPer;
      if (slot >= a.jcap) slot = 0;
      load_bucket<kWide, kFresh>(a.jslots, slot, w[r]);
    }
  }
}

// The same, aggregating every match into the group table (kMode: where the aggregates live;
// kKeep: L2 keep hints on the direct-array reads and the reductions).
// kBounded (one-column keys): the direct-array join aggregates behind the extreme bounds of a
// split pass; the hash-table walk keeps the plain reductions.
template <bool kWide, int kMode, bool kFresh = false, bool kKeep = false, bool kBounded = false>
__device__ __forceinline__ void probe_rows(const ProbeArgs& a, const SmemAggs& T, const Lookup& L, uint32_t bits,
                                           const uint64_t (&key)[4], const int64_t (&v)[4]) {
  if constexpr (kBounded && !kWide) {
    if (L.direct) {
      uint32_t gs[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t k = (uint32_t)key[r] - (uint32_t)L.kmin;
        gs[r] = (((bits >> r) & 1u) && k < L.range) ? __ldg(a.dslot + k) : kEmpty32;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (gs[r] != kEmpty32) aggregate<kMode, false, true>(a, T, gs[r], v[r]);
      return;
    }
  }
  probe_rows_emit<kWide, kFresh, 4, kKeep>(a, L, bits, key, v,
                                           [&](int, uint32_t gs, int64_t val) { aggregate<kMode, kKeep>(a, T, gs, val); });
}

// Filter, probe and aggregate the four rows of quad q (rows 4q .. 4q+3, all < n).
// Membership of a key in a semi-join dim: one bit of the bitmap, or a bucket walk of the hash
// set (read-only during the probe pass: non-coherent loads).
template <bool kWide>
__device__ __forceinline__ bool semi_contains(const SemiLookup& SL, uint64_t key) {
  if (!kWide && SL.bitmap) {
    const uint32_t k = (uint32_t)key - (uint32_t)SL.kmin;
    return k < SL.range && ((__ldg(SL.bits + (k >> 5)) >> (k & 31)) & 1u);
  }
  constexpr int kPer = kWide ? 2 : 4;
  uint32_t slot = kWide ? home_slot64(key, SL.jcap) : home_slot32((uint32_t)key, SL.jcap);
  for (uint32_t step = 0; step < SL.jcap; step += kPer) {
    uint64_t w[4];
    load_bucket<kWide>(SL.jslots, slot, w);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const uint64_t k = kWide ? w[2 * j] : (uint64_t)(uint32_t)w[j];
      const uint32_t p = kWide ? (uint32_t)w[2 * j + 1] : (uint32_t)(w[j] >> 32);
      if (p == kEmpty32) return false;
      if (k == key) return true;
    }
    slot += kPer;
    if (slot >= SL.jcap) slot = 0;
  }
  return false;
}

// Star query: drop the selected rows among row0 .. row0+3 (bit r of `bits`; rows below n)
// whose key into some semi-join dim has no qualifying partner there.  kVec: the four rows'
// keys come as one 16-byte load per key column (row0 a multiple of 4, columns 16-byte aligned).
template <bool kVec>
__device__ __forceinline__ uint32_t semi_filter(const SemiLookups& SL, int64_t row0, uint32_t bits) {
#pragma unroll
  for (int i = 0; i < kMaxSemi; ++i) {
    if (i >= SL.n || !bits) break;
    const SemiLookup& sl = SL.s[i];
    uint64_t key[4];
    if (kVec) {
      const int4 k4 = __ldcs(reinterpret_cast<const int4*>(sl.fk + row0));
      int4 h4 = make_int4(0, 0, 0, 0);
      if (sl.wide) h4 = __ldcs(reinterpret_cast<const int4*>(sl.fk_hi + row0));
      key[0] = sl.wide ? pack_key64(h4.x, k4.x) : (uint64_t)(uint32_t)k4.x;
      key[1] = sl.wide ? pack_key64(h4.y, k4.y) : (uint64_t)(uint32_t)k4.y;
      key[2] = sl.wide ? pack_key64(h4.z, k4.z) : (uint64_t)(uint32_t)k4.z;
      key[3] = sl.wide ? pack_key64(h4.w, k4.w) : (uint64_t)(uint32_t)k4.w;
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        key[r] = 0;
        if ((bits >> r) & 1u)
          key[r] = sl.wide ? pack_key64(sl.fk_hi[row0 + r], sl.fk[row0 + r]) : (uint64_t)(uint32_t)sl.fk[row0 + r];
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!((bits >> r) & 1u)) continue;
      const bool in = sl.wide ? semi_contains<true>(sl, key[r]) : semi_contains<false>(sl, key[r]);
      if (!in) bits &= ~(1u << r);
    }
  }
  return bits;
}

// The same for the 16-byte-load path, shaped for memory parallelism when every filter dim has
// one-column keys (two-column ones take the loop above): every dim's four keys are loaded
// first, then every membership of every selected row is looked up (independent reads), and
// the results are combined.
__device__ __forceinline__ uint32_t semi_filter_vec(const SemiLookups& SL, int64_t row0, uint32_t bits) {
  const int n = SL.n;
  bool narrow = true;
#pragma unroll
  for (int i = 0; i < kMaxSemi; ++i)
    if (i < n && SL.s[i].wide) narrow = false;
  if (!narrow) return semi_filter<true>(SL, row0, bits);
  uint32_t key[kMaxSemi][4];
#pragma unroll
  for (int i = 0; i < kMaxSemi; ++i) {
    if (i >= n) break;
    const int4 k4 = __ldcs(reinterpret_cast<const int4*>(SL.s[i].fk + row0));
    key[i][0] = (uint32_t)k4.x;
    key[i][1] = (uint32_t)k4.y;
    key[i][2] = (uint32_t)k4.z;
    key[i][3] = (uint32_t)k4.w;
  }
  uint32_t keep = bits;
#pragma unroll
  for (int i = 0; i < kMaxSemi; ++i) {
    if (i >= n) break;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (((bits >> r) & 1u) && !semi_contains<false>(SL.s[i], key[i][r])) keep &= ~(1u << r);
  }
  return keep;
}

// kPreload (16-byte-load path only): the quad's predicates, keys and values are all requested
// before any of them is used -- three column reads in flight per thread instead of one after
// another -- at the cost of reading the values of unselected rows (a quad's values are one
// 32-byte sector, needed whenever any of its rows is selected).
template <bool kWide, int kMode, bool kVec, bool kSemi = false, bool kPreload = false, bool kFresh = false,
          bool kBounded = false>
__device__ __forceinline__ void probe_quad(const ProbeArgs& a, const SmemAggs& T, const Lookup& L, int64_t q,
                                           const SemiLookups* SLp = nullptr) {
  const int64_t row0 = q << 2;
  uint32_t bits = 0;
  uint64_t key[4];
  int64_t v[4];
  if (kVec && kPreload && !kSemi) {
    const int4 p4 = __ldcs(reinterpret_cast<const int4*>(a.pred) + q);
    const int4 k4 = __ldcs(reinterpret_cast<const int4*>(a.fk) + q);
    int4 h4 = make_int4(0, 0, 0, 0);
    if (kWide) h4 = __ldcs(reinterpret_cast<const int4*>(a.fk_hi) + q);
    int64_t vv[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) vv[r] = __ldcs(a.val + row0 + r);
    bits = (uint32_t)cmp_op(p4.x, a.lit, a.op) | ((uint32_t)cmp_op(p4.y, a.lit, a.op) << 1) |
           ((uint32_t)cmp_op(p4.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(p4.w, a.lit, a.op) << 3);
    if (!bits) return;
    key[0] = kWide ? pack_key64(h4.x, k4.x) : (uint64_t)(uint32_t)k4.x;
    key[1] = kWide ? pack_key64(h4.y, k4.y) : (uint64_t)(uint32_t)k4.y;
    key[2] = kWide ? pack_key64(h4.z, k4.z) : (uint64_t)(uint32_t)k4.z;
    key[3] = kWide ? pack_key64(h4.w, k4.w) : (uint64_t)(uint32_t)k4.w;
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = ((bits >> r) & 1u) ? vv[r] : 0;
    probe_rows<kWide, kMode, kFresh, kSemi, kBounded>(a, T, L, bits, key, v);
    return;
  }
  if (kVec) {
    const int4 p4 = __ldcs(reinterpret_cast<const int4*>(a.pred) + q);
    bits = (uint32_t)cmp_op(p4.x, a.lit, a.op) | ((uint32_t)cmp_op(p4.y, a.lit, a.op) << 1) |
           ((uint32_t)cmp_op(p4.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(p4.w, a.lit, a.op) << 3);
    if (kSemi) {
      if (!bits) return;
      // star query: the join key's load goes out with the filter dims' loads
      const int4 k4 = __ldcs(reinterpret_cast<const int4*>(a.fk) + q);
      int4 h4 = make_int4(0, 0, 0, 0);
      if (kWide) h4 = __ldcs(reinterpret_cast<const int4*>(a.fk_hi) + q);
      bits = semi_filter_vec(*SLp, row0, bits);
      if (!bits) return;
      key[0] = kWide ? pack_key64(h4.x, k4.x) : (uint64_t)(uint32_t)k4.x;
      key[1] = kWide ? pack_key64(h4.y, k4.y) : (uint64_t)(uint32_t)k4.y;
      key[2] = kWide ? pack_key64(h4.z, k4.z) : (uint64_t)(uint32_t)k4.z;
      key[3] = kWide ? pack_key64(h4.w, k4.w) : (uint64_t)(uint32_t)k4.w;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = ((bits >> r) & 1u) ? __ldcs(a.val + row0 + r) : 0;
      probe_rows<kWide, kMode, kFresh, kSemi, kBounded>(a, T, L, bits, key, v);
      return;
    }
    if (!bits) return;
    const int4 k4 = __ldcs(reinterpret_cast<const int4*>(a.fk) + q);
    if (kWide) {
      const int4 h4 = __ldcs(reinterpret_cast<const int4*>(a.fk_hi) + q);
      key[0] = pack_key64(h4.x, k4.x);
      key[1] = pack_key64(h4.y, k4.y);
      key[2] = pack_key64(h4.z, k4.z);
      key[3] = pack_key64(h4.w, k4.w);
    } else {
      key[0] = (uint32_t)k4.x;
      key[1] = (uint32_t)k4.y;
      key[2] = (uint32_t)k4.z;
      key[3] = (uint32_t)k4.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (cmp_op(a.pred[row0 + r], a.lit, a.op)) bits |= 1u << r;
    if (kSemi && bits) bits = semi_filter<false>(*SLp, row0, bits);
    if (!bits) return;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      key[r] = kWide ? pack_key64(a.fk_hi[row0 + r], a.fk[row0 + r]) : (uint64_t)(uint32_t)a.fk[row0 + r];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) v[r] = ((bits >> r) & 1u) ? __ldcs(a.val + row0 + r) : 0;
  probe_rows<kWide, kMode, kFresh, kSemi, kBounded>(a, T, L, bits, key, v);
}

// Two quads (qa, qb, both below n/4; 16-byte loads; one-column keys joined through the direct
// array): every column read of both, then every direct-array read of both, in flight together
// before any aggregate update -- twice the memory parallelism of probe_quad for kernels with
// registers to spare (the single-launch kernel runs one block per SM).
template <int kMode, bool kFresh = false, bool kBounded = false>
__device__ __forceinline__ void probe_quad_pair_direct(const ProbeArgs& a, const SmemAggs& T, const Lookup& L,
                                                       int64_t qa, int64_t qb) {
  const int4 pa = __ldcs(reinterpret_cast<const int4*>(a.pred) + qa);
  const int4 pb = __ldcs(reinterpret_cast<const int4*>(a.pred) + qb);
  const int4 ka = __ldcs(reinterpret_cast<const int4*>(a.fk) + qa);
  const int4 kb = __ldcs(reinterpret_cast<const int4*>(a.fk) + qb);
  int64_t va[4], vb[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    va[r] = __ldcs(a.val + (qa << 2) + r);
    vb[r] = __ldcs(a.val + (qb << 2) + r);
  }
  const uint32_t ba = (uint32_t)cmp_op(pa.x, a.lit, a.op) | ((uint32_t)cmp_op(pa.y, a.lit, a.op) << 1) |
                      ((uint32_t)cmp_op(pa.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(pa.w, a.lit, a.op) << 3);
  const uint32_t bb = (uint32_t)cmp_op(pb.x, a.lit, a.op) | ((uint32_t)cmp_op(pb.y, a.lit, a.op) << 1) |
                      ((uint32_t)cmp_op(pb.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(pb.w, a.lit, a.op) << 3);
  const uint32_t kav[4] = {(uint32_t)ka.x, (uint32_t)ka.y, (uint32_t)ka.z, (uint32_t)ka.w};
  const uint32_t kbv[4] = {(uint32_t)kb.x, (uint32_t)kb.y, (uint32_t)kb.z, (uint32_t)kb.w};
  uint32_t ga[4], gb[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint32_t x = kav[r] - (uint32_t)L.kmin, y = kbv[r] - (uint32_t)L.kmin;
    ga[r] = (((ba >> r) & 1u) && x < L.range) ? (kFresh ? __ldcg(a.dslot + x) : __ldg(a.dslot + x)) : kEmpty32;
    gb[r] = (((bb >> r) & 1u) && y < L.range) ? (kFresh ? __ldcg(a.dslot + y) : __ldg(a.dslot + y)) : kEmpty32;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (ga[r] != kEmpty32) aggregate<kMode, false, kBounded>(a, T, ga[r], va[r]);
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (gb[r] != kEmpty32) aggregate<kMode, false, kBounded>(a, T, gb[r], vb[r]);
}

// Filter, probe and aggregate one single row r (< n): the ragged tail after the quads.
template <bool kWide, int kMode, bool kSemi = false, bool kFresh = false>
__device__ __forceinline__ void probe_one(const ProbeArgs& a, const SmemAggs& T, const Lookup& L, int64_t r,
                                          const SemiLookups* SLp = nullptr) {
  if (!cmp_op(a.pred[r], a.lit, a.op)) return;
  if (kSemi && !semi_filter<false>(*SLp, r, 1u)) return;
  uint64_t key[4] = {0, 0, 0, 0};
  int64_t v[4] = {0, 0, 0, 0};
  key[0] = kWide ? pack_key64(a.fk_hi[r], a.fk[r]) : (uint64_t)(uint32_t)a.fk[r];
  v[0] = a.val[r];
  probe_rows<kWide, kMode, kFresh, kSemi>(a, T, L, 1u, key, v);
}

// The dim-side predicate of a build (col == nullptr: every dim row takes part).
struct DimPred {
  const int32_t* col;
  int32_t op;
  int32_t lit;
};

// How a build enters its rows, decided from the key ranges its range pass recorded in the
// dim header.  Join entries: the direct array (one-column keys whose range fits it) or the hash
// table.  Group keys: when their range spans at most the group table's limit of distinct keys,
// slot = key - gmin directly (a dense group domain, such as a small integer attribute, needs
// no hashing, no compare-and-swap and no shared counter), else the hash table.  Either way a
// key has one slot, and the direct form is taken only where the hash table could not be full,
// so results and TABLE_FULL are the same.  With direct slots the build writes every slot's key
// (gmin + slot) once, coalesced, rather than each row its own: rows of one group would all
// store to one address.  Slots of keys no row has keep COUNT 0 and are never output.
struct BuildMode {
  bool direct = false;
  int32_t kmin = 0;
  bool gdirect = false;
  int64_t gmin = 0;
  int64_t grange = 0;  // direct group slots in use: gmax - gmin + 1
};

// The keys of direct group slots [i0, i1): slot i holds gmin + i.
__device__ __forceinline__ void fill_direct_group_keys(const DimView& d, const BuildMode& B, int64_t i0, int64_t i1,
                                                       int64_t step) {
  for (int64_t i = i0; i < i1; i += step) d.gkeys[i] = B.gmin + i;
}

// kFresh: the range pass ran earlier in the same launch (volatile header reads).
template <bool kFresh = false>
__device__ __forceinline__ BuildMode read_build_mode(const DimView& d, int64_t m, unsigned long long glimit,
                                                     bool allow_direct) {
  using DH = std::conditional_t<kFresh, const volatile DimHeader, const DimHeader>;
  DH* h = d.dhdr;
  BuildMode B;
  B.kmin = h->key_min;
  const int64_t range = (int64_t)h->key_max - (int64_t)B.kmin + 1;
  B.direct = allow_direct && d.key_width == 4 && d.dcap > 0 && m > 0 && range >= 1 && range <= d.dcap;
  B.gmin = h->gkey_min;
  const long long gmax = h->gkey_max;
  B.gdirect = m > 0 && gmax >= B.gmin && (unsigned long long)(gmax - B.gmin) < glimit;
  B.grange = B.gdirect ? gmax - B.gmin + 1 : 0;
  return B;
}

// Build step of one dim row j: unless the dim-side predicate leaves it out, enter its group
// key into the group table (slot gs), then (pk -> gs) into the join table -- and the key into
// the Bloom filter when there is one.  Returns false on TABLE_FULL.
// In direct mode the row claims dslot[key - kmin] with one CAS; finding it taken means a
// duplicate key (dup = true), which turns the direct array down for this dim.  With direct
// group slots the slot is the key's offset from gmin (the slot keys are written by the build
// beside its rows).
template <bool kWide>
__device__ __forceinline__ bool dim_build_row(const int32_t* pk, const int32_t* pk_hi, const int32_t* grp,
                                              const int8_t* flag, int64_t j, const DimView& d,
                                              unsigned long long glimit, bool& dup, const DimPred& P,
                                              const BuildMode& B) {
  if (P.col && !cmp_op(P.col[j], P.lit, P.op)) return true;
  const bool direct = B.direct;
  const int32_t kmin = B.kmin;
  const int64_t gk = group_key(grp[j], flag, j);
  int64_t gs;
  if (B.gdirect) {
    gs = gk - B.gmin;
  } else {
    gs = group_find_or_insert(d.gkeys, d.gcap, gk, &d.dhdr->distinct, glimit);
    if (gs < 0) return false;
  }
  if (kWide) {
    const uint64_t key = pack_key64(pk_hi[j], pk[j]);
    if (d.bloom) bloom_insert(d.bloom, d.bloom_mask, key);
    return join_insert64((ulonglong2*)d.jslots, d.jcap, key, (uint32_t)gs, dup);
  }
  const uint32_t key = (uint32_t)pk[j];
  if (direct) {
    if (atomicCAS(&d.dslot[key - (uint32_t)kmin], kEmpty32, (uint32_t)gs) != kEmpty32) dup = true;
    return true;
  }
  if (d.bloom) bloom_insert(d.bloom, d.bloom_mask, (uint64_t)key);
  return join_insert32((uint64_t*)d.jslots, d.jcap, key, (uint64_t)key | ((uint64_t)(uint32_t)gs << 32), dup);
}

// Whether a dim's build takes the direct array: one-column keys whose range fits dcap.
__device__ __forceinline__ bool direct_applies(const DimView& d, int64_t m) {
  if (d.key_width != 4 || d.dcap <= 0 || m <= 0) return false;
  const int64_t range = (int64_t)d.dhdr->key_max - (int64_t)d.dhdr->key_min + 1;
  return range >= 1 && range <= d.dcap;
}

// ------------------------------------------------------------------ grid-wide barrier
// Spins of one barrier wait (64 ns sleeps: about half a second) before it gives up.  Every block
// of a cooperative launch is resident, so a barrier normally completes within microseconds; the
// bound is reached only when blocks cannot run (the GPU time-sliced to another context for longer
// than the bound, or a fault), and the call then reports SIRIUS_ERR_TIMEOUT, which a caller may
// retry.
constexpr uint32_t kGridBarrierSpins = 1u << 23;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  return cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(*const_cast<uint32_t*>(p))
      .load(cuda::memory_order_acquire);
}

// Grid-wide barrier of the cooperative launches (the single-launch pipeline, the routed probe).  Thread 0 of each block arrives on `count`
// (zero when the launch started) and waits until `target` = barriers so far x blocks arrivals
// have been made; the fences order every block's writes before the barrier ahead of every
// read after it.  The wait is bounded (max_spins sleeps of 64 ns): when it runs out, the block
// records SIRIUS_ERR_TIMEOUT in the run header and the caller leaves the kernel.
__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t target, int32_t* status,
                                             uint32_t max_spins = kGridBarrierSpins) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(count, 1u);
    uint32_t spins = 0;
    while (ld_acquire_u32(count) < target) {
      if (++spins >= max_spins) {
        set_status(status, SIRIUS_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------ host phases
DimLayout dim_layout(int64_t m, bool wide, int64_t group_cap_hint, float load_factor, bool allow_direct,
                     bool bloom = false);
DimLayout dim_layout_for(const sirius_pipeline_desc* q);
DimLayout dim_layout_of_index(const sirius_dim_index* idx);
// n: fact rows of the run (sizes the partitioned-mode buffers); agg_mode as in the descriptor.
// bounds: room for the extreme bounds of a split probe pass (hot-group or global modes; the
// batched calls, which never split, leave it out)
RunLayout run_layout(int64_t gcap, int64_t n = 0, int agg_mode = kAggGlobal, bool bounds = true);
DimView dim_view(const DimLayout& L, char* base);
RunView run_view(const RunLayout& R, char* base);
sirius_status validate_dim(const sirius_pipeline_desc* q);
sirius_status validate_fact(const sirius_pipeline_desc* q);
int choose_mode(int agg_mode, int64_t gslots, int64_t n);
// Plan of the routed probe (agg_mode 5) for a group table of gslots slots; R = 0: not possible.
struct RoutePlan {
  int blocks = 0;   // blocks of the cooperative launch
  int logP = 0;     // owners = 2^logP
  uint32_t R = 0;   // slots per owner
  uint32_t C = 0;   // tuples per (owner, block) run and round
};
RoutePlan route_plan(int64_t gslots);
sirius_status dim_build(const sirius_pipeline_desc* q, const DimLayout& L, char* base, cudaStream_t s);
sirius_status run_init(const RunLayout& R, char* base, cudaStream_t s);
sirius_status run_probe(const sirius_pipeline_desc* q, const DimView& d, const RunView& r, int64_t gslots,
                        cudaStream_t s, const SemiView* semi = nullptr, int nsemi = 0);
sirius_status run_finalize(const sirius_pipeline_desc* q, const DimView& d, const RunView& r,
                           int64_t gslots, const PipeOut& out, cudaStream_t s);
sirius_status read_run_status(const RunView& r, sirius_result* res, cudaStream_t s);

}  // namespace sirius
