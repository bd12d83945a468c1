// A7: one fused pipeline -- build over the dim, then filter -> probe -> aggregate in a single
// pass over the fact table, then finalize (Sec. 3.2.2: pipeline execution model, push-based
// operators, late materialisation; Sec. 4.2: join, group-by and filter are where time goes).
//
// Build (pipeline breaker): each dim row's group key g is entered into the group table
// (insert-or-find, slot gs), and (pk -> gs) into the join table.  Because the group key is an
// attribute of the dim row, the join payload can be the group slot itself: the probe pass
// aggregates straight into slot gs, so no row ids, gathered columns or second hash lookup
// exist between the operators.  The probe pass streams pred / fk / val with 16-byte
// evict-first loads (each column byte is read once), probes four rows per thread with their
// first slot loads in flight together, and aggregates (agg_mode)
//   - into a per-block copy of the aggregates in shared memory when the group table is small
//     (few groups contend on chip, not in L2), merged into the global table at block exit;
//   - through a per-block cache of hot groups in shared memory, the rest with global
//     reductions, when it is large (the default for large tables);
//   - with global reductions only (SUM, COUNT, MIN, MAX: four fire-and-forget REDs);
//   - or partitioned: tuples (slot, value) scattered by slot range per tile, then one
//     shared-memory pass per partition (csrc/partagg.cuh).
// Finalize compacts the slots with COUNT > 0 into the caller's output arrays.
//
// The build side ("dim index") and the per-query run state live in separate memory, so a dim
// index can stay resident and serve many probes (the caching region, Sec. 3.2.3), and a fact
// table in host memory can be streamed through the probe pass chunk by chunk while the next
// chunk is copied (batch execution over data larger than device memory, Sec. 3.4).
#include "pipeline.cuh"
#include "partagg.cuh"
#include "probe_staged.cuh"
#include "routed.cuh"

namespace sirius {

namespace {

// Clears the dim index: headers (key range to its empty value), join slots (kEmpty), direct
// array (kEmpty32, as 16-byte words), group keys and the Bloom filter's words.  The join slots
// are only cleared when the hash table may be needed (`jpairs` is 0 when the direct array is
// certain to be used).
__device__ __forceinline__ void dim_init_rows(DimHeader* dhdr, JoinHeader* jhdr, ulonglong2* jwords2,
                                              int64_t jpairs, ulonglong2* dwords2, int64_t dpairs, int64_t* gkeys,
                                              int64_t gslots, uint64_t* bloom, int64_t bwords, int64_t tid,
                                              int64_t stride) {
  if (tid < 32) {
    // word 2 of the dim header holds (key_min, key_max): start at (INT32_MAX, INT32_MIN);
    // words 4 and 5 the group key range: start at (INT64_MAX, INT64_MIN)
    reinterpret_cast<uint64_t*>(dhdr)[tid] = tid == 2   ? 0x800000007FFFFFFFull
                                             : tid == 4 ? 0x7FFFFFFFFFFFFFFFull
                                             : tid == 5 ? 0x8000000000000000ull
                                                        : 0ull;
    reinterpret_cast<uint64_t*>(jhdr)[tid] = 0;
  }
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  for (int64_t i = tid; i < jpairs; i += stride) jwords2[i] = ones;
  for (int64_t i = tid; i < dpairs; i += stride) dwords2[i] = ones;
  for (int64_t i = tid; i < gslots; i += stride) gkeys[i] = kEmptyKey;
  for (int64_t i = tid; i < bwords; i += stride) bloom[i] = 0;
}
__global__ void dim_init_kernel(DimHeader* dhdr, JoinHeader* jhdr, ulonglong2* jwords2, int64_t jpairs,
                                ulonglong2* dwords2, int64_t dpairs, int64_t* gkeys, int64_t gslots,
                                uint64_t* bloom, int64_t bwords) {
  dim_init_rows(dhdr, jhdr, jwords2, jpairs, dwords2, dpairs, gkeys, gslots, bloom, bwords,
                blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Ranges of the one-column build keys (the direct-array decision) and of the group keys (the
// direct group-slot decision).
// Every thread of the block takes part: warp reductions, then one per block, so each block
// sends one atomic per range end to the header's shared address instead of one per warp.
__device__ __forceinline__ void dim_minmax_rows(const int32_t* __restrict__ pk, const int32_t* __restrict__ grp,
                                                const int8_t* __restrict__ flag, int64_t m, DimHeader* dhdr,
                                                int64_t tid, int64_t stride) {
  __shared__ int32_t s_lo[32], s_hi[32];
  __shared__ long long s_glo[32], s_ghi[32];
  int32_t lo = INT32_MAX, hi = INT32_MIN;
  long long glo = INT64_MAX, ghi = INT64_MIN;
  for (int64_t j = tid; j < m; j += stride) {
    const int32_t k = pk[j];
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
    const long long g = group_key(grp[j], flag, j);
    glo = g < glo ? g : glo;
    ghi = g > ghi ? g : ghi;
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  glo = warp_min_i64(glo);
  ghi = warp_max_i64(ghi);
  const unsigned w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_lo[w] = lo;
    s_hi[w] = hi;
    s_glo[w] = glo;
    s_ghi[w] = ghi;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool have = threadIdx.x < (blockDim.x >> 5);
    lo = __reduce_min_sync(0xffffffffu, have ? s_lo[threadIdx.x] : INT32_MAX);
    hi = __reduce_max_sync(0xffffffffu, have ? s_hi[threadIdx.x] : INT32_MIN);
    glo = warp_min_i64(have ? s_glo[threadIdx.x] : INT64_MAX);
    ghi = warp_max_i64(have ? s_ghi[threadIdx.x] : INT64_MIN);
    if (threadIdx.x == 0 && lo <= hi) {
      atomicMin(&dhdr->key_min, lo);
      atomicMax(&dhdr->key_max, hi);
      atomicMin(&dhdr->gkey_min, glo);
      atomicMax(&dhdr->gkey_max, ghi);
    }
  }
}
__global__ void dim_minmax_kernel(const int32_t* __restrict__ pk, const int32_t* __restrict__ grp,
                                  const int8_t* __restrict__ flag, int64_t m, DimHeader* dhdr) {
  dim_minmax_rows(pk, grp, flag, m, dhdr, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

// Build.  One-column keys whose range fits the direct array are entered there; otherwise (and
// for two-column keys) into the hash table.
// The build mode comes from the key ranges the caller read; every thread of every warp takes
// part.
template <bool kWide>
__device__ __forceinline__ void dim_build_rows(const int32_t* __restrict__ pk, const int32_t* __restrict__ pk_hi,
                                               const int32_t* __restrict__ grp, const int8_t* __restrict__ flag,
                                               int64_t m, const DimView& d, unsigned long long glimit,
                                               const DimPred& P, const BuildMode& B, int64_t tid, int64_t stride) {
  if (tid == 0) {
    d.dhdr->direct = B.direct ? 1u : 0u;
    if (!B.direct && d.bloom) d.dhdr->bloom = 1;
  }
  if (B.gdirect) fill_direct_group_keys(d, B, tid, B.grange, stride);
  bool dup = false;
  for (int64_t j = tid; j < m; j += stride) {
    if (!dim_build_row<kWide>(pk, pk_hi, grp, flag, j, d, glimit, dup, P, B))
      set_status(&d.dhdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) {
    if (B.direct) d.dhdr->direct_failed = 1;
    else d.jhdr->has_dups = 1;
  }
}
template <bool kWide>
__global__ void dim_build_kernel(const int32_t* __restrict__ pk, const int32_t* __restrict__ pk_hi,
                                 const int32_t* __restrict__ grp, const int8_t* __restrict__ flag,
                                 int64_t m, DimView d, unsigned long long glimit, DimPred P) {
  const BuildMode B = read_build_mode(d, m, glimit, !kWide);
  dim_build_rows<kWide>(pk, pk_hi, grp, flag, m, d, glimit, P, B, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                        (int64_t)gridDim.x * blockDim.x);
}

// Clears the join slots of a large table only when the hash table turns out to be needed:
// before the build (phase 0) when the key range does not fit the direct array, after it
// (phase 1) when a duplicate key turned the direct array down.
__global__ void dim_clear_join_kernel(DimView d, int64_t m, int phase, int64_t jpairs) {
  const bool need = phase == 0 ? !direct_applies(d, m) : (d.dhdr->direct && d.dhdr->direct_failed);
  if (!need) return;
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  ulonglong2* w = reinterpret_cast<ulonglong2*>(d.jslots);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < jpairs; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = ones;
}

// When a duplicate key turned the direct array down, enter every row into the hash table
// (the group keys are already in their table; finding them again returns the same slots).
// (Called only once the caller has seen the direct array turned down; B is the build's mode,
// whose group slots the rows find again.)
__device__ __forceinline__ void dim_fallback_rows(const int32_t* __restrict__ pk, const int32_t* __restrict__ grp,
                                                  const int8_t* __restrict__ flag, int64_t m, const DimView& d,
                                                  unsigned long long glimit, const DimPred& P, BuildMode B,
                                                  int64_t tid, int64_t stride) {
  if (tid == 0 && d.bloom) d.dhdr->bloom = 1;
  B.direct = false;
  bool dup = false;
  for (int64_t j = tid; j < m; j += stride) {
    if (!dim_build_row<false>(pk, nullptr, grp, flag, j, d, glimit, dup, P, B))
      set_status(&d.dhdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) d.jhdr->has_dups = 1;
}
__global__ void dim_fallback_kernel(const int32_t* __restrict__ pk, const int32_t* __restrict__ grp,
                                    const int8_t* __restrict__ flag, int64_t m, DimView d,
                                    unsigned long long glimit, DimPred P) {
  if (!(d.dhdr->direct && d.dhdr->direct_failed)) return;
  dim_fallback_rows(pk, grp, flag, m, d, glimit, P, read_build_mode(d, m, glimit, true),
                    blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__global__ void run_init_kernel(PipeHeader* phdr, Agg* aggs, int64_t gslots) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid < 32) reinterpret_cast<uint64_t*>(phdr)[tid] = 0;
  for (int64_t i = tid; i < gslots; i += (int64_t)gridDim.x * blockDim.x) agg_identity(&aggs[i]);
}

// ------------------------------------------------------------------ semi-join dims (star query)
struct SemiInput {
  const int32_t* pk;
  const int32_t* pk_hi;
  const int32_t* attr;
  int64_t m;
  int32_t op;
  int32_t lit;
};

__device__ __forceinline__ bool semi_row_qualifies(const SemiInput& in, int64_t j) {
  return !in.attr || cmp_op(in.attr[j], in.lit, in.op);
}

// Clears a semi-join dim's region: header (empty key range), bitmap and hash-set slots.
__global__ void semi_init_kernel(SemiView v, int64_t jpairs) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid < 32) {
    // word 0 of the header holds (key_min, key_max): start at (INT32_MAX, INT32_MIN)
    reinterpret_cast<uint64_t*>(v.hdr)[tid] = tid == 0 ? 0x800000007FFFFFFFull : 0ull;
    reinterpret_cast<uint64_t*>(v.jhdr)[tid] = 0;
  }
  for (int64_t i = tid; i < v.words; i += stride) v.bits[i] = 0;
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  for (int64_t i = tid; i < jpairs; i += stride) reinterpret_cast<ulonglong2*>(v.jslots)[i] = ones;
}

// Range of the qualifying rows' one-column keys.
__global__ void semi_minmax_kernel(SemiInput in, SemiHeader* h) {
  int32_t lo = INT32_MAX, hi = INT32_MIN;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < in.m; j += (int64_t)gridDim.x * blockDim.x) {
    if (!semi_row_qualifies(in, j)) continue;
    const int32_t k = in.pk[j];
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&h->key_min, lo);
    atomicMax(&h->key_max, hi);
  }
}

// Enters the qualifying rows' keys: into the bitmap when they are one column and their range
// spans at most 32 bits per dim row (also when no row qualifies: an empty range), else into
// the hash set (payload 0).
template <bool kWide>
__global__ void semi_build_kernel(SemiInput in, SemiView v) {
  const int64_t range = (int64_t)v.hdr->key_max - (int64_t)v.hdr->key_min + 1;
  const bool bitmap = !kWide && range <= 32 * (v.words - 2);
  const int32_t kmin = v.hdr->key_min;
  if (blockIdx.x == 0 && threadIdx.x == 0) v.hdr->bitmap = bitmap ? 1u : 0u;
  bool dup = false;  // duplicate keys change nothing in a membership test
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < in.m; j += (int64_t)gridDim.x * blockDim.x) {
    if (!semi_row_qualifies(in, j)) continue;
    if (kWide) {
      join_insert64((ulonglong2*)v.jslots, v.jcap, pack_key64(in.pk_hi[j], in.pk[j]), 0u, dup);
    } else if (bitmap) {
      const uint32_t k = (uint32_t)in.pk[j] - (uint32_t)kmin;
      atomicOr(&v.bits[k >> 5], 1u << (k & 31));
    } else {
      const uint32_t key = (uint32_t)in.pk[j];
      join_insert32((uint64_t*)v.jslots, v.jcap, key, (uint64_t)key, dup);
    }
  }
}

// kFresh: the build ran earlier in the same launch (the single-launch kernel): its headers and
// tables are read through L2 only.  Every thread of the block takes part.
// kBounded: the second phase of a split pass (one-column keys, hot-group cache or plain
// reductions; a.bounds set).
template <bool kWide, int kMode, bool kVec, bool kSemi, bool kFresh = false, bool kBounded = false>
__device__ __forceinline__ void probe_body(const ProbeArgs& a, const SemiArgs& sa) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int32_t dstatus = kFresh ? *(const volatile int32_t*)&a.dhdr->status : a.dhdr->status;
  if (dstatus != 0) return;  // the build failed: nothing to aggregate
  const Lookup L = read_lookup<kFresh>(a);
  // star query: the filter dims' lookups live in shared memory (read where used), not registers
  const SemiLookups* SLp = nullptr;
  if constexpr (kSemi) {
    __shared__ SemiLookups s_sl;
    if (threadIdx.x == 0) read_semi_lookup(sa, s_sl);
    __syncthreads();
    SLp = &s_sl;
  }
  const uint32_t slots = kMode == kAggSmem ? a.gslots : (kMode == kAggHot ? (uint32_t)kHotEntries : 0u);
  const SmemAggs T = smem_aggs(smem_raw, slots);
  if constexpr (kBounded) {
    // second phase of a split pass: the bounds into shared memory after the hot-group cache,
    // the extremes decoded (the hot-group cache's barrier below, or this one, publishes them)
    const uint4* src = reinterpret_cast<const uint4*>(a.bounds);
    uint4* dst = reinterpret_cast<uint4*>(smem_raw + (kMode == kAggHot ? kHotSmemBytes : 0));
    for (uint32_t i = threadIdx.x; i < kBoundsSmemBytes / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
      s_bound_floor = bound_decode(a.bounds->max_floor_enc);
      s_bound_ceil = bound_decode(~a.bounds->min_ceil_inv);
    }
    if (kMode == kAggGlobal) __syncthreads();
  }
  if (kMode == kAggSmem || kMode == kAggHot) {
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
      smem_identity(T, i);
      if (kMode == kAggHot) T.tag[i] = kEmpty32;
    }
    __syncthreads();
  }
  const int64_t nq = a.n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if constexpr ((kFresh || kBounded) && kVec && !kWide && !kSemi) {
    // two quads in flight per thread: the single launch (one block per SM, registers to spare)
    // and the second phase of a split pass (latency-bound once its L2 reductions are cut;
    // measured 3.44 -> 3.31 ms on the 600M-row query)
    if (L.direct)
      for (; q + stride < nq; q += 2 * stride) probe_quad_pair_direct<kMode, kFresh, kBounded>(a, T, L, q, q + stride);
  }
  for (; q < nq; q += stride) probe_quad<kWide, kMode, kVec, kSemi, false, kFresh, kBounded>(a, T, L, q, SLp);
  // ragged tail: the last n % 4 rows, one per thread of block 0
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < a.n - (nq << 2))
    probe_one<kWide, kMode, kSemi, kFresh>(a, T, L, (nq << 2) + threadIdx.x, SLp);
  if (kMode == kAggSmem || kMode == kAggHot) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
      if (kMode == kAggSmem) smem_merge(T, i, &a.tab[i], a.aggs);
      else if (T.tag[i] != kEmpty32) smem_merge(T, i, &a.tab[T.tag[i]], a.aggs);
    }
  }
}

// The fused probe pass: filter, probe and aggregate every fact row.  Held to 64 registers, so
// that two 512-thread blocks share an SM: the pass needs the resident warps to cover its
// memory latency (a 76-register build of the two-column-key variant ran one block per SM and
// took 15.0 ms instead of 8.4 on the 600M-row query).
template <bool kWide, int kMode, bool kVec, bool kSemi, bool kBounded = false>
__global__ void __launch_bounds__(512, 2)
probe_kernel(ProbeArgs a, SemiArgs sa) {
  probe_body<kWide, kMode, kVec, kSemi, false, kBounded>(a, sa);
}

// The same pass for a star query, held to 64 registers so that two 512-thread blocks share an
// SM: its filter dims add dependent reads per row, and it needs the resident warps to cover them.
template <bool kWide, int kMode, bool kVec>
__global__ void __launch_bounds__(512, 2)
probe_star_kernel(ProbeArgs a, SemiArgs sa) {
  probe_body<kWide, kMode, kVec, true>(a, sa);
}

// kFresh: the group table and its aggregates were written earlier in the same launch (read
// through L2 only).  Every thread of every block takes part.
template <bool kFresh = false>
__device__ __forceinline__ void finalize_body(const int64_t* __restrict__ gkeys, const Agg* __restrict__ tab,
                                              int64_t gslots, const DimHeader* __restrict__ dhdr, const PipeOut& out,
                                              PipeHeader* phdr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (gslots + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < gslots && (kFresh ? __ldcg(&tab[i].count) : tab[i].count) > 0;
    const uint64_t pos = warp_append(&phdr->groups, occ);
    if (occ && (int64_t)pos < out.cap) {
      Agg t;
      if (kFresh) {
        t.sum = __ldcg(&tab[i].sum);
        t.count = __ldcg(&tab[i].count);
        t.min = __ldcg(&tab[i].min);
        t.max = __ldcg(&tab[i].max);
      } else {
        t = tab[i];
      }
      if (out.keys) out.keys[pos] = kFresh ? __ldcg(&gkeys[i]) : gkeys[i];
      if (out.sum) out.sum[pos] = (int64_t)t.sum;
      if (out.count) out.count[pos] = (int64_t)t.count;
      if (out.min) out.min[pos] = t.min;
      if (out.max) out.max[pos] = t.max;
    }
  }
  // the last block to finish publishes G and the status
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&phdr->blocks_done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned long long g = *(volatile unsigned long long*)&phdr->groups;
      int32_t st = *(volatile const int32_t*)&dhdr->status;
      if (st == 0) st = *(volatile const int32_t*)&phdr->status;  // probe-pass errors (TIMEOUT)
      if (st == 0 && (int64_t)g > out.cap) st = SIRIUS_ERR_CAPACITY;
      phdr->status = st;
      if (out.d_groups) *out.d_groups = (int64_t)g;
      if (out.d_status) *out.d_status = st;
    }
  }
}
__global__ void finalize_kernel(const int64_t* __restrict__ gkeys, const Agg* __restrict__ tab, int64_t gslots,
                                const DimHeader* __restrict__ dhdr, PipeOut out, PipeHeader* phdr) {
  finalize_body(gkeys, tab, gslots, dhdr, out, phdr);
}

// ------------------------------------------------------------------ single-launch pipeline
// A small query is latency-bound: its seven phase kernels (clear, key range, build, fallback,
// run clear, probe, finalize) each take a few microseconds of dependent memory round trips
// and launch gaps, far more than its bytes need.  The single-launch form runs the same phases
// in one cooperative launch (every block resident), separated by grid-wide barriers, so no
// phase waits for a kernel boundary.  Tables written by one phase and read by a later one are
// read through L2 only (volatile header reads, ld.global.cg table reads): another SM's L1 or
// read-only cache may hold a line from before the write.
struct SingleArgs {
  const int32_t* pk;
  const int32_t* pk_hi;
  const int32_t* grp;
  const int8_t* flag;
  int64_t m;
  DimPred P;
  DimView d;
  unsigned long long glimit;
  int64_t jpairs, dpairs, bwords;  // extents the clearing phase covers (16-byte pairs, words)
  ProbeArgs a;                     // the probe pass (a.tab = the run's aggregates)
  PipeHeader* phdr;                // cleared by the caller (it holds the barrier counter)
  PipeOut out;
};

template <bool kWide, int kMode, bool kVec>
__global__ void __launch_bounds__(512, 1)
single_query_kernel(SingleArgs g) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t* bar = reinterpret_cast<uint32_t*>(&g.phdr->pad[0]);
  int32_t* status = &g.phdr->status;
  uint32_t passed = 0;
  const DimView& d = g.d;
  // 1. clear the dim index (headers, join slots, direct array, group keys, Bloom words) and
  //    the run's aggregates; the run header was cleared before the launch
  dim_init_rows(d.dhdr, d.jhdr, (ulonglong2*)d.jslots, g.jpairs, (ulonglong2*)d.dslot, g.dpairs, d.gkeys,
                (int64_t)d.gcap + 1, d.bloom, g.bwords, tid, stride);
  for (int64_t i = tid; i < (int64_t)g.a.gslots; i += stride) agg_identity(&g.a.tab[i]);
  if (!grid_barrier(bar, ++passed * gridDim.x, status)) return;
  if (g.m > 0) {
    // 2. ranges of the build keys and of the group keys (the direct-array and direct group-slot
    //    decisions)
    dim_minmax_rows(g.pk, g.grp, g.flag, g.m, d.dhdr, tid, stride);
    if (!grid_barrier(bar, ++passed * gridDim.x, status)) return;
    // 3. build
    const volatile DimHeader* vh = d.dhdr;
    const BuildMode B = read_build_mode<true>(d, g.m, g.glimit, !kWide);
    dim_build_rows<kWide>(g.pk, g.pk_hi, g.grp, g.flag, g.m, d, g.glimit, g.P, B, tid, stride);
    if (!grid_barrier(bar, ++passed * gridDim.x, status)) return;
    // 4. a duplicate key turned the direct array down: every row into the (cleared) hash table
    if (!kWide && vh->direct && vh->direct_failed) {
      dim_fallback_rows(g.pk, g.grp, g.flag, g.m, d, g.glimit, g.P, B, tid, stride);
      if (!grid_barrier(bar, ++passed * gridDim.x, status)) return;
    }
    // 5. filter, probe and aggregate the fact rows
    if (g.a.n > 0) {
      probe_body<kWide, kMode, kVec, false, true>(g.a, SemiArgs{});
      if (!grid_barrier(bar, ++passed * gridDim.x, status)) return;
    }
  }
  // 6. compact the occupied group slots into the outputs; the last block publishes G and status
  finalize_body<true>(d.gkeys, g.a.tab, (int64_t)g.a.gslots, d.dhdr, g.out, g.phdr);
}

// Self-test of the grid barrier's bounded wait: the blocks of a small cooperative launch
// arrive, and wait for `target` arrivals; a target above the block count is a wait nothing can
// satisfy, which must run out and record SIRIUS_ERR_TIMEOUT.  Blocks that pass count themselves
// in blocks_done.
__global__ void barrier_selftest_kernel(PipeHeader* phdr, uint32_t target, uint32_t max_spins) {
  uint32_t* bar = reinterpret_cast<uint32_t*>(&phdr->pad[0]);
  if (!grid_barrier(bar, target, &phdr->status, max_spins)) return;
  if (threadIdx.x == 0) atomicAdd(&phdr->blocks_done, 1u);
}

template <typename K>
int occupancy_blocks(K kernel, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return b > 0 ? b : 1;
}

template <bool kWide, int kMode, bool kVec, bool kSemi, bool kBounded = false>
sirius_status launch_probe(const ProbeArgs& a, const SemiArgs& sa, int threads, int blocks_per_sm, size_t smem,
                           cudaStream_t s) {
  void (*k)(ProbeArgs, SemiArgs);
  if constexpr (kSemi) k = probe_star_kernel<kWide, kMode, kVec>;
  else k = probe_kernel<kWide, kMode, kVec, false, kBounded>;
  if (kMode == kAggSmem || kMode == kAggHot) {
    static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
    SIRIUS_CUDA_TRY(ensure_smem_limit(k, 200 * 1024, smem_set));
  }
  int per_sm = blocks_per_sm;
  if (per_sm <= 0) {
    // residency depends on the block size (and on the shared-memory table when there is one)
    static int occ_by_warps[17] = {};
    if (kMode == kAggSmem || kMode == kAggHot) {
      per_sm = occupancy_blocks(k, threads, smem);
    } else {
      int& c = occ_by_warps[(threads / 32) & 15];
      if (c == 0) c = occupancy_blocks(k, threads, 0);
      per_sm = c;
    }
  }
  int64_t want = ((a.n >> 2) + threads - 1) / threads;
  if (want < 1) want = 1;
  int64_t g = (int64_t)sm_count() * per_sm;
  if (g > want) g = want;
  k<<<(unsigned)g, threads, smem, s>>>(a, sa);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

// Partitioned aggregation: pass 1 fused with filter and probe, then pass 2 per partition.
template <bool kWide>
sirius_status launch_part(const ProbeArgs& a, const part::PartArgs& pa, bool vec, cudaStream_t s) {
  static int per_sm = 0;
  auto k1 = vec ? part::part_scatter_kernel<kWide, true> : part::part_scatter_kernel<kWide, false>;
  if (per_sm == 0) per_sm = occupancy_blocks(k1, part::kScatterThreads, 0);
  int64_t g1 = (int64_t)sm_count() * per_sm;
  if (g1 > pa.ntiles) g1 = pa.ntiles;
  if (g1 < 1) g1 = 1;
  {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_PROBE);
    k1<<<(unsigned)g1, part::kScatterThreads, 0, s>>>(a, pa);
    SIRIUS_LAUNCH_CHECK();
  }
  PhaseTimer pt2(s, SIRIUS_PHASE_PIPE_AGGREGATE);
  const size_t smem = (size_t)part::kPartSlots * sizeof(Agg);
  static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(part::part_agg_kernel, (int)smem, smem_set));
  // about three waves of one block per SM over all partitions
  int64_t kb = ((int64_t)sm_count() * 3 + pa.parts - 1) / pa.parts;
  if (kb < 1) kb = 1;
  const int64_t per = (pa.ntiles + kb - 1) / kb;
  kb = (pa.ntiles + per - 1) / per;
  if (kb < 1) kb = 1;
  part::part_agg_kernel<<<dim3((unsigned)kb, (unsigned)pa.parts), part::kAggThreads, smem, s>>>(
      pa, a.tab, a.gslots, a.aggs, per);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

template <bool kWide>
sirius_status launch_staged(const ProbeArgs& a, PipeHeader* phdr, cudaStream_t s) {
  auto k = staged::probe_staged_kernel<kWide>;
  const size_t smem = staged::smem_bytes(kWide);
  static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(k, (int)smem, smem_set));
  const int64_t tiles = (((a.n >> 2) << 2) + staged::kTile - 1) / staged::kTile;
  int64_t g = sm_count();
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  k<<<(unsigned)g, staged::kThreads, smem, s>>>(a, &phdr->status);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

// The routed probe: one cooperative launch of every resident block (the exchange was sized for
// r.route_blocks); its barrier counter is cleared first.
template <bool kWide>
sirius_status launch_routed(const ProbeArgs& a, const RunView& r, bool vec, cudaStream_t s) {
  auto k = vec ? routed::probe_routed_kernel<kWide, true> : routed::probe_routed_kernel<kWide, false>;
  const size_t smem = routed::smem_bytes(r.route_R);
  SIRIUS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int per_sm = occupancy_blocks(k, routed::kThreads, smem);
  int blocks = sm_count() * (per_sm < routed::kBlocksPerSm ? per_sm : routed::kBlocksPerSm);
  if (blocks > r.route_blocks) blocks = r.route_blocks;
  // fewer resident blocks than planned: fewer owners, each with a larger share (the exchange,
  // sized for the plan, holds the smaller plan: P' x B' x C' <= P x B x C)
  int logP = r.route_logP;
  while (logP > 0 && (1 << logP) > blocks) --logP;
  const int64_t R = ((int64_t)a.gslots + (1 << logP) - 1) >> logP;
  if (logP != r.route_logP && (R > (int64_t)routed::kMaxOwnerSlots || routed::smem_bytes((uint32_t)R) > smem)) {
    set_error("pipeline: routed aggregation needs %d resident blocks, %d fit", r.route_blocks, blocks);
    return SIRIUS_ERR_INVALID;
  }
  routed::RouteArgs ra;
  ra.tval = r.rval;
  ra.tls = r.rls;
  ra.fill = r.rfill;
  ra.bar = reinterpret_cast<uint32_t*>(&r.phdr->pad[1]);
  ra.status = &r.phdr->status;
  ra.logP = logP;
  ra.R = (uint32_t)R;
  ra.C = routed::run_capacity(1 << logP, routed::kIters);
  ra.iters = routed::kIters;
  const int64_t per_round = (int64_t)blocks * routed::kIters * routed::kThreads;  // quads
  ra.rounds = ((a.n >> 2) + per_round - 1) / per_round;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(ra.bar, 0, sizeof(uint32_t), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)routed::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SIRIUS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, a, ra));
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

template <bool kWide, bool kSemi>
sirius_status dispatch_probe(const ProbeArgs& a, const SemiArgs& sa, int mode, bool vec, int threads, int bps,
                             size_t smem, cudaStream_t s) {
  if (mode == kAggSmem)
    return vec ? launch_probe<kWide, kAggSmem, true, kSemi>(a, sa, threads, bps, smem, s)
               : launch_probe<kWide, kAggSmem, false, kSemi>(a, sa, threads, bps, smem, s);
  if constexpr (!kWide && !kSemi) {
    if (a.bounds) {  // second phase of a split pass: the bounds' copy follows the hot-group cache
      constexpr size_t bb = kBoundsSmemBytes;
      if (mode == kAggHot)
        return vec ? launch_probe<false, kAggHot, true, false, true>(a, sa, threads, bps, kHotSmemBytes + bb, s)
                   : launch_probe<false, kAggHot, false, false, true>(a, sa, threads, bps, kHotSmemBytes + bb, s);
      return vec ? launch_probe<false, kAggGlobal, true, false, true>(a, sa, threads, bps, bb, s)
                 : launch_probe<false, kAggGlobal, false, false, true>(a, sa, threads, bps, bb, s);
    }
  }
  if (mode == kAggHot)
    return vec ? launch_probe<kWide, kAggHot, true, kSemi>(a, sa, threads, bps, kHotSmemBytes, s)
               : launch_probe<kWide, kAggHot, false, kSemi>(a, sa, threads, bps, kHotSmemBytes, s);
  return vec ? launch_probe<kWide, kAggGlobal, true, kSemi>(a, sa, threads, bps, 0, s)
             : launch_probe<kWide, kAggGlobal, false, kSemi>(a, sa, threads, bps, 0, s);
}

// The single-launch pipeline: the run header is cleared (it holds the grid barrier's counter),
// then one cooperative launch of `per_sm` blocks per SM (at most the resident maximum), fewer
// when the query has less work than that.
template <bool kWide, int kMode, bool kVec>
sirius_status launch_single(const SingleArgs& g, int threads, int per_sm, size_t smem, cudaStream_t s) {
  auto k = single_query_kernel<kWide, kMode, kVec>;
  static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(k, 200 * 1024, smem_set));
  // One block per SM (the default) always fits: 512 threads at the 128 registers the launch
  // bound allows, and the shared memory raised above; only a larger request asks the runtime
  // (a query per call would add its host time to every small query).
  if (per_sm <= 0) per_sm = 1;
  if (per_sm > 1) {
    const int occ = occupancy_blocks(k, threads, smem);
    if (per_sm > occ) per_sm = occ;
  }
  int64_t work = (g.a.n >> 2) > g.m ? (g.a.n >> 2) : g.m;
  const int64_t other[4] = {g.jpairs, g.dpairs, (int64_t)g.a.gslots, g.bwords};
  for (int64_t w : other) work = w > work ? w : work;
  int64_t grid = (work + threads - 1) / threads;
  const int64_t most = (int64_t)sm_count() * per_sm;
  if (grid > most) grid = most;
  if (grid < 1) grid = 1;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(g.phdr, 0, sizeof(PipeHeader), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SIRIUS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, g));
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

template <bool kWide>
sirius_status dispatch_single(const SingleArgs& g, int mode, bool vec, int threads, int per_sm, size_t smem,
                              cudaStream_t s) {
  if (mode == kAggSmem)
    return vec ? launch_single<kWide, kAggSmem, true>(g, threads, per_sm, smem, s)
               : launch_single<kWide, kAggSmem, false>(g, threads, per_sm, smem, s);
  if (mode == kAggHot)
    return vec ? launch_single<kWide, kAggHot, true>(g, threads, per_sm, kHotSmemBytes, s)
               : launch_single<kWide, kAggHot, false>(g, threads, per_sm, kHotSmemBytes, s);
  return vec ? launch_single<kWide, kAggGlobal, true>(g, threads, per_sm, 0, s)
             : launch_single<kWide, kAggGlobal, false>(g, threads, per_sm, 0, s);
}

}  // namespace

// ------------------------------------------------------------------ layouts and validation
DimLayout dim_layout(int64_t m, bool wide, int64_t hint, float lf, bool allow_direct, bool bloom) {
  DimLayout L;
  L.key_width = wide ? 8 : 4;
  L.jcap = sirius_join_table_capacity(m, lf > 0 ? lf : 0.5);
  L.gcap = group_capacity_for(hint > 0 ? hint : (m > 0 ? m : 1));
  // direct array: key ranges up to 2m values (64-entry granules), one-column keys only
  L.dcap = (!wide && allow_direct && m > 0) ? ((2 * m + 63) / 64) * 64 : 0;
  L.off_join = 256;
  L.off_gkeys = align_up(L.off_join + 256 + (size_t)L.jcap * (wide ? 16 : 8), 256);
  L.off_direct = align_up(L.off_gkeys + (size_t)(L.gcap + 1) * 8, 256);
  L.off_bloom = align_up(L.off_direct + (size_t)L.dcap * 4, 256);
  // Bloom filter: 16 bits per dim row (a 64-bit word per four rows), at least 64 words
  if (bloom && m > 0) {
    L.bloom_log2 = 6;
    while ((1ll << L.bloom_log2) < (m + 3) / 4) ++L.bloom_log2;
  }
  L.total = align_up(L.off_bloom + (L.bloom_log2 > 0 ? (size_t)8 << L.bloom_log2 : 0), 256);
  return L;
}

// The Bloom filter is built when asked for (bloom = 2), or by default when a dim-side
// predicate leaves dim rows out of the join, so that probe keys often find no partner.
static bool bloom_wanted(const sirius_pipeline_desc* q) {
  return q->bloom == 2 || (q->bloom == 0 && q->dpred != nullptr);
}

DimLayout dim_layout_for(const sirius_pipeline_desc* q) {
  return dim_layout(q->m, q->pk_hi != nullptr || q->fk_hi != nullptr, q->group_cap_hint, q->load_factor,
                    q->join_mode == 0, bloom_wanted(q));
}

// The layout of a built dim index, from the capacities its build recorded.
DimLayout dim_layout_of_index(const sirius_dim_index* idx) {
  DimLayout L;
  L.key_width = idx->key_width;
  L.jcap = idx->join_capacity;
  L.gcap = idx->group_capacity;
  L.dcap = idx->direct_capacity;
  L.off_join = 256;
  L.off_gkeys = align_up(L.off_join + 256 + (size_t)L.jcap * (L.key_width == 8 ? 16 : 8), 256);
  L.off_direct = align_up(L.off_gkeys + (size_t)(L.gcap + 1) * 8, 256);
  L.off_bloom = align_up(L.off_direct + (size_t)L.dcap * 4, 256);
  L.bloom_log2 = idx->bloom_log2;
  L.total = align_up(L.off_bloom + (L.bloom_log2 > 0 ? (size_t)8 << L.bloom_log2 : 0), 256);
  return L;
}

RunLayout run_layout(int64_t gcap, int64_t n, int agg_mode, bool bounds) {
  RunLayout R;
  R.gslots = gcap + 1;
  R.mode = choose_mode(agg_mode, R.gslots, n);
  R.off_aggs = 256;
  size_t end = align_up(R.off_aggs + (size_t)R.gslots * sizeof(Agg), 256);
  if (R.mode == kAggRouted) {
    const RoutePlan rp = route_plan(R.gslots);
    R.route_blocks = rp.blocks;
    R.route_logP = rp.logP;
    R.route_R = rp.R;
    R.route_C = rp.C;
    const size_t tuples = (size_t)2 * ((size_t)1 << rp.logP) * rp.blocks * rp.C;
    R.off_rval = end;
    R.off_rls = align_up(R.off_rval + tuples * 8, 256);
    R.off_rfill = align_up(R.off_rls + tuples * 2, 256);
    end = align_up(R.off_rfill + (size_t)2 * rp.blocks * ((size_t)1 << rp.logP) * 4, 256);
  }
  if (R.mode == kAggPart) {
    R.parts = part::parts_for(R.gslots);
    R.ntiles = part::tiles_for(n);
    const size_t tuples = (size_t)R.ntiles * part::kPartTile;
    R.off_tgs = end;
    R.off_tval = align_up(R.off_tgs + tuples * 4, 256);
    R.off_prefix = align_up(R.off_tval + tuples * 8, 256);
    end = align_up(R.off_prefix + (size_t)R.ntiles * (R.parts + 1) * 4, 256);
  }
  if (bounds && (R.mode == kAggHot || R.mode == kAggGlobal)) {
    R.off_bounds = end;
    end = align_up(end + sizeof(ExtremeBounds), 256);
  }
  R.total = end;
  return R;
}

DimView dim_view(const DimLayout& L, char* base) {
  DimView d;
  d.dhdr = (DimHeader*)base;
  d.jhdr = (JoinHeader*)(base + L.off_join);
  d.jslots = base + L.off_join + 256;
  d.gkeys = (int64_t*)(base + L.off_gkeys);
  d.dslot = (uint32_t*)(base + L.off_direct);
  d.bloom = L.bloom_log2 > 0 ? (uint64_t*)(base + L.off_bloom) : nullptr;
  d.bloom_mask = L.bloom_log2 > 0 ? (uint32_t)((1ull << L.bloom_log2) - 1) : 0u;
  d.jcap = (uint32_t)L.jcap;
  d.gcap = (uint32_t)L.gcap;
  d.dcap = L.dcap;
  d.key_width = L.key_width;
  return d;
}

RunView run_view(const RunLayout& R, char* base) {
  RunView r;
  r.phdr = (PipeHeader*)base;
  r.aggs = (Agg*)(base + R.off_aggs);
  r.mode = R.mode;
  r.parts = R.parts;
  r.ntiles = R.ntiles;
  const bool rt = R.mode == kAggRouted;
  r.rval = rt ? (int64_t*)(base + R.off_rval) : nullptr;
  r.rls = rt ? (uint16_t*)(base + R.off_rls) : nullptr;
  r.rfill = rt ? (uint32_t*)(base + R.off_rfill) : nullptr;
  r.route_blocks = R.route_blocks;
  r.route_logP = R.route_logP;
  r.route_R = R.route_R;
  r.route_C = R.route_C;
  r.tgs = R.mode == kAggPart ? (uint32_t*)(base + R.off_tgs) : nullptr;
  r.tval = R.mode == kAggPart ? (int64_t*)(base + R.off_tval) : nullptr;
  r.prefix = R.mode == kAggPart ? (int32_t*)(base + R.off_prefix) : nullptr;
  r.bounds = R.off_bounds ? (ExtremeBounds*)(base + R.off_bounds) : nullptr;
  return r;
}

sirius_status validate_dim(const sirius_pipeline_desc* q) {
  SIRIUS_REQUIRE(q, "pipeline: NULL descriptor");
  SIRIUS_REQUIRE(q->m >= 0 && q->m <= kMaxRows, "pipeline: m=%lld out of range", (long long)q->m);
  SIRIUS_REQUIRE(q->m == 0 || (q->pk && q->grp), "pipeline: NULL dim column");
  SIRIUS_REQUIRE(q->load_factor >= 0 && q->load_factor <= 0.95f, "pipeline: load_factor out of (0, 0.95]");
  const int64_t hint = q->group_cap_hint > 0 ? q->group_cap_hint : q->m;
  SIRIUS_REQUIRE(hint < (1ll << 30), "pipeline: group_cap_hint too large");
  SIRIUS_REQUIRE(q->join_mode == 0 || q->join_mode == 1, "pipeline: bad join_mode %d", q->join_mode);
  SIRIUS_REQUIRE(!q->dpred || (q->dop >= 0 && q->dop <= 5), "pipeline: bad dim comparison %d", q->dop);
  SIRIUS_REQUIRE(q->bloom >= 0 && q->bloom <= 2, "pipeline: bad bloom %d", q->bloom);
  return SIRIUS_OK;
}

sirius_status validate_fact(const sirius_pipeline_desc* q) {
  SIRIUS_REQUIRE(q, "pipeline: NULL descriptor");
  SIRIUS_REQUIRE(q->n >= 0 && q->n <= kMaxRows, "pipeline: n=%lld out of range", (long long)q->n);
  SIRIUS_REQUIRE(q->n == 0 || (q->fk && q->pred && q->val), "pipeline: NULL fact column");
  SIRIUS_REQUIRE(q->op >= SIRIUS_LT && q->op <= SIRIUS_NE, "pipeline: bad comparison %d", q->op);
  SIRIUS_REQUIRE(q->aggs <= SIRIUS_AGG_ALL, "pipeline: bad aggregate mask");
  SIRIUS_REQUIRE(q->agg_mode >= 0 && q->agg_mode <= kAggRouted, "pipeline: bad agg_mode %d", q->agg_mode);
  SIRIUS_REQUIRE(q->split_probe >= 0 && q->split_probe <= 2, "pipeline: bad split_probe %d", q->split_probe);
  SIRIUS_REQUIRE(q->block_threads == 0 || (q->block_threads % 32 == 0 && q->block_threads >= 64 &&
                                           q->block_threads <= 512),
                 "pipeline: block_threads must be a multiple of 32 in [64, 512]");
  SIRIUS_REQUIRE(q->blocks_per_sm >= 0 && q->blocks_per_sm <= 32, "pipeline: blocks_per_sm out of range");
  SIRIUS_REQUIRE(q->probe_variant >= 0 && q->probe_variant <= 3, "pipeline: bad probe_variant %d",
                 q->probe_variant);
  return SIRIUS_OK;
}

static sirius_status validate_pair(const sirius_pipeline_desc* q) {
  sirius_status st = validate_dim(q);
  if (st != SIRIUS_OK) return st;
  st = validate_fact(q);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE((q->fk_hi == nullptr) == (q->pk_hi == nullptr) || q->n == 0 || q->m == 0,
                 "pipeline: fact and dim keys must both be one- or two-column");
  return SIRIUS_OK;
}

// Shared-memory table when the group table fits a block; otherwise partitioned aggregation
// for large inputs whose group table has at most kMaxParts partitions; otherwise reductions.
// The routed probe's plan for a group table of gslots slots: the blocks of its cooperative
// launch (all resident), owners = the largest power of two not above min(blocks, 256), slots
// per owner, run capacity.  R = 0 when the owners' shares do not fit shared memory.
RoutePlan route_plan(int64_t gslots) {
  RoutePlan p;
  p.blocks = sm_count() * routed::kBlocksPerSm;
  int P = 1, logP = 0;
  while (2 * P <= p.blocks && 2 * P <= routed::kMaxOwners) {
    P *= 2;
    ++logP;
  }
  p.logP = logP;
  const int64_t R = (gslots + P - 1) / P;
  p.R = R <= (int64_t)routed::kMaxOwnerSlots ? (uint32_t)R : 0u;
  p.C = routed::run_capacity(P, routed::kIters);
  return p;
}

int choose_mode(int agg_mode, int64_t gslots, int64_t n) {
  const bool fits = (int64_t)smem_aggs_bytes((uint32_t)(gslots < (1 << 30) ? gslots : (1 << 30)), false) <= kSmemAggMaxBytes;
  const bool part_ok = gslots <= (int64_t)part::kMaxParts * part::kPartSlots && n > 0;
  if (agg_mode == kAggSmem && fits) return kAggSmem;
  if (agg_mode == kAggGlobal) return kAggGlobal;
  if (agg_mode == kAggPart) return part_ok ? kAggPart : kAggGlobal;
  if (agg_mode == kAggHot) return n > 0 ? kAggHot : kAggGlobal;
  if (agg_mode == kAggRouted) return (n > 0 && route_plan(gslots).R > 0) ? kAggRouted : (n > 0 ? kAggHot : kAggGlobal);
  if (fits) return kAggSmem;
  // large group tables: the hot-group cache (measured: skewed 300M-row query 38.5 -> 3.3 ms,
  // uniform 600M-row query 5.31 -> 5.15 ms against plain reductions)
  return n >= (1 << 20) ? kAggHot : kAggGlobal;
}

// ------------------------------------------------------------------ host phases
sirius_status dim_build(const sirius_pipeline_desc* q, const DimLayout& L, char* base, cudaStream_t s) {
  DimView d = dim_view(L, base);
  const int64_t jpairs = (L.jcap * (L.key_width == 8 ? 16 : 8) + 15) / 16;
  const int64_t dpairs = L.dcap / 4;
  const int64_t gslots = L.gcap + 1;
  // a large join table is cleared only once the build knows the hash table is needed
  const bool lazy_join = L.dcap > 0 && jpairs * 16 > (16ll << 20);
  {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_INIT);
    const int64_t init_jpairs = lazy_join ? 0 : jpairs;
    int64_t work = init_jpairs > gslots ? init_jpairs : gslots;
    work = dpairs > work ? dpairs : work;
    const int64_t bwords = L.bloom_log2 > 0 ? (1ll << L.bloom_log2) : 0;
    work = bwords > work ? bwords : work;
    dim_init_kernel<<<grid_for(work, 256), 256, 0, s>>>(d.dhdr, d.jhdr, (ulonglong2*)d.jslots, init_jpairs,
                                                       (ulonglong2*)d.dslot, dpairs, d.gkeys, gslots, d.bloom,
                                                       bwords);
    SIRIUS_LAUNCH_CHECK();
  }
  if (q->m > 0) {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_BUILD);
    const int g = grid_for(q->m, 256);
    const unsigned long long lim = group_limit_for(L.gcap);
    const DimPred P{q->dpred, q->dop, q->dliteral};
    dim_minmax_kernel<<<g, 256, 0, s>>>(q->pk, q->grp, q->flag, q->m, d.dhdr);
    SIRIUS_LAUNCH_CHECK();
    if (L.key_width == 8) {
      dim_build_kernel<true><<<g, 256, 0, s>>>(q->pk, q->pk_hi, q->grp, q->flag, q->m, d, lim, P);
      SIRIUS_LAUNCH_CHECK();
    } else {
      if (L.dcap > 0) {
        if (lazy_join) {
          dim_clear_join_kernel<<<grid_for(jpairs, 256), 256, 0, s>>>(d, q->m, 0, jpairs);
          SIRIUS_LAUNCH_CHECK();
        }
      }
      dim_build_kernel<false><<<g, 256, 0, s>>>(q->pk, nullptr, q->grp, q->flag, q->m, d, lim, P);
      SIRIUS_LAUNCH_CHECK();
      if (L.dcap > 0) {
        if (lazy_join) {
          dim_clear_join_kernel<<<grid_for(jpairs, 256), 256, 0, s>>>(d, q->m, 1, jpairs);
          SIRIUS_LAUNCH_CHECK();
        }
        dim_fallback_kernel<<<g, 256, 0, s>>>(q->pk, q->grp, q->flag, q->m, d, lim, P);
        SIRIUS_LAUNCH_CHECK();
      }
    }
  }
  return SIRIUS_OK;
}

sirius_status run_init(const RunLayout& R, char* base, cudaStream_t s) {
  RunView r = run_view(R, base);
  PhaseTimer pt(s, SIRIUS_PHASE_PIPE_INIT);
  run_init_kernel<<<grid_for(R.gslots, 256), 256, 0, s>>>(r.phdr, r.aggs, R.gslots);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

static ProbeArgs probe_args(const sirius_pipeline_desc* q, const DimView& d, const RunView& r, int64_t gslots) {
  ProbeArgs a;
  a.fk = q->fk;
  a.fk_hi = q->fk_hi;
  a.pred = q->pred;
  a.val = q->val;
  a.n = q->n;
  a.op = q->op;
  a.lit = q->literal;
  a.aggs = q->aggs;
  a.jcap = d.jcap;
  a.jslots = d.jslots;
  a.jhdr = d.jhdr;
  a.dhdr = d.dhdr;
  a.dslot = d.dslot;
  a.bloom = d.bloom;
  a.bloom_mask = d.bloom_mask;
  a.tab = r.aggs;
  a.gslots = (uint32_t)gslots;
  return a;
}

// 16-byte loads of the probe columns need every one 16-byte aligned.
// The split probe pass, for queries with one-column keys that ask for MIN or MAX, aggregated
// with the hot-group cache or plain reductions (not the star kernel: its probe keeps one pass):
// when the descriptor's split_probe asks for it, or by default for large queries with many rows
// per group slot and no dim-side predicate.  The first 1/kSplitFirstDiv of the rows give every
// frequent group enough rows that the bounds rule out most later MIN / MAX reductions.  Only the
// direct-array join takes the bounds in the second phase; a hash-table join runs it with plain
// reductions.
constexpr int64_t kSplitMinRows = 1ll << 26;
constexpr int64_t kSplitRowsPerSlot = 256;
constexpr int64_t kSplitFirstDiv = 16;
static bool split_applies(const sirius_pipeline_desc* q, const DimView& d, const RunView& r, int mode,
                          int64_t gslots) {
  if (q->split_probe == 1 || r.bounds == nullptr || d.key_width != 4 || (mode != kAggHot && mode != kAggGlobal) ||
      (q->aggs & (SIRIUS_AGG_MIN | SIRIUS_AGG_MAX)) == 0 || q->n < 64)
    return false;
  if (q->split_probe == 2) return true;
  // auto: large queries with many rows per group slot, whose pass is bound by the reductions (a
  // dim-side predicate leaves few joined rows: the column stream bounds those passes; a forced
  // hash-table join takes no bounds)
  return q->n >= kSplitMinRows && q->n >= kSplitRowsPerSlot * gslots && q->dpred == nullptr && q->join_mode == 0;
}

static bool vec_columns(const sirius_pipeline_desc* q) {
  return ((uintptr_t)q->pred & 15) == 0 && ((uintptr_t)q->fk & 15) == 0 &&
         (!q->fk_hi || ((uintptr_t)q->fk_hi & 15) == 0);
}

sirius_status run_probe(const sirius_pipeline_desc* q, const DimView& d, const RunView& r, int64_t gslots,
                        cudaStream_t s, const SemiView* semi, int nsemi) {
  if (q->n == 0) return SIRIUS_OK;
  const ProbeArgs a = probe_args(q, d, r, gslots);
  SemiArgs sa;
  sa.nsemi = nsemi;
  for (int i = 0; i < kMaxSemi; ++i) sa.semi[i] = i < nsemi ? semi[i] : SemiView{};
  const int mode = (r.mode == kAggRouted && nsemi > 0) ? kAggHot : r.mode;
  bool vec = vec_columns(q);
  for (int i = 0; i < nsemi; ++i)  // a star query's key columns take the vector loads too
    vec = vec && ((uintptr_t)semi[i].fk & 15) == 0 && (!semi[i].fk_hi || ((uintptr_t)semi[i].fk_hi & 15) == 0);
  if (mode == kAggPart) {
    part::PartArgs pa{r.tgs, r.tval, r.prefix, r.ntiles, r.parts, 0};
    return d.key_width == 8 ? launch_part<true>(a, pa, vec, s) : launch_part<false>(a, pa, vec, s);
  }
  if (mode == kAggRouted && nsemi == 0) {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_PROBE);
    return d.key_width == 8 ? launch_routed<true>(a, r, vec, s) : launch_routed<false>(a, r, vec, s);
  }
  const bool staged_ok = mode == kAggGlobal && vec && ((uintptr_t)q->val & 15) == 0;
  if (staged_ok && q->probe_variant == 2 && nsemi == 0) {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_PROBE);
    return d.key_width == 8 ? launch_staged<true>(a, r.phdr, s) : launch_staged<false>(a, r.phdr, s);
  }
  const int threads = q->block_threads > 0 ? q->block_threads : (mode == kAggSmem || mode == kAggHot ? 512 : 256);
  const size_t smem = mode == kAggSmem ? smem_aggs_bytes((uint32_t)gslots, false) : 0;  // hot cache: fixed size
  PhaseTimer pt(s, SIRIUS_PHASE_PIPE_PROBE);
  if (nsemi > 0)
    return d.key_width == 8 ? dispatch_probe<true, true>(a, sa, mode, vec, threads, q->blocks_per_sm, smem, s)
                            : dispatch_probe<false, true>(a, sa, mode, vec, threads, q->blocks_per_sm, smem, s);
  auto probe = [&](const ProbeArgs& x) {
    return d.key_width == 8 ? dispatch_probe<true, false>(x, sa, mode, vec, threads, q->blocks_per_sm, smem, s)
                            : dispatch_probe<false, false>(x, sa, mode, vec, threads, q->blocks_per_sm, smem, s);
  };
  if (!split_applies(q, d, r, mode, gslots)) return probe(a);
  // Split pass: the first rows aggregate in full; then the extreme bounds over the group table
  // so far; then the other rows skip the MIN / MAX reductions those bounds rule out.
  const int64_t n0 = ((q->n / kSplitFirstDiv) >> 2) << 2;  // a multiple of 4: column alignment kept
  ProbeArgs a1 = a;
  a1.n = n0;
  sirius_status st = probe(a1);
  if (st != SIRIUS_OK) return st;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(r.bounds, 0xFF, 2 * sizeof(unsigned long long), s));
  extreme_bounds_kernel<<<kBoundSlots / 256, 256, 0, s>>>(r.aggs, (uint32_t)gslots, r.bounds);
  SIRIUS_LAUNCH_CHECK();
  ProbeArgs a2 = a;
  a2.fk = q->fk + n0;
  a2.fk_hi = q->fk_hi ? q->fk_hi + n0 : nullptr;
  a2.pred = q->pred + n0;
  a2.val = q->val + n0;
  a2.n = q->n - n0;
  a2.bounds = r.bounds;
  return probe(a2);
}

sirius_status run_finalize(const sirius_pipeline_desc* q, const DimView& d, const RunView& r, int64_t gslots,
                           const PipeOut& out, cudaStream_t s) {
  (void)q;
  PhaseTimer pt(s, SIRIUS_PHASE_PIPE_FINALIZE);
  finalize_kernel<<<grid_for(gslots, 256), 256, 0, s>>>(d.gkeys, r.aggs, gslots, d.dhdr, out, r.phdr);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

// Queries up to these sizes take the single launch by default (probe_variant 0).
constexpr int64_t kSingleMaxRows = 1ll << 22;
constexpr int64_t kSingleMaxDimRows = 1ll << 20;

// Whether sirius_run_pipeline runs the query as one launch: not for star queries or
// partitioned aggregation; always when asked for (probe_variant 3); by default when the query
// is small and no probe launch shape is forced.
static bool single_applies(const sirius_pipeline_desc* q, const RunLayout& R) {
  if (q->nsemi > 0 || R.mode == kAggPart) return false;
  if (q->probe_variant == 3) return true;
  if (q->probe_variant != 0 || q->block_threads > 0 || q->blocks_per_sm > 0) return false;
  return q->n <= kSingleMaxRows && q->m <= kSingleMaxDimRows;
}

static sirius_status run_single(const sirius_pipeline_desc* q, const DimLayout& L, const DimView& d, const RunView& r,
                                int64_t gslots, const PipeOut& out, cudaStream_t s) {
  SingleArgs g;
  g.pk = q->pk;
  g.pk_hi = q->pk_hi;
  g.grp = q->grp;
  g.flag = q->flag;
  g.m = q->m;
  g.P = DimPred{q->dpred, q->dop, q->dliteral};
  g.d = d;
  g.glimit = group_limit_for(L.gcap);
  g.jpairs = (L.jcap * (L.key_width == 8 ? 16 : 8) + 15) / 16;
  g.dpairs = L.dcap / 4;
  g.bwords = L.bloom_log2 > 0 ? (1ll << L.bloom_log2) : 0;
  g.a = probe_args(q, d, r, gslots);
  g.phdr = r.phdr;
  g.out = out;
  const int threads = q->block_threads > 0 ? q->block_threads : 512;
  const int per_sm = q->blocks_per_sm > 0 ? q->blocks_per_sm : 1;
  const size_t smem = r.mode == kAggSmem ? smem_aggs_bytes((uint32_t)gslots, false) : 0;
  PhaseTimer pt(s, SIRIUS_PHASE_PIPE_SINGLE);
  return L.key_width == 8 ? dispatch_single<true>(g, r.mode, vec_columns(q), threads, per_sm, smem, s)
                          : dispatch_single<false>(g, r.mode, vec_columns(q), threads, per_sm, smem, s);
}

sirius_status read_run_status(const RunView& r, sirius_result* res, cudaStream_t s) {
  PipeHeader h;
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, r.phdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
  res->groups = (int64_t)h.groups;
  res->status = h.status;
  if (h.status == SIRIUS_ERR_TABLE_FULL) {
    set_error("pipeline: more distinct group keys in the dim than group_cap_hint allows");
  } else if (h.status == SIRIUS_ERR_CAPACITY) {
    set_error("pipeline: %llu groups exceed out_cap %lld", h.groups, (long long)res->out_cap);
  } else if (h.status) {
    set_error("pipeline: device status %d", h.status);
  }
  return (sirius_status)h.status;
}

static PipeOut pipe_out(const sirius_result* r) {
  return PipeOut{r->keys, r->sum, r->count, r->min, r->max, r->out_cap, r->d_groups, r->d_status};
}

static sirius_status validate_result(const sirius_result* r) {
  SIRIUS_REQUIRE(r, "pipeline: NULL result");
  SIRIUS_REQUIRE(r->out_cap >= 0, "pipeline: negative out_cap");
  SIRIUS_REQUIRE(r->out_cap == 0 || r->keys || r->count, "pipeline: no output arrays");
  return SIRIUS_OK;
}

}  // namespace sirius

using namespace sirius;

// ------------------------------------------------------------------ single query
// ------------------------------------------------------------------ semi-join dims, host side
SemiLayout semi_layout(const sirius_semijoin& sj) {
  SemiLayout S;
  S.key_width = (sj.pk_hi || sj.fk_hi) ? 8 : 4;
  S.words = sj.m + 2;
  S.jcap = sirius_join_table_capacity(sj.m > 0 ? sj.m : 1, 0.5);
  S.off_bits = 256;
  S.off_join = align_up(S.off_bits + (size_t)S.words * 4, 256);
  S.total = align_up(S.off_join + 256 + (size_t)S.jcap * (S.key_width == 8 ? 16 : 8), 256);
  return S;
}

static size_t semi_bytes(const sirius_pipeline_desc* q) {
  size_t b = 0;
  for (int i = 0; i < q->nsemi && i < kMaxSemi; ++i) b += semi_layout(q->semi[i]).total;
  return b;
}

static SemiView semi_view(const SemiLayout& S, char* base, const sirius_semijoin& sj) {
  SemiView v;
  v.fk = sj.fk;
  v.fk_hi = sj.fk_hi;
  v.hdr = (SemiHeader*)base;
  v.bits = (uint32_t*)(base + S.off_bits);
  v.jhdr = (JoinHeader*)(base + S.off_join);
  v.jslots = base + S.off_join + 256;
  v.jcap = (uint32_t)S.jcap;
  v.words = S.words;
  v.key_width = S.key_width;
  return v;
}

sirius_status validate_semi(const sirius_pipeline_desc* q) {
  SIRIUS_REQUIRE(q->nsemi >= 0 && q->nsemi <= kMaxSemi, "pipeline: nsemi=%d out of [0, %d]", q->nsemi, kMaxSemi);
  for (int i = 0; i < q->nsemi; ++i) {
    const sirius_semijoin& sj = q->semi[i];
    SIRIUS_REQUIRE(sj.m >= 0 && sj.m <= kMaxRows, "pipeline: semi-join %d: m=%lld out of range", i, (long long)sj.m);
    SIRIUS_REQUIRE(sj.m == 0 || sj.pk, "pipeline: semi-join %d: NULL dim key column", i);
    SIRIUS_REQUIRE(q->n == 0 || sj.fk, "pipeline: semi-join %d: NULL fact key column", i);
    SIRIUS_REQUIRE((sj.pk_hi == nullptr) == (sj.fk_hi == nullptr) || sj.m == 0 || q->n == 0,
                   "pipeline: semi-join %d: key widths of the two sides differ", i);
    SIRIUS_REQUIRE(!sj.attr || (sj.op >= 0 && sj.op <= 5), "pipeline: semi-join %d: bad comparison %d", i, sj.op);
  }
  return SIRIUS_OK;
}

// Builds the semi-join dims into `base` (one region after another); fills views[0 .. nsemi).
static sirius_status semi_build(const sirius_pipeline_desc* q, char* base, SemiView* views, cudaStream_t s) {
  for (int i = 0; i < q->nsemi; ++i) {
    const sirius_semijoin& sj = q->semi[i];
    const SemiLayout S = semi_layout(sj);
    views[i] = semi_view(S, base, sj);
    base += S.total;
    const int64_t jpairs = (S.jcap * (S.key_width == 8 ? 16 : 8) + 15) / 16;
    const int64_t work = jpairs > S.words ? jpairs : S.words;
    semi_init_kernel<<<grid_for(work, 256), 256, 0, s>>>(views[i], jpairs);
    SIRIUS_LAUNCH_CHECK();
    if (sj.m == 0) continue;
    const SemiInput in{sj.pk, sj.pk_hi, sj.attr, sj.m, sj.op, sj.literal};
    const int g = grid_for(sj.m, 256);
    if (S.key_width == 8) {
      semi_build_kernel<true><<<g, 256, 0, s>>>(in, views[i]);
    } else {
      semi_minmax_kernel<<<g, 256, 0, s>>>(in, views[i].hdr);
      SIRIUS_LAUNCH_CHECK();
      semi_build_kernel<false><<<g, 256, 0, s>>>(in, views[i]);
    }
    SIRIUS_LAUNCH_CHECK();
  }
  return SIRIUS_OK;
}

// A star query takes neither partitioned nor routed aggregation (its probe pass is the star
// kernel): those requests run with global reductions or the hot-group cache.
static int star_agg_mode(const sirius_pipeline_desc* q) {
  if (q->nsemi <= 0) return q->agg_mode;
  if (q->agg_mode == kAggPart) return kAggGlobal;
  if (q->agg_mode == kAggRouted) return kAggHot;
  return q->agg_mode;
}

extern "C" size_t sirius_pipeline_scratch_bytes(const sirius_pipeline_desc* q) {
  if (!q) return 0;
  const DimLayout L = dim_layout_for(q);
  return L.total + run_layout(L.gcap, q->n, star_agg_mode(q)).total + semi_bytes(q);
}

extern "C" sirius_status sirius_run_pipeline(const sirius_pipeline_desc* q, sirius_result* result,
                                             void* d_scratch, size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = validate_pair(q);
  if (st != SIRIUS_OK) return st;
  st = validate_result(result);
  if (st != SIRIUS_OK) return st;
  if ((st = validate_semi(q)) != SIRIUS_OK) return st;
  const DimLayout L = dim_layout_for(q);
  const RunLayout R = run_layout(L.gcap, q->n, star_agg_mode(q));
  Scratch sc;
  st = sc.acquire(d_scratch, scratch_bytes, L.total + R.total + semi_bytes(q), s);
  if (st != SIRIUS_OK) return st;
  const DimView d = dim_view(L, sc.base);
  const RunView r = run_view(R, sc.base + L.total);
  if (single_applies(q, R)) {
    if ((st = run_single(q, L, d, r, R.gslots, pipe_out(result), s)) != SIRIUS_OK) return st;
    if (result->sync) return read_run_status(r, result, s);
    return SIRIUS_OK;
  }
  if ((st = dim_build(q, L, sc.base, s)) != SIRIUS_OK) return st;
  SemiView semi[kMaxSemi];
  if (q->nsemi > 0) {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_BUILD);
    if ((st = semi_build(q, sc.base + L.total + R.total, semi, s)) != SIRIUS_OK) return st;
  }
  if ((st = run_init(R, sc.base + L.total, s)) != SIRIUS_OK) return st;
  if (q->m > 0 && (st = run_probe(q, d, r, R.gslots, s, semi, q->nsemi)) != SIRIUS_OK) return st;
  if ((st = run_finalize(q, d, r, R.gslots, pipe_out(result), s)) != SIRIUS_OK) return st;
  if (result->sync) return read_run_status(r, result, s);
  return SIRIUS_OK;
}

// ------------------------------------------------------------------ resident build side
extern "C" size_t sirius_dim_index_bytes(const sirius_pipeline_desc* q) {
  if (!q) return 0;
  return dim_layout_for(q).total;
}

extern "C" sirius_status sirius_dim_index_build(const sirius_pipeline_desc* q, sirius_dim_index* idx,
                                                int32_t* h_status, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = validate_dim(q);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(idx && idx->d_mem, "dim index: NULL memory");
  SIRIUS_REQUIRE(((uintptr_t)idx->d_mem & 255) == 0, "dim index: memory must be 256-byte aligned");
  const DimLayout L = dim_layout_for(q);
  if (idx->bytes < L.total) {
    set_error("dim index: %zu bytes given, %zu needed", idx->bytes, L.total);
    return SIRIUS_ERR_SCRATCH;
  }
  idx->join_capacity = L.jcap;
  idx->group_capacity = L.gcap;
  idx->direct_capacity = L.dcap;
  idx->key_width = L.key_width;
  idx->bloom_log2 = L.bloom_log2;
  if ((st = dim_build(q, L, (char*)idx->d_mem, s)) != SIRIUS_OK) return st;
  if (h_status) {
    DimHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, idx->d_mem, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_status = h.status;
    if (h.status) {
      set_error("dim index: device status %d (more distinct group keys than group_cap_hint allows)", h.status);
      return (sirius_status)h.status;
    }
  }
  return SIRIUS_OK;
}

static DimLayout layout_of(const sirius_dim_index* idx) { return dim_layout_of_index(idx); }

extern "C" size_t sirius_probe_scratch_bytes(const sirius_pipeline_desc* q, const sirius_dim_index* idx) {
  if (!idx || !q) return 0;
  return run_layout(idx->group_capacity, q->n, q->agg_mode).total;
}

extern "C" sirius_status sirius_run_probe(const sirius_pipeline_desc* q, const sirius_dim_index* idx,
                                          sirius_result* result, void* d_scratch, size_t scratch_bytes,
                                          sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = validate_fact(q);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(q->nsemi == 0, "probe: semi-join dims are taken by sirius_run_pipeline only");
  st = validate_result(result);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(idx && idx->d_mem && idx->join_capacity > 0 && idx->group_capacity > 0,
                 "probe: dim index not built");
  SIRIUS_REQUIRE(idx->key_width == (q->fk_hi ? 8 : 4) || q->n == 0, "probe: key width differs from the dim index");
  const DimLayout L = layout_of(idx);
  const RunLayout R = run_layout(L.gcap, q->n, q->agg_mode);
  Scratch sc;
  st = sc.acquire(d_scratch, scratch_bytes, R.total, s);
  if (st != SIRIUS_OK) return st;
  const DimView d = dim_view(L, (char*)idx->d_mem);
  const RunView r = run_view(R, sc.base);
  if ((st = run_init(R, sc.base, s)) != SIRIUS_OK) return st;
  if ((st = run_probe(q, d, r, R.gslots, s)) != SIRIUS_OK) return st;
  if ((st = run_finalize(q, d, r, R.gslots, pipe_out(result), s)) != SIRIUS_OK) return st;
  if (result->sync) return read_run_status(r, result, s);
  return SIRIUS_OK;
}

// ------------------------------------------------------------------ host-resident columns
namespace {
struct HostLayout {
  DimLayout L;
  RunLayout R;
  int64_t chunk = 0;
  size_t off_run = 0, off_dimcols = 0, off_chunks = 0, chunk_bytes = 0, off_out = 0, total = 0;
};

HostLayout host_layout(const sirius_pipeline_desc* q, int64_t chunk_rows, int64_t out_cap) {
  HostLayout H;
  const bool wide = q->pk_hi != nullptr || q->fk_hi != nullptr;
  H.L = dim_layout_for(q);
  if (chunk_rows < 0) {
    H.chunk = 0;  // columns read in place: no staging buffers
  } else {
    H.chunk = chunk_rows > 0 ? chunk_rows : (16ll << 20);
    if (H.chunk > q->n && q->n > 0) H.chunk = (q->n + 3) / 4 * 4;
    H.chunk = (H.chunk + 3) / 4 * 4;
  }
  H.R = run_layout(H.L.gcap, chunk_rows < 0 ? q->n : H.chunk, q->agg_mode);
  H.off_run = H.L.total;
  H.off_dimcols = H.off_run + H.R.total;
  const size_t m = (size_t)q->m;
  const size_t dimcols =
      align_up(m * 4, 256) * ((wide ? 3 : 2) + (q->dpred ? 1 : 0)) + align_up(q->flag ? m : 0, 256);
  H.off_chunks = H.off_dimcols + dimcols;
  H.chunk_bytes = align_up((size_t)H.chunk * 4, 256) * (wide ? 3 : 2) + align_up((size_t)H.chunk * 8, 256);
  H.off_out = H.off_chunks + 2 * H.chunk_bytes;
  H.total = H.off_out + 5 * align_up((size_t)(out_cap > 0 ? out_cap : 1) * 8, 256) + 256;
  return H;
}
}  // namespace

extern "C" size_t sirius_pipeline_host_scratch_bytes(const sirius_pipeline_desc* q, int64_t chunk_rows,
                                                     int64_t out_cap) {
  if (!q) return 0;
  return host_layout(q, chunk_rows, out_cap).total;
}

extern "C" sirius_status sirius_run_pipeline_host(const sirius_pipeline_desc* q, sirius_result* result,
                                                  int64_t chunk_rows, void* d_scratch, size_t scratch_bytes,
                                                  sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = validate_pair(q);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(q->nsemi == 0, "host columns: semi-join dims are taken by sirius_run_pipeline only");
  st = validate_result(result);
  if (st != SIRIUS_OK) return st;
  const HostLayout H = host_layout(q, chunk_rows, result->out_cap);
  Scratch sc;
  st = sc.acquire(d_scratch, scratch_bytes, H.total, s);
  if (st != SIRIUS_OK) return st;
  char* base = sc.base;
  const bool wide = H.L.key_width == 8;
  const size_t m = (size_t)q->m;

  // dim columns to the device, then the build (on the compute stream)
  sirius_pipeline_desc dq = *q;
  {
    PhaseTimer pt(s, SIRIUS_PHASE_COPY);
    char* p = base + H.off_dimcols;
    auto put = [&](const void* src, size_t bytes, void** dst) -> cudaError_t {
      *dst = p;
      p += align_up(bytes, 256);
      return bytes ? cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    void* d_pk = nullptr;
    void* d_pk_hi = nullptr;
    void* d_grp = nullptr;
    void* d_flag = nullptr;
    void* d_dpred = nullptr;
    SIRIUS_CUDA_TRY(put(q->pk, m * 4, &d_pk));
    if (wide) SIRIUS_CUDA_TRY(put(q->pk_hi, m * 4, &d_pk_hi));
    SIRIUS_CUDA_TRY(put(q->grp, m * 4, &d_grp));
    if (q->flag) SIRIUS_CUDA_TRY(put(q->flag, m, &d_flag));
    if (q->dpred) SIRIUS_CUDA_TRY(put(q->dpred, m * 4, &d_dpred));
    dq.pk = (const int32_t*)d_pk;
    dq.pk_hi = (const int32_t*)d_pk_hi;
    dq.grp = (const int32_t*)d_grp;
    dq.flag = (const int8_t*)d_flag;
    dq.dpred = (const int32_t*)d_dpred;
  }
  const DimView d = dim_view(H.L, base);
  const RunView r = run_view(H.R, base + H.off_run);
  if ((st = dim_build(&dq, H.L, base, s)) != SIRIUS_OK) return st;
  if ((st = run_init(H.R, base + H.off_run, s)) != SIRIUS_OK) return st;

  // fact chunks: each column copied on a stream of its own (several copy engines at once),
  // double-buffered against the probe pass; or, with chunk_rows < 0, no staging at all: the
  // probe pass reads the pinned host columns in place over the host link
  constexpr int kCols = 4;  // fk, pred, fk_hi, val
  cudaStream_t c[kCols] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_ready[2][kCols] = {}, ev_free[2] = {nullptr, nullptr};
  sirius_status fail = SIRIUS_OK;
  const bool zero_copy = chunk_rows < 0;
  if (zero_copy) {
    const void* cols[kCols] = {q->fk, q->pred, q->fk_hi, q->val};
    for (int k = 0; k < kCols && fail == SIRIUS_OK; ++k) {
      if (!cols[k] || q->n == 0) continue;
      cudaPointerAttributes pa;
      if (cudaPointerGetAttributes(&pa, cols[k]) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        set_error("pipeline_host: reading columns in place needs pinned (page-locked) host memory");
        return SIRIUS_ERR_INVALID;
      }
    }
    if (q->m > 0) {
      sirius_pipeline_desc cq = dq;
      cq.fk = q->fk;
      cq.pred = q->pred;
      cq.fk_hi = q->fk_hi;
      cq.val = q->val;
      if ((st = run_probe(&cq, d, r, H.R.gslots, s)) != SIRIUS_OK) fail = st;
    }
  }
  for (int k = 0; k < kCols && fail == SIRIUS_OK && !zero_copy; ++k)
    if (cudaStreamCreateWithFlags(&c[k], cudaStreamNonBlocking) != cudaSuccess) fail = SIRIUS_ERR_CUDA;
  for (int b = 0; b < 2 && fail == SIRIUS_OK && !zero_copy; ++b) {
    if (cudaEventCreateWithFlags(&ev_free[b], cudaEventDisableTiming) != cudaSuccess) fail = SIRIUS_ERR_CUDA;
    for (int k = 0; k < kCols && fail == SIRIUS_OK; ++k)
      if (cudaEventCreateWithFlags(&ev_ready[b][k], cudaEventDisableTiming) != cudaSuccess) fail = SIRIUS_ERR_CUDA;
  }
  const int64_t nchunks = (q->m > 0 && !zero_copy) ? (q->n + H.chunk - 1) / H.chunk : 0;
  for (int64_t i = 0; i < nchunks && fail == SIRIUS_OK; ++i) {
    const int b = (int)(i & 1);
    const int64_t r0 = i * H.chunk;
    const int64_t rows = (q->n - r0) < H.chunk ? (q->n - r0) : H.chunk;
    char* buf = base + H.off_chunks + (size_t)b * H.chunk_bytes;
    const size_t a4 = align_up((size_t)H.chunk * 4, 256);
    sirius_pipeline_desc cq = dq;
    cq.fk = (const int32_t*)buf;
    cq.pred = (const int32_t*)(buf + a4);
    cq.fk_hi = wide ? (const int32_t*)(buf + 2 * a4) : nullptr;
    cq.val = (const int64_t*)(buf + (wide ? 3 : 2) * a4);
    cq.n = rows;
    void* dst[kCols] = {(void*)cq.fk, (void*)cq.pred, (void*)cq.fk_hi, (void*)cq.val};
    const void* src[kCols] = {q->fk + r0, q->pred + r0, wide ? (const void*)(q->fk_hi + r0) : nullptr, q->val + r0};
    const size_t bytes[kCols] = {(size_t)rows * 4, (size_t)rows * 4, (size_t)rows * 4, (size_t)rows * 8};
    for (int k = 0; k < kCols && fail == SIRIUS_OK; ++k) {
      if (!src[k]) continue;
      if ((i >= 2 && cudaStreamWaitEvent(c[k], ev_free[b], 0) != cudaSuccess) ||
          cudaMemcpyAsync(dst[k], src[k], bytes[k], cudaMemcpyHostToDevice, c[k]) != cudaSuccess ||
          cudaEventRecord(ev_ready[b][k], c[k]) != cudaSuccess || cudaStreamWaitEvent(s, ev_ready[b][k], 0) != cudaSuccess)
        fail = SIRIUS_ERR_CUDA;
    }
    if (fail != SIRIUS_OK) break;
    if ((st = run_probe(&cq, d, r, H.R.gslots, s)) != SIRIUS_OK) { fail = st; break; }
    if (cudaEventRecord(ev_free[b], s) != cudaSuccess) { fail = SIRIUS_ERR_CUDA; break; }
  }
  if (fail == SIRIUS_ERR_CUDA) set_error("pipeline_host: CUDA error %s", cudaGetErrorString(cudaGetLastError()));
  // results: finalize into device arrays, then copy the G rows back into the host arrays
  int64_t* dout[5];
  for (int k = 0; k < 5; ++k)
    dout[k] = (int64_t*)(base + H.off_out + (size_t)k * align_up((size_t)(result->out_cap > 0 ? result->out_cap : 1) * 8, 256));
  PipeOut out{result->keys ? dout[0] : nullptr, result->sum ? dout[1] : nullptr, result->count ? dout[2] : nullptr,
              result->min ? dout[3] : nullptr, result->max ? dout[4] : nullptr, result->out_cap, nullptr, nullptr};
  if (fail == SIRIUS_OK) fail = run_finalize(&dq, d, r, H.R.gslots, out, s);
  if (fail == SIRIUS_OK) {
    fail = read_run_status(r, result, s);
    if (fail == SIRIUS_OK && result->groups > 0) {
      PhaseTimer pt(s, SIRIUS_PHASE_COPY);
      int64_t* hosts[5] = {result->keys, result->sum, result->count, result->min, result->max};
      for (int k = 0; k < 5 && fail == SIRIUS_OK; ++k)
        if (hosts[k] && cudaMemcpyAsync(hosts[k], dout[k], (size_t)result->groups * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
          fail = SIRIUS_ERR_CUDA;
      if (fail == SIRIUS_OK && cudaStreamSynchronize(s) != cudaSuccess) fail = SIRIUS_ERR_CUDA;
      if (fail == SIRIUS_ERR_CUDA) set_error("pipeline_host: result copy failed");
    }
  }
  for (int k = 0; k < kCols; ++k)
    if (c[k]) cudaStreamSynchronize(c[k]);
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < kCols; ++k)
      if (ev_ready[b][k]) cudaEventDestroy(ev_ready[b][k]);
    if (ev_free[b]) cudaEventDestroy(ev_free[b]);
  }
  for (int k = 0; k < kCols; ++k)
    if (c[k]) cudaStreamDestroy(c[k]);
  return fail;
}

// ------------------------------------------------------------------ self-test of the barrier wait
extern "C" sirius_status sirius_selftest_grid_barrier(int32_t blocks, int32_t missing, uint32_t max_spins,
                                                     void* d_mem, size_t bytes, int32_t* h_status,
                                                     int32_t* h_passed, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(blocks >= 1 && blocks <= sm_count(), "selftest: blocks=%d outside [1, %d]", blocks, sm_count());
  SIRIUS_REQUIRE(missing >= 0 && missing <= 1, "selftest: missing=%d must be 0 or 1", missing);
  SIRIUS_REQUIRE(max_spins >= 1 && max_spins <= kGridBarrierSpins, "selftest: max_spins out of [1, 2^23]");
  SIRIUS_REQUIRE(d_mem && bytes >= sizeof(PipeHeader) && ((uintptr_t)d_mem & 255) == 0,
                 "selftest: need %zu bytes of 256-byte aligned device memory", sizeof(PipeHeader));
  SIRIUS_REQUIRE(h_status && h_passed, "selftest: NULL host result");
  PipeHeader* phdr = (PipeHeader*)d_mem;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(phdr, 0, sizeof(PipeHeader), s));
  const uint32_t target = (uint32_t)(blocks + missing);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SIRIUS_CUDA_TRY(cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, phdr, target, max_spins));
  SIRIUS_LAUNCH_CHECK();
  PipeHeader h;
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, phdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
  *h_status = h.status;
  *h_passed = (int32_t)h.blocks_done;
  return SIRIUS_OK;
}
