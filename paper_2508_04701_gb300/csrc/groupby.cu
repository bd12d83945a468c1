// A5 / A6: hash group-by aggregation and finalize (Sec. 3.2.2; Sec. 4.2: group-by with few
// groups suffers from memory contention).
//
// Group table (scratch): a 256-byte header, keys[cap + 1] (int64, kEmptyKey = empty; slot cap
// holds the one key equal to kEmptyKey) and Agg[cap + 1] {sum, count, min, max}.
//
// A first pass over the keys records their range.  When the range spans at most the table's
// limit of distinct keys (a dense key domain: dictionary codes, surrogate keys, small integer
// attributes), a key's slot is its offset from the smallest key -- no hashing, no
// compare-and-swap, no key array to clear or read -- and only the range's slots are cleared and
// finalized.  Such a table can never hold more keys than the hash table would, so TABLE_FULL
// is unchanged.  Otherwise keys are hashed into the table as before.
// Small tables (cap <= kSmemMaxCap): every block first aggregates its rows into a private copy
// of the table in shared memory (shared-memory atomics), then merges its occupied slots into
// the global table -- the contention of few groups stays on chip.  Large tables: with direct
// slots, four rows per thread (16-byte loads) go to the global table behind a per-block cache
// of hot groups in shared memory (skewed keys aggregate on chip); hashed keys go straight to the
// global table, lanes of a warp holding the same key combined first (match_any), so a hot key
// costs one global atomic per warp instead of one per row.
#include "pipeline.cuh"

namespace sirius {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kSmemMaxCap = 2048;  // (2048 + 1) * 40 B = 82 KB of shared memory

struct GroupHeader {
  int32_t status;
  int32_t pad0;
  unsigned long long distinct;
  unsigned long long groups;
  // key range, order-preserving unsigned images (key ^ sign bit): the largest in kmax_enc, the
  // complement of the smallest in kmin_inv, so that the cleared header (zeros) is the identity
  // of both atomicMax reductions
  unsigned long long kmax_enc;
  unsigned long long kmin_inv;
  unsigned long long pad[27];
};
static_assert(sizeof(GroupHeader) == 256, "group header is 256 bytes");

constexpr unsigned long long kSign = 0x8000000000000000ull;

// The key range as the range pass recorded it, and whether direct slots apply: n > 0 and
// kmax - kmin < limit (so range = kmax - kmin + 1 <= limit slots).
struct KeyRange {
  int64_t kmin;
  uint64_t range;  // kmax - kmin + 1 when direct, else 0
  bool direct;
};
__device__ __forceinline__ KeyRange key_range(const GroupHeader* hdr, int64_t n, unsigned long long limit) {
  KeyRange r;
  const unsigned long long mx = hdr->kmax_enc, mn = ~hdr->kmin_inv;
  r.kmin = (int64_t)(mn ^ kSign);
  const uint64_t span = (mx ^ kSign) - (mn ^ kSign);  // two's-complement difference, exact
  r.direct = n > 0 && mx >= mn && span < limit;
  r.range = r.direct ? span + 1 : 0;
  return r;
}

__device__ __forceinline__ int64_t load_key(const void* keys, int key_width, int64_t i) {
  return key_width == 4 ? (int64_t)((const int32_t*)keys)[i] : ((const int64_t*)keys)[i];
}

// Range pass: the smallest and largest key (warp reductions, one pair of atomics per warp).
__global__ void __launch_bounds__(256)
group_range_kernel(const void* __restrict__ keys, int key_width, int64_t n, GroupHeader* hdr) {
  unsigned long long hi = 0, lo_inv = 0;  // identities of max(enc) and max(~enc)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long e = (unsigned long long)load_key(keys, key_width, i) ^ kSign;
    hi = e > hi ? e : hi;
    lo_inv = ~e > lo_inv ? ~e : lo_inv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, lo_inv, o);
    hi = a > hi ? a : hi;
    lo_inv = b > lo_inv ? b : lo_inv;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&hdr->kmax_enc, hi);
    atomicMax(&hdr->kmin_inv, lo_inv);
  }
}

// Clears the slots the aggregation will use: the range's aggregates (direct slots), or every
// key and aggregate of the hash table.
__global__ void group_init_kernel(int64_t* keys, Agg* aggs, int64_t slots, const GroupHeader* hdr, int64_t n,
                                  unsigned long long limit) {
  const KeyRange kr = key_range(hdr, n, limit);
  const int64_t use = kr.direct ? (int64_t)kr.range : slots;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < use;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!kr.direct) keys[i] = kEmptyKey;
    agg_identity(&aggs[i]);
  }
}

// Combine the lanes of a warp that hold the same key; returns true in the one lane per key
// that must apply the combined (sum, count, min, max).
__device__ __forceinline__ bool warp_combine(bool active, int64_t key, int64_t v,
                                             unsigned long long& sum, unsigned long long& cnt,
                                             long long& mn, long long& mx) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  const unsigned peers = __match_any_sync(0xffffffffu, active ? key : (int64_t)0x7ead7ead7ead7eadll) & act;
  sum = active ? (unsigned long long)v : 0;
  cnt = active ? 1 : 0;
  mn = active ? v : INT64_MAX;
  mx = active ? v : INT64_MIN;
  if (!active) return false;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  // every lane of a peer group walks the same peer set, so the shuffles stay convergent
  unsigned long long s = 0, c = 0;
  long long lo = INT64_MAX, hi = INT64_MIN;
  for (unsigned rem = peers; rem; rem &= rem - 1) {
    const int src = __ffs(rem) - 1;
    const long long pv = __shfl_sync(peers, (long long)v, src);
    s += (unsigned long long)pv;
    c += 1;
    lo = pv < lo ? pv : lo;
    hi = pv > hi ? pv : hi;
  }
  sum = s;
  cnt = c;
  mn = lo;
  mx = hi;
  return lane == leader;
}

__global__ void __launch_bounds__(kThreads)
group_global_kernel(const void* __restrict__ keys_in, int key_width, const int64_t* __restrict__ vals,
                    int64_t n, uint32_t aggs, int64_t* keys, Agg* tab, uint32_t cap,
                    GroupHeader* hdr, unsigned long long limit) {
  if (key_range(hdr, n, limit).direct) return;  // group_direct_kernel aggregates these keys
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool active = i < n;
    const int64_t key = active ? load_key(keys_in, key_width, i) : 0;
    const int64_t v = active ? vals[i] : 0;
    unsigned long long s, c;
    long long mn, mx;
    const bool lead = warp_combine(active, key, v, s, c, mn, mx);
    if (lead) {
      const int64_t slot = group_find_or_insert(keys, cap, key, &hdr->distinct, limit);
      if (slot < 0) {
        set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
      } else {
        agg_merge_global(&tab[slot], s, c, mn, mx, aggs);
      }
    }
  }
}

// Direct slots, large table: four rows per thread (16-byte loads when the columns are 16-byte
// aligned), every row's aggregates behind the block's cache of hot groups.
// One launch per pass over the rows when the range's aggregates exceed what L2 keeps: pass p
// aggregates only the slots [p * kPassSlots, (p + 1) * kPassSlots), so its reductions hit a
// 48 MB window of the table that stays in L2 instead of fetching and writing back random DRAM
// sectors; every pass reads the keys, and a value only where its quad has a row in the window.
constexpr uint64_t kPassSlots = (48ull << 20) / sizeof(Agg);
// Split pass of the direct-slot group-by: for inputs with many rows per group slot that ask for
// MIN or MAX and fit one window (the same technique as the fused probe's split pass).
constexpr int64_t kGroupSplitMinRows = 1ll << 24;
constexpr int64_t kGroupSplitRowsPerSlot = 256;

//
// kBounded: the second phase of a split pass (one window covers every slot; `bounds` set):
// the rows skip the MIN / MAX reductions that the extreme bounds taken after the first phase
// rule out, as in the fused probe's split pass.
template <int kKeyWidth, bool kVec, bool kBounded = false>
__global__ void __launch_bounds__(512)
group_direct_kernel(const void* __restrict__ keys_in, const int64_t* __restrict__ vals, int64_t n, uint32_t aggs,
                    Agg* tab, const GroupHeader* hdr, unsigned long long limit, int pass,
                    const ExtremeBounds* bounds) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const KeyRange kr = key_range(hdr, n, limit);
  if (!kr.direct) return;  // hashed keys: group_global_kernel
  const uint64_t lo = (uint64_t)pass * kPassSlots;
  if (lo >= kr.range) return;  // the range ends before this pass's window
  const uint64_t width = kr.range - lo < kPassSlots ? kr.range - lo : kPassSlots;  // window [lo, lo + width)
  const bool whole = lo == 0 && width == kr.range;  // one pass covers every slot
  ProbeArgs a{};
  a.tab = tab;
  a.aggs = aggs;
  a.bounds = bounds;
  const SmemAggs T = smem_aggs(smem_raw, kHotEntries);
  if constexpr (kBounded) {
    // the bounds into shared memory after the hot-group cache, the extremes decoded (published
    // by the barrier below)
    const uint4* src = reinterpret_cast<const uint4*>(bounds);
    uint4* dst = reinterpret_cast<uint4*>(smem_raw + kHotSmemBytes);
    for (uint32_t i = threadIdx.x; i < kBoundsSmemBytes / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
      s_bound_floor = bound_decode(bounds->max_floor_enc);
      s_bound_ceil = bound_decode(~bounds->min_ceil_inv);
    }
  }
  for (uint32_t i = threadIdx.x; i < (uint32_t)kHotEntries; i += blockDim.x) {
    smem_identity(T, i);
    T.tag[i] = kEmpty32;
  }
  __syncthreads();
  const int64_t nq = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += stride) {
    int64_t k[4], v[4];
    if (kVec) {
      if (kKeyWidth == 4) {
        const int4 k4 = __ldcs(reinterpret_cast<const int4*>(keys_in) + q);
        k[0] = k4.x, k[1] = k4.y, k[2] = k4.z, k[3] = k4.w;
      } else {
        const longlong2 a0 = __ldcs(reinterpret_cast<const longlong2*>(keys_in) + 2 * q);
        const longlong2 a1 = __ldcs(reinterpret_cast<const longlong2*>(keys_in) + 2 * q + 1);
        k[0] = a0.x, k[1] = a0.y, k[2] = a1.x, k[3] = a1.y;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) k[r] = load_key(keys_in, kKeyWidth, 4 * q + r);
    }
    uint32_t in = 0;  // rows whose slot is in this pass's window
#pragma unroll
    for (int r = 0; r < 4; ++r) in |= (uint32_t)(whole || (uint64_t)(k[r] - kr.kmin) - lo < width) << r;
    if (!in) continue;
    if (kVec) {
      const longlong2 v0 = __ldcs(reinterpret_cast<const longlong2*>(vals) + 2 * q);
      const longlong2 v1 = __ldcs(reinterpret_cast<const longlong2*>(vals) + 2 * q + 1);
      v[0] = v0.x, v[1] = v0.y, v[2] = v1.x, v[3] = v1.y;
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = ((in >> r) & 1u) ? vals[4 * q + r] : 0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if ((in >> r) & 1u) aggregate<kAggHot, false, kBounded>(a, T, (uint32_t)(uint64_t)(k[r] - kr.kmin), v[r]);
  }
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < n - (nq << 2)) {
    const int64_t i = (nq << 2) + threadIdx.x;
    const uint64_t slot = (uint64_t)(load_key(keys_in, kKeyWidth, i) - kr.kmin);
    if (slot - lo < width) aggregate<kAggHot>(a, T, (uint32_t)slot, vals[i]);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < (uint32_t)kHotEntries; i += blockDim.x)
    if (T.tag[i] != kEmpty32) smem_merge(T, i, &tab[T.tag[i]], aggs);
}

__global__ void __launch_bounds__(kThreads)
group_smem_kernel(const void* __restrict__ keys_in, int key_width, const int64_t* __restrict__ vals,
                  int64_t n, uint32_t aggs, int64_t* keys, Agg* tab, uint32_t cap,
                  GroupHeader* hdr, unsigned long long limit) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  Agg* s_tab = reinterpret_cast<Agg*>(smem_raw);
  int64_t* s_keys = reinterpret_cast<int64_t*>(smem_raw + sizeof(Agg) * (cap + 1));
  __shared__ unsigned long long s_distinct;
  for (uint32_t i = threadIdx.x; i <= cap; i += blockDim.x) {
    s_keys[i] = kEmptyKey;
    agg_identity(&s_tab[i]);
  }
  if (threadIdx.x == 0) s_distinct = 0;
  __syncthreads();
  const KeyRange kr = key_range(hdr, n, limit);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t key = load_key(keys_in, key_width, i);
    const long long v = vals[i];
    int64_t slot;
    if (kr.direct) {
      slot = (int64_t)(uint64_t)(key - kr.kmin);  // < range <= limit < cap
    } else if (key == kEmptyKey) {
      slot = cap;
    } else {
      slot = -1;
      uint32_t s = home_slot64((uint64_t)key, cap);
      for (uint32_t step = 0; step < cap; ++step) {
        int64_t cur = s_keys[s];
        if (cur == kEmptyKey) {
          cur = (int64_t)atomicCAS((unsigned long long*)&s_keys[s], (unsigned long long)kEmptyKey,
                                   (unsigned long long)key);
          if (cur == kEmptyKey) {
            if (atomicAdd(&s_distinct, 1ull) < limit) slot = s;
            break;
          }
        }
        if (cur == key) {
          slot = s;
          break;
        }
        s = (s + 1 == cap) ? 0 : s + 1;
      }
    }
    if (slot < 0) {
      // the block's private table is full: this row goes to the global table directly
      const int64_t g = group_find_or_insert(keys, cap, key, &hdr->distinct, limit);
      if (g < 0) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
      else agg_update_global(&tab[g], v, aggs);
      continue;
    }
    Agg* a = &s_tab[slot];
    if (aggs & SIRIUS_AGG_SUM) atomicAdd(&a->sum, (unsigned long long)v);
    atomicAdd(&a->count, 1ull);
    if (aggs & SIRIUS_AGG_MIN) atomicMin(&a->min, v);
    if (aggs & SIRIUS_AGG_MAX) atomicMax(&a->max, v);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i <= cap; i += blockDim.x) {
    const Agg a = s_tab[i];
    if (a.count == 0) continue;
    const int64_t g = (kr.direct || i == cap) ? (int64_t)i
                                               : group_find_or_insert(keys, cap, s_keys[i], &hdr->distinct, limit);
    if (g < 0) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
    else agg_merge_global(&tab[g], a.sum, a.count, a.min, a.max, aggs);
  }
}

__global__ void group_finalize_kernel(const int64_t* __restrict__ keys, const Agg* __restrict__ tab,
                                      int64_t slots, uint32_t cap, uint32_t aggs, int64_t* out_keys,
                                      int64_t* out_sum, int64_t* out_count, int64_t* out_min,
                                      int64_t* out_max, int64_t out_cap, GroupHeader* hdr,
                                      int64_t n, unsigned long long limit) {
  const KeyRange kr = key_range(hdr, n, limit);
  if (kr.direct) slots = (int64_t)kr.range;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (slots + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < slots && tab[i].count > 0;
    const uint64_t pos = warp_append(&hdr->groups, occ);
    if (occ && (int64_t)pos < out_cap) {
      const Agg a = tab[i];
      if (out_keys) out_keys[pos] = kr.direct ? kr.kmin + i : ((i == cap) ? kEmptyKey : keys[i]);
      if (out_sum) out_sum[pos] = (int64_t)a.sum;
      if (out_count) out_count[pos] = (int64_t)a.count;
      if (out_min) out_min[pos] = a.min;
      if (out_max) out_max[pos] = a.max;
    }
  }
}

__global__ void copy_groups_kernel(const GroupHeader* hdr, int64_t* d_groups) {
  *d_groups = (int64_t)hdr->groups;
}

}  // namespace

size_t groupby_scratch_bytes(int64_t hint) {
  const int64_t cap = group_capacity_for(hint);
  return 256 + align_up((size_t)(cap + 1) * 8, 256) + align_up((size_t)(cap + 1) * sizeof(Agg), 256) +
         align_up(sizeof(ExtremeBounds), 256) + 256;
}

}  // namespace sirius

using namespace sirius;

extern "C" int64_t sirius_groupby_capacity(int64_t hint) { return group_capacity_for(hint); }
extern "C" size_t sirius_groupby_scratch_bytes(int64_t hint) { return groupby_scratch_bytes(hint); }

extern "C" sirius_status sirius_groupby_agg(const void* d_keys, int32_t key_width, const int64_t* d_vals,
                                            int64_t n, uint32_t aggs, int64_t hint,
                                            int64_t* d_out_keys, int64_t* d_sum, int64_t* d_count,
                                            int64_t* d_min, int64_t* d_max, int64_t out_cap,
                                            int64_t* d_groups, int64_t* h_groups, void* d_scratch,
                                            size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(key_width == 4 || key_width == 8, "groupby: key_width must be 4 or 8");
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "groupby: n out of range");
  SIRIUS_REQUIRE(n == 0 || (d_keys && d_vals), "groupby: NULL input");
  SIRIUS_REQUIRE(out_cap >= 0, "groupby: negative out_cap");
  SIRIUS_REQUIRE(aggs <= SIRIUS_AGG_ALL, "groupby: bad aggregate mask");
  const int64_t cap = group_capacity_for(hint);
  SIRIUS_REQUIRE(cap < (1ll << 31), "groupby: group_cap_hint too large");
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, groupby_scratch_bytes(hint), s);
  if (st != SIRIUS_OK) return st;
  GroupHeader* hdr = (GroupHeader*)sc.take(256);
  int64_t* keys = (int64_t*)sc.take((size_t)(cap + 1) * 8);
  Agg* tab = (Agg*)sc.take((size_t)(cap + 1) * sizeof(Agg));
  ExtremeBounds* bounds = (ExtremeBounds*)sc.take(sizeof(ExtremeBounds));
  const unsigned long long limit = group_limit_for(cap);
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256, s));
  if (n > 0) {
    group_range_kernel<<<grid_for(n, 256) < sm_count() * 8 ? grid_for(n, 256) : sm_count() * 8, 256, 0, s>>>(
        d_keys, key_width, n, hdr);
    SIRIUS_LAUNCH_CHECK();
  }
  group_init_kernel<<<grid_for(cap + 1, kThreads), kThreads, 0, s>>>(keys, tab, cap + 1, hdr, n, limit);
  SIRIUS_LAUNCH_CHECK();
  PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
  if (n > 0) {
    if (cap <= kSmemMaxCap) {
      const size_t smem = (size_t)(cap + 1) * (sizeof(Agg) + 8);
      static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
      SIRIUS_CUDA_TRY(ensure_smem_limit(group_smem_kernel, 100 * 1024, smem_set));
      int64_t want = (n + kThreads * 16 - 1) / (kThreads * 16);
      int64_t maxg = (int64_t)sm_count() * 2;
      int g = (int)(want < maxg ? (want > 0 ? want : 1) : maxg);
      group_smem_kernel<<<g, kThreads, smem, s>>>(d_keys, key_width, d_vals, n, aggs, keys, tab,
                                                  (uint32_t)cap, hdr, limit);
    } else {
      // direct slots (decided on the device from the key range) or the hash table: each kernel
      // returns at once when the other applies
      const bool vec = ((uintptr_t)d_keys & 15) == 0 && ((uintptr_t)d_vals & 15) == 0;
      auto kd = key_width == 4 ? (vec ? group_direct_kernel<4, true> : group_direct_kernel<4, false>)
                               : (vec ? group_direct_kernel<8, true> : group_direct_kernel<8, false>);
      {
        static std::atomic<uint64_t> smem_set[4] = {};  // per kernel: devices with the limit raised
        SIRIUS_CUDA_TRY(ensure_smem_limit(kd, (int)kHotSmemBytes,
                                          smem_set[(key_width == 8 ? 2 : 0) + (vec ? 1 : 0)]));
      }
      int64_t gd = ((n >> 2) + 511) / 512;
      const int64_t most = (int64_t)sm_count() * 3;  // three 64 KB caches per SM
      gd = gd < 1 ? 1 : (gd > most ? most : gd);
      // passes over windows of the direct slots (the range is known on the device only: a pass
      // whose window starts past it returns at once)
      const int passes = (int)((group_limit_for(cap) + kPassSlots - 1) / kPassSlots);
      if (passes == 1 && (aggs & (SIRIUS_AGG_MIN | SIRIUS_AGG_MAX)) && n >= kGroupSplitMinRows &&
          n >= kGroupSplitRowsPerSlot * (cap + 1)) {
        // split pass: the first 1/16 of the rows in full, the extreme bounds, then the rest
        // behind them (one block fewer per SM: the bounds' copy follows each 64 KB cache)
        const int64_t n0 = ((n / 16) >> 2) << 2;
        const size_t kw = (size_t)key_width;
        kd<<<(unsigned)gd, 512, kHotSmemBytes, s>>>(d_keys, d_vals, n0, aggs, tab, hdr, limit, 0, nullptr);
        SIRIUS_LAUNCH_CHECK();
        SIRIUS_CUDA_TRY(cudaMemsetAsync(bounds, 0xFF, 2 * sizeof(unsigned long long), s));
        extreme_bounds_kernel<<<kBoundSlots / 256, 256, 0, s>>>(tab, (uint32_t)(cap + 1), bounds);
        SIRIUS_LAUNCH_CHECK();
        auto kb = key_width == 4 ? (vec ? group_direct_kernel<4, true, true> : group_direct_kernel<4, false, true>)
                                 : (vec ? group_direct_kernel<8, true, true> : group_direct_kernel<8, false, true>);
        const size_t smem = kHotSmemBytes + kBoundsSmemBytes;
        static std::atomic<uint64_t> smem_set_b[4] = {};
        SIRIUS_CUDA_TRY(ensure_smem_limit(kb, (int)smem, smem_set_b[(key_width == 8 ? 2 : 0) + (vec ? 1 : 0)]));
        const int64_t most2 = (int64_t)sm_count() * 2;
        const int64_t gd2 = gd > most2 ? most2 : gd;
        kb<<<(unsigned)gd2, 512, smem, s>>>(static_cast<const char*>(d_keys) + n0 * kw, d_vals + n0, n - n0, aggs,
                                           tab, hdr, limit, 0, bounds);
        SIRIUS_LAUNCH_CHECK();
      } else {
        for (int p = 0; p < passes; ++p) {
          kd<<<(unsigned)gd, 512, kHotSmemBytes, s>>>(d_keys, d_vals, n, aggs, tab, hdr, limit, p, nullptr);
          SIRIUS_LAUNCH_CHECK();
        }
      }
      group_global_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(d_keys, key_width, d_vals, n, aggs,
                                                                     keys, tab, (uint32_t)cap, hdr, limit);
    }
    SIRIUS_LAUNCH_CHECK();
  }
  group_finalize_kernel<<<grid_for(cap + 1, kThreads), kThreads, 0, s>>>(
      keys, tab, cap + 1, (uint32_t)cap, aggs, d_out_keys, d_sum, d_count, d_min, d_max, out_cap, hdr,
      n, limit);
  SIRIUS_LAUNCH_CHECK();
  if (d_groups) {
    copy_groups_kernel<<<1, 1, 0, s>>>(hdr, d_groups);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_groups) {
    GroupHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_groups = (int64_t)h.groups;
    if (h.status) {
      set_error("groupby: device status %d (more distinct keys than the table takes)", h.status);
      return (sirius_status)h.status;
    }
    if ((int64_t)h.groups > out_cap) {
      set_error("groupby: %llu groups exceed out_cap %lld", h.groups, (long long)out_cap);
      return SIRIUS_ERR_CAPACITY;
    }
  }
  return SIRIUS_OK;
}
