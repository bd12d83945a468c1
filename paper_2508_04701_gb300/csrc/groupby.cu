// A5 / A6: hash group-by aggregation and finalize (Sec. 3.2.2; Sec. 4.2: group-by with few
// groups suffers from memory contention).
//
// Group table (scratch): a 256-byte header, keys[cap + 1] (int64, kEmptyKey = empty; slot cap
// holds the one key equal to kEmptyKey) and Agg[cap + 1] {sum, count, min, max}.
// Small tables (cap <= kSmemMaxCap): every block first aggregates its rows into a private copy
// of the table in shared memory (shared-memory atomics), then merges its occupied slots into
// the global table -- the contention of few groups stays on chip.  Large tables: rows go
// straight to the global table; lanes of a warp holding the same key are combined first
// (match_any), so a hot key costs one global atomic per warp instead of one per row.
#include "tables.cuh"

namespace sirius {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kSmemMaxCap = 2048;  // (2048 + 1) * 40 B = 82 KB of shared memory

struct GroupHeader {
  int32_t status;
  int32_t pad0;
  unsigned long long distinct;
  unsigned long long groups;
  unsigned long long pad[29];
};
static_assert(sizeof(GroupHeader) == 256, "group header is 256 bytes");

__global__ void group_init_kernel(int64_t* keys, Agg* aggs, int64_t slots) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = kEmptyKey;
    agg_identity(&aggs[i]);
  }
}

__device__ __forceinline__ int64_t load_key(const void* keys, int key_width, int64_t i) {
  return key_width == 4 ? (int64_t)((const int32_t*)keys)[i] : ((const int64_t*)keys)[i];
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
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t key = load_key(keys_in, key_width, i);
    const long long v = vals[i];
    int64_t slot;
    if (key == kEmptyKey) {
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
    const int64_t g = (i == cap) ? (int64_t)cap
                                 : group_find_or_insert(keys, cap, s_keys[i], &hdr->distinct, limit);
    if (g < 0) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
    else agg_merge_global(&tab[g], a.sum, a.count, a.min, a.max, aggs);
  }
}

__global__ void group_finalize_kernel(const int64_t* __restrict__ keys, const Agg* __restrict__ tab,
                                      int64_t slots, uint32_t cap, uint32_t aggs, int64_t* out_keys,
                                      int64_t* out_sum, int64_t* out_count, int64_t* out_min,
                                      int64_t* out_max, int64_t out_cap, GroupHeader* hdr,
                                      int64_t* d_groups) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (slots + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < slots && tab[i].count > 0;
    const uint64_t pos = warp_append(&hdr->groups, occ);
    if (occ && (int64_t)pos < out_cap) {
      const Agg a = tab[i];
      if (out_keys) out_keys[pos] = (i == cap) ? kEmptyKey : keys[i];
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
  return 256 + align_up((size_t)(cap + 1) * 8, 256) + (size_t)(cap + 1) * sizeof(Agg) + 256;
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
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256, s));
  group_init_kernel<<<grid_for(cap + 1, kThreads), kThreads, 0, s>>>(keys, tab, cap + 1);
  SIRIUS_LAUNCH_CHECK();
  const unsigned long long limit = group_limit_for(cap);
  PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
  if (n > 0) {
    if (cap <= kSmemMaxCap) {
      const size_t smem = (size_t)(cap + 1) * (sizeof(Agg) + 8);
      static bool attr_set = false;
      if (!attr_set) {
        SIRIUS_CUDA_TRY(cudaFuncSetAttribute(group_smem_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        attr_set = true;
      }
      int64_t want = (n + kThreads * 16 - 1) / (kThreads * 16);
      int64_t maxg = (int64_t)sm_count() * 2;
      int g = (int)(want < maxg ? (want > 0 ? want : 1) : maxg);
      group_smem_kernel<<<g, kThreads, smem, s>>>(d_keys, key_width, d_vals, n, aggs, keys, tab,
                                                  (uint32_t)cap, hdr, limit);
    } else {
      group_global_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(d_keys, key_width, d_vals, n, aggs,
                                                                     keys, tab, (uint32_t)cap, hdr, limit);
    }
    SIRIUS_LAUNCH_CHECK();
  }
  group_finalize_kernel<<<grid_for(cap + 1, kThreads), kThreads, 0, s>>>(
      keys, tab, cap + 1, (uint32_t)cap, aggs, d_out_keys, d_sum, d_count, d_min, d_max, out_cap, hdr,
      d_groups);
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
