// Partitioned aggregation for group tables too large for shared memory (Sec. 4.2: group-by
// cost; the fused probe pass otherwise spends four L2 atomics per joined row).
//
// Pass 1 (fused with filter and probe) cuts the fact table into tiles of kPartTile rows.  Each
// joined row yields a tuple (group slot, value); its partition is slot / kPartSlots.  A block
// histograms its tile's tuples by partition in shared memory (lanes of a warp with the same
// partition combined by match_any), scans the histogram, writes the tile's prefix row and
// then each tuple to its place in the tile's own output region -- grouped by partition, no
// global atomics.  Pass 2 gives each (partition, tile range) a block whose shared-memory table
// covers the partition's kPartSlots group slots: warps walk 32 tiles at a time (one tile
// segment per lane, segments concatenated by a warp scan), aggregate with shared-memory
// atomics and, at the end, merge the occupied slots into the global table with reductions.
// Traffic: 12 bytes per joined row written and read back, instead of four L2 atomics.
#pragma once

#include "pipeline.cuh"

namespace sirius {
namespace part {

constexpr int kPartSlots = 4096;     // group slots per partition (128 KB of Agg in pass 2)
constexpr int kPartShift = 12;
constexpr int kPartTile = 4096;      // fact rows per pass-1 tile
constexpr int kScatterThreads = 512; // two quads per thread and tile
constexpr int kAggThreads = 512;
constexpr int kMaxParts = 256;       // partitioned mode needs gslots <= kMaxParts * kPartSlots

struct PartArgs {
  uint32_t* tgs;     // [ntiles * kPartTile] group slot of each tuple
  int64_t* tval;     // [ntiles * kPartTile] value of each tuple
  int32_t* prefix;   // [ntiles * (P + 1)] start of each partition's segment within its tile
  int64_t ntiles;
  int32_t parts;     // P
  int32_t pad;
};

inline int parts_for(int64_t gslots) { return (int)((gslots + kPartSlots - 1) / kPartSlots); }
inline int64_t tiles_for(int64_t n) { return (n + kPartTile - 1) / kPartTile; }

// First match of one selected row: its group slot, or kEmpty32.  Further matches (a hash
// table holding duplicate keys) are aggregated at once with global reductions.
template <bool kWide>
__device__ __forceinline__ uint32_t first_match(const ProbeArgs& a, const Lookup& L, uint64_t key, int64_t v) {
  if (!kWide && L.direct) {
    const uint32_t k = (uint32_t)key - (uint32_t)L.kmin;
    return k < L.range ? __ldg(a.dslot + k) : kEmpty32;
  }
  constexpr int kPer = kWide ? 2 : 4;
  uint32_t slot = kWide ? home_slot64(key, a.jcap) : home_slot32((uint32_t)key, a.jcap);
  uint32_t first = kEmpty32;
  for (uint32_t step = 0; step < a.jcap; step += kPer) {
    uint64_t w[4];
    load_bucket<kWide>(a.jslots, slot, w);
    bool stop = false;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const uint64_t k = kWide ? w[2 * j] : (uint64_t)(uint32_t)w[j];
      const uint32_t p = kWide ? (uint32_t)w[2 * j + 1] : (uint32_t)(w[j] >> 32);
      if (!stop) {
        if (p == kEmpty32) {
          stop = true;
        } else if (k == key) {
          if (first == kEmpty32) first = p;
          else agg_update_global(&a.tab[p], v, a.aggs);
          stop = !L.dups;
        }
      }
    }
    if (stop) break;
    slot += kPer;
    if (slot >= a.jcap) slot = 0;
  }
  return first;
}

template <bool kWide, bool kVec>
__global__ void __launch_bounds__(kScatterThreads)
part_scatter_kernel(ProbeArgs a, PartArgs pa) {
  __shared__ int hist[kMaxParts + 1];
  __shared__ int offs[kMaxParts];
  if (a.dhdr->status != 0) return;  // the build failed
  const Lookup L = read_lookup(a);
  const int P = pa.parts;
  const int64_t nq = a.n >> 2;
  const unsigned lt = lanemask_lt();
  for (int64_t t = blockIdx.x; t < pa.ntiles; t += gridDim.x) {
    for (int i = threadIdx.x; i <= P; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // ---- filter + probe this thread's two quads; up to 8 tuples in registers
    uint32_t gs[8];
    int64_t vv[8];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t q = t * (kPartTile / 4) + threadIdx.x + k * kScatterThreads;
#pragma unroll
      for (int r = 0; r < 4; ++r) gs[4 * k + r] = kEmpty32;
      if (q >= nq) continue;
      const int64_t row0 = q << 2;
      uint32_t bits = 0;
      uint64_t key[4];
      if (kVec) {
        const int4 p4 = __ldcs(reinterpret_cast<const int4*>(a.pred) + q);
        bits = (uint32_t)cmp_op(p4.x, a.lit, a.op) | ((uint32_t)cmp_op(p4.y, a.lit, a.op) << 1) |
               ((uint32_t)cmp_op(p4.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(p4.w, a.lit, a.op) << 3);
        if (!bits) continue;
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
        if (!bits) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          key[r] = kWide ? pack_key64(a.fk_hi[row0 + r], a.fk[row0 + r]) : (uint64_t)(uint32_t)a.fk[row0 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (!((bits >> r) & 1u)) continue;
        vv[4 * k + r] = __ldcs(a.val + row0 + r);
        gs[4 * k + r] = first_match<kWide>(a, L, key[r], vv[4 * k + r]);
      }
    }
    // ---- histogram by partition (warp lanes with equal partitions combined)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool has = gs[j] != kEmpty32;
      const int p = has ? (int)(gs[j] >> kPartShift) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, p);
      if (has && (peers & lt) == 0) atomicAdd(&hist[p], __popc(peers));
    }
    __syncthreads();
    // ---- exclusive scan of the histogram (one warp), prefix row to global memory
    if (threadIdx.x < 32) {
      int carry = 0;
      for (int base = 0; base <= P; base += 32) {
        const int i = base + (int)threadIdx.x;
        const int v = i < P ? hist[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, incl, o);
          if ((int)threadIdx.x >= o) incl += u;
        }
        const int excl = carry + incl - v;
        if (i < P) offs[i] = excl;
        if (i <= P) pa.prefix[t * (P + 1) + i] = excl;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    // ---- scatter the tuples into the tile's region, grouped by partition
    const int64_t base = t * (int64_t)kPartTile;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool has = gs[j] != kEmpty32;
      const int p = has ? (int)(gs[j] >> kPartShift) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, p);
      int start = 0;
      const int leader = __ffs(peers) - 1;
      if (has && (int)(threadIdx.x & 31) == leader) start = atomicAdd(&offs[p], __popc(peers));
      start = __shfl_sync(0xffffffffu, start, leader);
      if (has) {
        const int64_t pos = base + start + __popc(peers & lt);
        pa.tgs[pos] = gs[j];
        pa.tval[pos] = vv[j];
      }
    }
    __syncthreads();
  }
  // ragged tail (n % 4 rows): aggregated directly
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < a.n - (nq << 2))
    probe_one<kWide, kAggGlobal>(a, SmemAggs{}, L, (nq << 2) + threadIdx.x);
}

// Pass 2: block (k, p) aggregates partition p over tiles [k * per, (k + 1) * per).
__global__ void __launch_bounds__(kAggThreads)
part_agg_kernel(PartArgs pa, Agg* tab, int64_t gslots, uint32_t aggs, int64_t tiles_per_block) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  Agg* s_tab = reinterpret_cast<Agg*>(smem_raw);
  const int p = blockIdx.y;
  const int P = pa.parts;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int i = threadIdx.x; i < kPartSlots; i += blockDim.x) agg_identity(&s_tab[i]);
  __syncthreads();
  const int64_t t0 = blockIdx.x * tiles_per_block;
  const int64_t t1 = t0 + tiles_per_block < pa.ntiles ? t0 + tiles_per_block : pa.ntiles;
  const uint32_t slot0 = (uint32_t)p << kPartShift;
  for (int64_t tb = t0 + (int64_t)warp * 32; tb < t1; tb += (int64_t)nwarps * 32) {
    // lane l owns tile tb + l: its segment [off, off + cnt) of partition p
    const int64_t t = tb + lane;
    int off = 0, cnt = 0;
    if (t < t1) {
      off = pa.prefix[t * (P + 1) + p];
      cnt = pa.prefix[t * (P + 1) + p + 1] - off;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - cnt;
    // walk the concatenated segments: element e belongs to the lane whose range holds it
    for (int e0 = 0; e0 < total; e0 += 32) {
      const int e = e0 + lane;
      int owner = 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {  // binary search of e over the lanes' exclusive prefixes
        const int probe_lane = owner + o;
        const int ex = __shfl_sync(0xffffffffu, excl, probe_lane < 32 ? probe_lane : 31);
        if (probe_lane < 32 && ex <= e) owner = probe_lane;
      }
      const int oex = __shfl_sync(0xffffffffu, excl, owner);
      const int ooff = __shfl_sync(0xffffffffu, off, owner);
      if (e < total) {
        const int64_t pos = (tb + owner) * (int64_t)kPartTile + ooff + (e - oex);
        const uint32_t g = pa.tgs[pos] - slot0;
        const long long v = pa.tval[pos];
        Agg* s = &s_tab[g];
        if (aggs & SIRIUS_AGG_SUM) atomicAdd(&s->sum, (unsigned long long)v);
        atomicAdd(&s->count, 1ull);
        if (aggs & SIRIUS_AGG_MIN) atomicMin(&s->min, v);
        if (aggs & SIRIUS_AGG_MAX) atomicMax(&s->max, v);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPartSlots; i += blockDim.x) {
    const int64_t g = (int64_t)slot0 + i;
    if (g >= gslots) break;
    const Agg s = s_tab[i];
    if (s.count) agg_merge_global(&tab[g], s.sum, s.count, s.min, s.max, aggs);
  }
}

}  // namespace part
}  // namespace sirius
