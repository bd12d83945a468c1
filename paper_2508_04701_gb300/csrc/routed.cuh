// The fused probe pass with routed aggregation (agg_mode 5): every joined row's (group slot,
// value) is sent to the block that owns the slot, which aggregates it in shared memory.
//
// With many groups spread evenly (the 600M-row query: 100 000 groups over 180M joined rows) no
// block sees a group often enough to pre-aggregate it, and reducing into the global table costs
// four L2 reductions per joined row (SUM, COUNT, MIN, MAX) on top of the column stream -- the
// L2's request rate, not DRAM, bounds that pass.  Here the group slots are dealt out to the
// first P blocks (P a power of two; slot g belongs to block g & (P-1), at local index g >> logP),
// each holding its share of the aggregates in shared memory for the whole launch, and the rows
// travel to their owner through an L2-resident exchange:
//
//   * the fact rows are processed in rounds; in each round every block filters and probes
//     `iters` tiles of 4 x blockDim rows, sorts each tile's (slot, value) tuples by owner in
//     shared memory, and appends each owner's run to its own region of the exchange buffer
//     [buffer][owner][block][C] with coalesced stores (a few L2 requests per run instead of four
//     reductions per row);
//   * one grid-wide barrier per round; after it, each owner reads what every block sent it in
//     the round before (two buffers alternate, so a round's tuples are consumed while the next
//     round is produced) and applies them with shared-memory atomics;
//   * at the end each owner merges its slots into the global table (four reductions per group,
//     not per row).
//
// A run longer than C (skewed groups) sends its extra tuples straight to the global table as
// reductions, so any distribution gives the exact result.  Duplicate build keys (a row may
// match many build rows) take the global-reduction pass for the whole launch.  Every block is
// resident (cooperative launch); the barrier waits are bounded and end the launch with
// SIRIUS_ERR_TIMEOUT in the run header when they run out.
#pragma once

#include "pipeline.cuh"

namespace sirius {
namespace routed {

constexpr int kThreads = 512;                   // one quad (four rows) per thread per tile
constexpr int kTileRows = 4 * kThreads;
constexpr int kMaxOwners = 256;
constexpr int kIters = 16;                      // tiles per block per round
constexpr size_t kMaxOwnerBytes = 56000;         // owner table in shared memory: 2000 slots, so
                                                // that two blocks fit an SM
constexpr uint32_t kMaxOwnerSlots = (uint32_t)(kMaxOwnerBytes / 28);
constexpr int kBlocksPerSm = 2;

struct RouteArgs {
  int64_t* tval;      // [2][P][B][C] values
  uint16_t* tls;      // [2][P][B][C] owner-local slots
  uint32_t* fill;     // [2][B][P] tuples block b sent owner p in the round (runs longer than C
                      //            sent the rest to the global table)
  uint32_t* bar;      // grid barrier arrivals (zero at launch)
  int32_t* status;    // run status word
  int32_t logP;       // P = 1 << logP owners, P <= gridDim.x
  uint32_t R;         // slots per owner: ceil(gslots / P)
  uint32_t C;         // tuple capacity of one (owner, block) run per round
  int32_t iters;      // tiles per block per round
  int64_t rounds;
};

// Shared memory of one block: owner table (28 bytes per slot), one tile's tuples twice -- as
// produced (value, owner and local slot, rank among the owner's tuples) and grouped by owner
// (value, local slot, owner) -- and counters.  Keeping the produced tuples in shared memory
// rather than in registers across the tile's barriers keeps the kernel within the registers of
// two resident blocks per SM.
__host__ __device__ constexpr size_t stage_bytes() { return (size_t)kTileRows * (8 + 4 + 2 + 8 + 2 + 2); }
__host__ __device__ constexpr size_t owner_bytes(uint32_t R) { return ((size_t)R * 28 + 15) / 16 * 16; }
__host__ __device__ constexpr size_t counter_bytes() { return (size_t)(2 + 1 + 2) * kMaxOwners * 4 + 16; }
__host__ __device__ constexpr size_t smem_bytes(uint32_t R) {
  return owner_bytes(R) + stage_bytes() + counter_bytes();
}

// Capacity of one (owner, block) run: twice the mean share of a round's tiles when every row
// joins, in whole 32-tuple chunks.
inline uint32_t run_capacity(int P, int iters) {
  const int64_t mean = (int64_t)iters * kTileRows / P;
  return (uint32_t)(((2 * mean + 31) / 32) * 32);
}

// Load, filter and probe quad q (rows 4q .. 4q+3, below n); row r's match goes to
// emit(r, group slot, value).  No duplicate build keys: at most one match per row.
template <bool kWide, bool kVec, class Emit>
__device__ __forceinline__ void route_quad(const ProbeArgs& a, const Lookup& L, int64_t q, Emit&& emit) {
  const int64_t row0 = q << 2;
  uint32_t bits = 0;
  uint64_t key[4];
  int64_t vv[4];
  if (kVec) {
    // the quad's predicates, keys and values requested together (a quad's values are one
    // 32-byte sector, needed whenever any of its rows is selected)
    const int4 p4 = __ldcs(reinterpret_cast<const int4*>(a.pred) + q);
    const int4 k4 = __ldcs(reinterpret_cast<const int4*>(a.fk) + q);
    int4 h4 = make_int4(0, 0, 0, 0);
    if (kWide) h4 = __ldcs(reinterpret_cast<const int4*>(a.fk_hi) + q);
#pragma unroll
    for (int r = 0; r < 4; ++r) vv[r] = __ldcs(a.val + row0 + r);
    bits = (uint32_t)cmp_op(p4.x, a.lit, a.op) | ((uint32_t)cmp_op(p4.y, a.lit, a.op) << 1) |
           ((uint32_t)cmp_op(p4.z, a.lit, a.op) << 2) | ((uint32_t)cmp_op(p4.w, a.lit, a.op) << 3);
    key[0] = kWide ? pack_key64(h4.x, k4.x) : (uint64_t)(uint32_t)k4.x;
    key[1] = kWide ? pack_key64(h4.y, k4.y) : (uint64_t)(uint32_t)k4.y;
    key[2] = kWide ? pack_key64(h4.z, k4.z) : (uint64_t)(uint32_t)k4.z;
    key[3] = kWide ? pack_key64(h4.w, k4.w) : (uint64_t)(uint32_t)k4.w;
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool sel = cmp_op(a.pred[row0 + r], a.lit, a.op);
      bits |= (uint32_t)sel << r;
      key[r] = sel ? (kWide ? pack_key64(a.fk_hi[row0 + r], a.fk[row0 + r]) : (uint64_t)(uint32_t)a.fk[row0 + r])
                   : 0;
      vv[r] = sel ? __ldcs(a.val + row0 + r) : 0;
    }
  }
  if (!bits) return;
  if (!kWide && L.direct) {
    probe_rows_emit<kWide, false>(a, L, bits, key, vv, emit);
    return;
  }
  // hash table: two rows' buckets at a time (the registers of two resident blocks per SM)
  probe_rows_emit<kWide, false, 2>(a, L, bits & 3u, key, vv, emit);
  const uint64_t k2[4] = {key[2], key[3], 0, 0};
  const int64_t v2[4] = {vv[2], vv[3], 0, 0};
  probe_rows_emit<kWide, false, 2>(a, L, (bits >> 2) & 3u, k2, v2,
                                   [&](int r, uint32_t g, int64_t val) { emit(r + 2, g, val); });
}

template <bool kWide, bool kVec>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) probe_routed_kernel(ProbeArgs a, RouteArgs ra) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  if (a.dhdr->status != 0) return;  // the build failed: nothing to aggregate (every block leaves)
  const Lookup L = read_lookup(a);
  const int64_t nq = a.n >> 2;
  const int tid = threadIdx.x;
  if (L.dups) {
    // a row may match many build rows: global reductions for the whole launch (every block)
    for (int64_t q = blockIdx.x * (int64_t)kThreads + tid; q < nq; q += (int64_t)gridDim.x * kThreads)
      route_quad<kWide, kVec>(a, L, q, [&](int, uint32_t g, int64_t val) { agg_update_global(&a.tab[g], val, a.aggs); });
    if (blockIdx.x == 0 && tid < a.n - (nq << 2)) {
      const SmemAggs none{};
      probe_one<kWide, kAggGlobal>(a, none, L, (nq << 2) + tid);
    }
    return;
  }
  const int B = gridDim.x;
  const int logP = ra.logP;
  const uint32_t P = 1u << logP;
  const uint32_t R = ra.R;
  const uint32_t C = ra.C;
  const bool owner = blockIdx.x < P;
  // shared memory
  const SmemAggs T = smem_aggs(smem_raw, R);
  unsigned char* p = smem_raw + owner_bytes(R);
  int64_t* s_val = reinterpret_cast<int64_t*>(p);                          // grouped by owner
  int64_t* u_val = reinterpret_cast<int64_t*>(p + (size_t)kTileRows * 8);  // as produced
  uint32_t* u_dl = reinterpret_cast<uint32_t*>(p + (size_t)kTileRows * 16);
  uint16_t* u_rank = reinterpret_cast<uint16_t*>(p + (size_t)kTileRows * 20);
  uint16_t* s_ls = reinterpret_cast<uint16_t*>(p + (size_t)kTileRows * 22);
  uint16_t* s_dst = reinterpret_cast<uint16_t*>(p + (size_t)kTileRows * 24);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(p + stage_bytes());  // [2][kMaxOwners]
  uint32_t* s_off = s_cnt + 2 * kMaxOwners;                              // [kMaxOwners + 1]
  uint32_t* s_fill = s_off + kMaxOwners + 4;                             // [2][kMaxOwners]
  if (owner)
    for (uint32_t i = tid; i < R; i += kThreads) smem_identity(T, i);
  for (int i = tid; i < 2 * kMaxOwners; i += kThreads) {
    s_cnt[i] = 0;
    s_fill[i] = 0;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kThreads / 32;
  uint32_t passed = 0;
  for (int64_t r = 0; r <= ra.rounds; ++r) {
    const int buf = (int)(r & 1);
    if (r < ra.rounds) {
      // ---- produce round r into buffer `buf`
      for (int it = 0; it < ra.iters; ++it) {
        const int par = it & 1;
        uint32_t* cnt = s_cnt + par * kMaxOwners;
        const int64_t q = ((r * ra.iters + it) * B + blockIdx.x) * (int64_t)kThreads + tid;
#pragma unroll
        for (int k = 0; k < 4; ++k) u_dl[tid * 4 + k] = kEmpty32;
        if (q < nq)
          route_quad<kWide, kVec>(a, L, q, [&](int k, uint32_t g, int64_t val) {
            const int u = tid * 4 + k;
            const uint32_t d = g & (P - 1);
            u_rank[u] = (uint16_t)atomicAdd(&cnt[d], 1u);
            u_dl[u] = (d << 16) | (g >> logP);
            u_val[u] = val;
          });
        __syncthreads();
        if (warp == 0) {
          // exclusive scan of the owners' counts (each lane eight consecutive owners); the run
          // bases of the next tile; counters of this parity cleared for the tile after next
          constexpr int kPer = kMaxOwners / 32;
          uint32_t c[kPer], sum = 0;
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const uint32_t d = lane * kPer + j;
            c[j] = d < P ? cnt[d] : 0u;
            sum += c[j];
          }
          uint32_t incl = sum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          uint32_t run = incl - sum;
#pragma unroll
          for (int j = 0; j < kPer; ++j) {
            const uint32_t d = lane * kPer + j;
            if (d < P) {
              s_off[d] = run;
              s_fill[(par ^ 1) * kMaxOwners + d] = s_fill[par * kMaxOwners + d] + c[j];
              cnt[d] = 0;
            }
            run += c[j];
          }
          if (lane == 31) s_off[kMaxOwners] = incl;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int u = tid * 4 + k;
          const uint32_t dl = u_dl[u];
          if (dl != kEmpty32) {
            const uint32_t d = dl >> 16;
            const uint32_t pos = s_off[d] + u_rank[u];
            s_val[pos] = u_val[u];
            s_ls[pos] = (uint16_t)(dl & 0xFFFFu);
            s_dst[pos] = (uint16_t)d;
          }
        }
        __syncthreads();
        // the tile's tuples, grouped by owner, appended to the owners' runs of this block
        const uint32_t total = s_off[kMaxOwners];
        const uint32_t* fill0 = s_fill + par * kMaxOwners;
        for (uint32_t i = tid; i < total; i += kThreads) {
          const uint32_t d = s_dst[i];
          const uint32_t at = fill0[d] + (i - s_off[d]);
          const int64_t val = s_val[i];
          const uint16_t ls = s_ls[i];
          if (at < C) {
            const size_t idx = (((size_t)buf * P + d) * B + blockIdx.x) * C + at;
            ra.tval[idx] = val;
            ra.tls[idx] = ls;
          } else {
            agg_update_global(&a.tab[((uint32_t)ls << logP) | d], val, a.aggs);
          }
        }
      }
      // publish the round's run lengths (their final values sit in the parity after the last tile)
      const uint32_t* fin = s_fill + (ra.iters & 1) * kMaxOwners;
      __syncthreads();
      for (uint32_t d = tid; d < P; d += kThreads) {
        ra.fill[((size_t)buf * B + blockIdx.x) * P + d] = fin[d];
      }
      __syncthreads();
      for (uint32_t d = tid; d < P; d += kThreads) {  // the next round's runs start empty
        s_fill[d] = 0;
        s_fill[kMaxOwners + d] = 0;
      }
    }
    if (r > 0 && owner) {
      // ---- consume round r-1: the runs every block sent this owner, two runs per warp at once
      const int cb = (int)((r - 1) & 1);
      for (int j0 = warp; j0 < B; j0 += 32 * kWarps) {
        const int srcl = j0 + lane * kWarps;  // this lane holds the length of run `srcl`
        uint32_t c = 0;
        if (srcl < B) {
          c = __ldcg(&ra.fill[((size_t)cb * B + srcl) * P + blockIdx.x]);
          c = c < C ? c : C;
        }
        for (int k = 0; k < 32 && j0 + k * kWarps < B; k += 2) {
          const uint32_t c0 = __shfl_sync(0xffffffffu, c, k);
          const uint32_t c1 = __shfl_sync(0xffffffffu, c, k + 1);
          const int s0 = j0 + k * kWarps, s1 = j0 + (k + 1) * kWarps;
          const size_t b0 = (((size_t)cb * P + blockIdx.x) * B + s0) * C;
          const size_t b1 = (((size_t)cb * P + blockIdx.x) * B + (s1 < B ? s1 : s0)) * C;
          const uint32_t cmax = c0 > c1 ? c0 : c1;
          for (uint32_t off = lane; off < cmax; off += 64) {
            const bool x0 = off < c0, y0 = off + 32 < c0, x1 = off < c1, y1 = off + 32 < c1;
            const int64_t v0 = x0 ? __ldcg(ra.tval + b0 + off) : 0;
            const int64_t w0 = y0 ? __ldcg(ra.tval + b0 + off + 32) : 0;
            const int64_t v1 = x1 ? __ldcg(ra.tval + b1 + off) : 0;
            const int64_t w1 = y1 ? __ldcg(ra.tval + b1 + off + 32) : 0;
            const uint16_t l0 = x0 ? __ldcg(ra.tls + b0 + off) : 0;
            const uint16_t m0 = y0 ? __ldcg(ra.tls + b0 + off + 32) : 0;
            const uint16_t l1 = x1 ? __ldcg(ra.tls + b1 + off) : 0;
            const uint16_t m1 = y1 ? __ldcg(ra.tls + b1 + off + 32) : 0;
            if (x0) agg_update_smem(T, l0, v0, a.aggs);
            if (y0) agg_update_smem(T, m0, w0, a.aggs);
            if (x1) agg_update_smem(T, l1, v1, a.aggs);
            if (y1) agg_update_smem(T, m1, w1, a.aggs);
          }
        }
      }
    }
    if (r < ra.rounds) {
      if (!grid_barrier(ra.bar, ++passed * (uint32_t)B, ra.status)) return;
    }
  }
  // the last n % 4 rows: straight to the global table
  if (blockIdx.x == 0 && tid < a.n - (nq << 2)) {
    const SmemAggs none{};
    probe_one<kWide, kAggGlobal>(a, none, L, (nq << 2) + tid);
  }
  if (owner) {
    __syncthreads();
    for (uint32_t i = tid; i < R; i += kThreads) {
      const uint32_t g = (i << logP) | blockIdx.x;
      if (g < a.gslots) smem_merge(T, i, &a.tab[g], a.aggs);
    }
  }
}

}  // namespace routed
}  // namespace sirius
