// The staged probe pass: the same filter -> probe -> aggregate work as probe_quad, organised so
// that a thread never waits on its own memory accesses one at a time.
//
// A persistent block (one per SM, 16 warps) walks tiles of 512 fact rows.  Thread 0 streams
// the column slices of a tile (pred, fk [, fk_hi], val) into shared memory with 1-D TMA bulk
// copies, kColStages - 1 tiles ahead, each stage tracked by an mbarrier.  Each warp owns 32
// rows of a tile, one per lane: it evaluates the predicate, ranks the selected rows with one
// ballot and popcount (stream compaction), writes a (key, val) record per selected row into a
// ring slot and issues the gather of that row's 32-byte home bucket with two cp.async copies
// into the same slot -- no register waits on it.  The records of tile i are examined kDelay
// iterations later, when their buckets have landed: match, aggregate (global reductions),
// and only when a home bucket is full without a decision does the walk go on in global memory.
// Bounded waits: an mbarrier wait that exceeds its bound reports TIMEOUT in the run status.
#pragma once

#include "pipeline.cuh"

namespace sirius {
namespace staged {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = kWarps * 32;  // 512 rows, one per thread
constexpr int kColStages = 4;       // column tiles: the one being selected + 3 in flight
constexpr int kDelay = 4;           // iterations between a gather's issue and its use
constexpr int kRing = kDelay + 1;   // record/bucket ring slots
constexpr int kSpin = 1 << 22;

struct __align__(16) Rec {
  uint64_t key;
  int64_t val;
};

__host__ __device__ constexpr size_t stage_bytes(bool wide) { return (size_t)kTile * (wide ? 20 : 16); }
__host__ __device__ constexpr size_t smem_bytes(bool wide) {
  return kColStages * stage_bytes(wide)                 // column tiles
         + (size_t)kRing * kTile * (sizeof(Rec) + 32)   // records + gathered buckets
         + (size_t)kRing * kWarps * 4                   // selected rows per warp and slot
         + kColStages * 8 + 16;                         // mbarriers + timeout flag
}

// Continue a probe in global memory from the bucket after `slot` (the home bucket was full).
template <bool kWide>
__device__ __noinline__ void walk_global(const ProbeArgs& a, bool dups, uint64_t key, int64_t v, uint32_t slot) {
  constexpr int kPer = kWide ? 2 : 4;
  for (uint32_t step = kPer; step < a.jcap; step += kPer) {
    slot += kPer;
    if (slot >= a.jcap) slot = 0;
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
          agg_update_global(&a.tab[p], v, a.aggs);
          stop = !dups;
        }
      }
    }
    if (stop) return;
  }
}

template <bool kWide>
__global__ void __launch_bounds__(kThreads, 1) probe_staged_kernel(ProbeArgs a, int32_t* run_status) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr size_t kStage = stage_bytes(kWide);
  unsigned char* cols = sm;
  Rec* recs = reinterpret_cast<Rec*>(sm + kColStages * kStage);               // [kRing][kTile]
  uint4* bkts = reinterpret_cast<uint4*>(recs + (size_t)kRing * kTile);        // [kRing][kTile][2]
  int* cnt = reinterpret_cast<int*>(bkts + (size_t)kRing * kTile * 2);         // [kRing][kWarps]
  uint64_t* bars = reinterpret_cast<uint64_t*>(cnt + kRing * kWarps);          // [kColStages]
  int* timed_out = reinterpret_cast<int*>(bars + kColStages);

  if (a.dhdr->status != 0) return;  // the build failed: nothing to aggregate
  const Lookup L = read_lookup(a);
  const bool dups = L.dups;
  if (L.direct) {
    // dense keys: the direct array needs no gathered buckets; probe the rows in place
    const int64_t nq = a.n >> 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x)
      probe_quad<kWide, kAggGlobal, true>(a, SmemAggs{}, L, q);
    if (blockIdx.x == 0 && (int64_t)threadIdx.x < a.n - (nq << 2))
      probe_one<kWide, kAggGlobal>(a, SmemAggs{}, L, (nq << 2) + threadIdx.x);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nfull = (a.n >> 2) << 2;  // rows moved by TMA; the n % 4 tail goes scalar
  const int64_t ntiles = (nfull + kTile - 1) / kTile;
  const int64_t nlocal = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kColStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    *timed_out = 0;
  }
  __syncthreads();

  auto issue = [&](int64_t i) {  // thread 0: TMA of local tile i into column stage i % kColStages
    const int64_t r0 = (blockIdx.x + i * gridDim.x) * (int64_t)kTile;
    const uint32_t rows = (uint32_t)(nfull - r0 < kTile ? nfull - r0 : kTile);
    unsigned char* st = cols + (i % kColStages) * kStage;
    uint64_t* bar = &bars[i % kColStages];
    fence_proxy_async_smem();
    mbar_expect_tx(bar, rows * (kWide ? 20u : 16u));
    tma_load_1d(st, a.pred + r0, rows * 4, bar);
    tma_load_1d(st + kTile * 4, a.fk + r0, rows * 4, bar);
    if (kWide) tma_load_1d(st + kTile * 8, a.fk_hi + r0, rows * 4, bar);
    tma_load_1d(st + kTile * (kWide ? 12 : 8), a.val + r0, rows * 8, bar);
  };
  if (threadIdx.x == 0)
    for (int64_t i = 0; i < kColStages - 1 && i < nlocal; ++i) issue(i);

  for (int64_t i = 0; i < nlocal + kDelay; ++i) {
    if (threadIdx.x == 0 && i + kColStages - 1 < nlocal) issue(i + kColStages - 1);
    if (i < nlocal) {
      // ---- select tile i, write records, issue the bucket gathers
      const int slot = (int)(i % kRing);
      if (!mbar_wait(&bars[i % kColStages], (uint32_t)((i / kColStages) & 1), kSpin)) *timed_out = 1;
      const unsigned char* st = cols + (i % kColStages) * kStage;
      const int32_t* pred_s = reinterpret_cast<const int32_t*>(st);
      const int32_t* fk_s = reinterpret_cast<const int32_t*>(st + kTile * 4);
      const int32_t* fkh_s = reinterpret_cast<const int32_t*>(st + kTile * 8);
      const int64_t* val_s = reinterpret_cast<const int64_t*>(st + kTile * (kWide ? 12 : 8));
      const int64_t r0 = (blockIdx.x + i * gridDim.x) * (int64_t)kTile;
      const int rows = (int)(nfull - r0 < kTile ? nfull - r0 : kTile);
      const int r = warp * 32 + lane;
      const bool sel = r < rows && cmp_op(pred_s[r], a.lit, a.op);
      const unsigned b = __ballot_sync(0xffffffffu, sel);
      if (sel) {
        const int e = warp * 32 + __popc(b & lanemask_lt());
        const uint64_t key = kWide ? pack_key64(fkh_s[r], fk_s[r]) : (uint64_t)(uint32_t)fk_s[r];
        recs[(size_t)slot * kTile + e] = Rec{key, val_s[r]};
        const uint32_t home = kWide ? home_slot64(key, a.jcap) : home_slot32((uint32_t)key, a.jcap);
        const char* src = reinterpret_cast<const char*>(a.jslots) + (size_t)home * (kWide ? 16 : 8);
        uint4* dst = bkts + ((size_t)slot * kTile + e) * 2;
        cp_async16(dst, src);
        cp_async16(dst + 1, src + 16);
      }
      if (lane == 0) cnt[slot * kWarps + warp] = __popc(b);
    }
    cp_async_commit();
    if (i >= kDelay) {
      // ---- examine the records of tile i - kDelay: their buckets have landed
      cp_async_wait<kDelay>();
      __syncwarp();
      const int slot = (int)((i - kDelay) % kRing);
      if (lane < cnt[slot * kWarps + warp]) {
        const size_t e = (size_t)slot * kTile + warp * 32 + lane;
        const Rec rc = recs[e];
        const uint4 q0 = bkts[e * 2], q1 = bkts[e * 2 + 1];
        const uint64_t w[4] = {((uint64_t)q0.y << 32) | q0.x, ((uint64_t)q0.w << 32) | q0.z,
                               ((uint64_t)q1.y << 32) | q1.x, ((uint64_t)q1.w << 32) | q1.z};
        constexpr int kPer = kWide ? 2 : 4;
        bool stop = false;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const uint64_t k = kWide ? w[2 * j] : (uint64_t)(uint32_t)w[j];
          const uint32_t p = kWide ? (uint32_t)w[2 * j + 1] : (uint32_t)(w[j] >> 32);
          if (!stop) {
            if (p == kEmpty32) {
              stop = true;
            } else if (k == rc.key) {
              agg_update_global(&a.tab[p], rc.val, a.aggs);
              stop = !dups;
            }
          }
        }
        if (!stop) {
          const uint32_t home = kWide ? home_slot64(rc.key, a.jcap) : home_slot32((uint32_t)rc.key, a.jcap);
          walk_global<kWide>(a, dups, rc.key, rc.val, home);
        }
      }
    }
    __syncthreads();  // column stage i % kColStages may be refilled from the next iteration on
  }
  cp_async_wait<0>();
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < a.n - nfull)
    probe_one<kWide, kAggGlobal>(a, SmemAggs{}, L, nfull + threadIdx.x);
  if (threadIdx.x == 0 && *timed_out) set_status(run_status, SIRIUS_ERR_TIMEOUT);
}

}  // namespace staged
}  // namespace sirius
