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
// first slot loads in flight together, and aggregates
//   - into a per-block copy of the aggregates in shared memory when the group table is small
//     (few groups contend on chip, not in L2), merged into the global table at block exit;
//   - with global atomics otherwise (SUM and COUNT as reductions; MIN/MAX only when the value
//     beats the one already stored).
// Finalize compacts the slots with COUNT > 0 into the caller's output arrays.
#include "tables.cuh"
#include "pipeline.cuh"

namespace sirius {

namespace {

__global__ void pipe_init_kernel(PipeHeader* phdr, JoinHeader* jhdr, ulonglong2* jwords2,
                                 int64_t jpairs, int64_t* gkeys, Agg* aggs, int64_t gslots) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid < 32) {
    reinterpret_cast<uint64_t*>(phdr)[tid] = 0;
    if (jhdr) reinterpret_cast<uint64_t*>(jhdr)[tid] = 0;
  }
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  for (int64_t i = tid; i < jpairs; i += stride) jwords2[i] = ones;
  for (int64_t i = tid; i < gslots; i += stride) {
    gkeys[i] = kEmptyKey;
    agg_identity(&aggs[i]);
  }
}

template <bool kWide>
__global__ void pipe_build_kernel(const int32_t* __restrict__ pk, const int32_t* __restrict__ pk_hi,
                                  const int32_t* __restrict__ grp, const int8_t* __restrict__ flag,
                                  int64_t m, void* jslots, uint32_t jcap, JoinHeader* jhdr,
                                  int64_t* gkeys, uint32_t gcap, PipeHeader* phdr,
                                  unsigned long long glimit) {
  bool dup = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gk = group_key(grp[j], flag, j);
    const int64_t gs = group_find_or_insert(gkeys, gcap, gk, &phdr->distinct, glimit);
    if (gs < 0) {
      set_status(&phdr->status, SIRIUS_ERR_TABLE_FULL);
      continue;
    }
    bool ok;
    if (kWide) {
      ok = join_insert64((ulonglong2*)jslots, jcap, pack_key64(pk_hi[j], pk[j]), (uint32_t)gs, dup);
    } else {
      const uint32_t key = (uint32_t)pk[j];
      ok = join_insert32((uint64_t*)jslots, jcap, key, (uint64_t)key | ((uint64_t)(uint32_t)gs << 32), dup);
    }
    if (!ok) set_status(&phdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) jhdr->has_dups = 1;
}

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
  Agg* tab;
  uint32_t gslots;
  const PipeHeader* phdr;
};

// One join-table slot as (key, payload); payload kEmpty32 = empty.
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

template <int kMode>
__device__ __forceinline__ void aggregate(const ProbeArgs& a, Agg* s_tab, uint32_t gs, int64_t v) {
  if (kMode == kAggSmem) {
    Agg* t = &s_tab[gs];
    if (a.aggs & SIRIUS_AGG_SUM) atomicAdd(&t->sum, (unsigned long long)v);
    atomicAdd(&t->count, 1ull);
    if ((a.aggs & SIRIUS_AGG_MIN) && v < t->min) atomicMin(&t->min, (long long)v);
    if ((a.aggs & SIRIUS_AGG_MAX) && v > t->max) atomicMax(&t->max, (long long)v);
  } else {
    agg_update_global(&a.tab[gs], v, a.aggs);
  }
}

// Probe `cnt` (<= 4) rows whose selection bits, keys and values are given; the first slot of
// every selected row is loaded before any walk continues.
template <bool kWide, int kMode>
__device__ __forceinline__ void probe_rows(const ProbeArgs& a, Agg* s_tab, bool dups, uint32_t bits,
                                           const uint64_t (&key)[4], const int64_t (&v)[4]) {
  uint32_t s[4];
  uint64_t sk[4];
  uint32_t pl[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if ((bits >> r) & 1u) {
      s[r] = kWide ? home_slot64(key[r], a.jcap) : home_slot32((uint32_t)key[r], a.jcap);
      load_slot<kWide>(a.jslots, s[r], sk[r], pl[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (!((bits >> r) & 1u)) continue;
    uint32_t slot = s[r];
    uint64_t k = sk[r];
    uint32_t p = pl[r];
    for (uint32_t step = 0; step < a.jcap && p != kEmpty32; ++step) {
      if (k == key[r]) {
        aggregate<kMode>(a, s_tab, p, v[r]);
        if (!dups) break;
      }
      slot = (slot + 1 == a.jcap) ? 0 : slot + 1;
      load_slot<kWide>(a.jslots, slot, k, p);
    }
  }
}

template <bool kWide, int kMode, bool kVec>
__global__ void __launch_bounds__(512)
pipe_probe_kernel(ProbeArgs a) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  Agg* s_tab = reinterpret_cast<Agg*>(smem_raw);
  if (a.phdr->status != 0) return;  // the build failed: nothing to aggregate
  const bool dups = a.jhdr->has_dups != 0;
  if (kMode == kAggSmem) {
    for (uint32_t i = threadIdx.x; i < a.gslots; i += blockDim.x) agg_identity(&s_tab[i]);
    __syncthreads();
  }
  const int64_t nq = a.n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += stride) {
    const int64_t row0 = q << 2;
    uint32_t bits = 0;
    uint64_t key[4];
    int64_t v[4];
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
    for (int r = 0; r < 4; ++r) v[r] = ((bits >> r) & 1u) ? __ldcs(a.val + row0 + r) : 0;
    probe_rows<kWide, kMode>(a, s_tab, dups, bits, key, v);
  }
  // ragged tail: the last n % 4 rows, one per thread of block 0
  const int64_t tail0 = nq << 2;
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < a.n - tail0) {
    const int64_t r = tail0 + threadIdx.x;
    if (cmp_op(a.pred[r], a.lit, a.op)) {
      uint64_t key[4] = {0, 0, 0, 0};
      int64_t v[4] = {0, 0, 0, 0};
      key[0] = kWide ? pack_key64(a.fk_hi[r], a.fk[r]) : (uint64_t)(uint32_t)a.fk[r];
      v[0] = a.val[r];
      probe_rows<kWide, kMode>(a, s_tab, dups, 1u, key, v);
    }
  }
  if (kMode == kAggSmem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < a.gslots; i += blockDim.x) {
      const Agg t = s_tab[i];
      if (t.count) agg_merge_global(&a.tab[i], t.sum, t.count, t.min, t.max, a.aggs);
    }
  }
}

__global__ void pipe_finalize_kernel(const int64_t* __restrict__ gkeys, const Agg* __restrict__ tab,
                                     int64_t gslots, uint32_t aggs, PipeOut out, PipeHeader* phdr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (gslots + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < gslots && tab[i].count > 0;
    const uint64_t pos = warp_append(&phdr->groups, occ);
    if (occ && (int64_t)pos < out.cap) {
      const Agg t = tab[i];
      if (out.keys) out.keys[pos] = gkeys[i];
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
      const int32_t st = *(volatile int32_t*)&phdr->status;
      if (out.d_groups) *out.d_groups = (int64_t)g;
      if (out.d_status) *out.d_status = (st == 0 && (int64_t)g > out.cap) ? SIRIUS_ERR_CAPACITY : st;
    }
  }
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

template <bool kWide, int kMode, bool kVec>
sirius_status launch_probe(const ProbeArgs& a, int threads, int blocks_per_sm, size_t smem, cudaStream_t s) {
  auto k = pipe_probe_kernel<kWide, kMode, kVec>;
  if (kMode == kAggSmem) {
    static bool attr = false;
    if (!attr) {
      SIRIUS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr = true;
    }
  }
  int per_sm = blocks_per_sm > 0 ? blocks_per_sm : occupancy_blocks(k, threads, smem);
  int64_t want = ((a.n >> 2) + threads - 1) / threads;
  if (want < 1) want = 1;
  int64_t g = (int64_t)sm_count() * per_sm;
  if (g > want) g = want;
  k<<<(unsigned)g, threads, smem, s>>>(a);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

template <bool kWide>
sirius_status dispatch_probe(const ProbeArgs& a, int mode, bool vec, int threads, int bps, size_t smem,
                             cudaStream_t s) {
  if (mode == kAggSmem)
    return vec ? launch_probe<kWide, kAggSmem, true>(a, threads, bps, smem, s)
               : launch_probe<kWide, kAggSmem, false>(a, threads, bps, smem, s);
  return vec ? launch_probe<kWide, kAggGlobal, true>(a, threads, bps, 0, s)
             : launch_probe<kWide, kAggGlobal, false>(a, threads, bps, 0, s);
}

}  // namespace

PipeLayout pipe_layout(const sirius_pipeline_desc* q) {
  PipeLayout L;
  L.key_width = q->fk_hi ? 8 : 4;
  L.jcap = sirius_join_table_capacity(q->m, q->load_factor > 0 ? q->load_factor : 0.5);
  const int64_t hint = q->group_cap_hint > 0 ? q->group_cap_hint : (q->m > 0 ? q->m : 1);
  L.gcap = group_capacity_for(hint);
  L.off_phdr = 0;
  L.off_join = 256;
  L.off_gkeys = align_up(L.off_join + 256 + (size_t)L.jcap * (L.key_width == 8 ? 16 : 8), 256);
  L.off_aggs = align_up(L.off_gkeys + (size_t)(L.gcap + 1) * 8, 256);
  L.total = align_up(L.off_aggs + (size_t)(L.gcap + 1) * sizeof(Agg), 256);
  return L;
}

sirius_status validate_desc(const sirius_pipeline_desc* q) {
  SIRIUS_REQUIRE(q, "pipeline: NULL descriptor");
  SIRIUS_REQUIRE(q->n >= 0 && q->n <= kMaxRows && q->m >= 0 && q->m <= kMaxRows,
                 "pipeline: n=%lld m=%lld out of range", (long long)q->n, (long long)q->m);
  SIRIUS_REQUIRE(q->n == 0 || (q->fk && q->pred && q->val), "pipeline: NULL fact column");
  SIRIUS_REQUIRE(q->m == 0 || (q->pk && q->grp), "pipeline: NULL dim column");
  SIRIUS_REQUIRE((q->fk_hi == nullptr) == (q->pk_hi == nullptr) || q->n == 0 || q->m == 0,
                 "pipeline: fact and dim keys must both be one- or two-column");
  SIRIUS_REQUIRE(q->op >= SIRIUS_LT && q->op <= SIRIUS_NE, "pipeline: bad comparison %d", q->op);
  SIRIUS_REQUIRE(q->aggs <= SIRIUS_AGG_ALL, "pipeline: bad aggregate mask");
  SIRIUS_REQUIRE(q->agg_mode >= 0 && q->agg_mode <= 2, "pipeline: bad agg_mode %d", q->agg_mode);
  SIRIUS_REQUIRE(q->load_factor >= 0 && q->load_factor <= 0.95f, "pipeline: load_factor out of (0, 0.95]");
  SIRIUS_REQUIRE(q->block_threads == 0 || (q->block_threads % 32 == 0 && q->block_threads >= 64 &&
                                           q->block_threads <= 512),
                 "pipeline: block_threads must be a multiple of 32 in [64, 512]");
  const int64_t hint = q->group_cap_hint > 0 ? q->group_cap_hint : q->m;
  SIRIUS_REQUIRE(hint < (1ll << 30), "pipeline: group_cap_hint too large");
  return SIRIUS_OK;
}

int choose_mode(const sirius_pipeline_desc* q, const PipeLayout& L) {
  const bool fits = (L.gcap + 1) * (int64_t)sizeof(Agg) <= kSmemAggMaxBytes;
  if (q->agg_mode == kAggGlobal || !fits) return kAggGlobal;
  return kAggSmem;
}

sirius_status pipe_launch(const sirius_pipeline_desc* q, const PipeLayout& L, char* base,
                          const PipeOut& out, cudaStream_t s, bool build) {
  PipeHeader* phdr = (PipeHeader*)(base + L.off_phdr);
  JoinHeader* jhdr = (JoinHeader*)(base + L.off_join);
  void* jslots = base + L.off_join + 256;
  int64_t* gkeys = (int64_t*)(base + L.off_gkeys);
  Agg* tab = (Agg*)(base + L.off_aggs);
  const int64_t gslots = L.gcap + 1;
  const int64_t jpairs = build ? (L.jcap * (L.key_width == 8 ? 16 : 8) + 15) / 16 : 0;
  const int64_t init_n = jpairs > gslots ? jpairs : gslots;
  {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_INIT);
    pipe_init_kernel<<<grid_for(init_n, 256), 256, 0, s>>>(phdr, build ? jhdr : nullptr, (ulonglong2*)jslots,
                                                           jpairs, gkeys, tab, gslots);
    SIRIUS_LAUNCH_CHECK();
  }
  if (build && q->m > 0) {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_BUILD);
    const int g = grid_for(q->m, 256);
    if (L.key_width == 8)
      pipe_build_kernel<true><<<g, 256, 0, s>>>(q->pk, q->pk_hi, q->grp, q->flag, q->m, jslots,
                                                (uint32_t)L.jcap, jhdr, gkeys, (uint32_t)L.gcap, phdr,
                                                group_limit_for(L.gcap));
    else
      pipe_build_kernel<false><<<g, 256, 0, s>>>(q->pk, nullptr, q->grp, q->flag, q->m, jslots,
                                                 (uint32_t)L.jcap, jhdr, gkeys, (uint32_t)L.gcap, phdr,
                                                 group_limit_for(L.gcap));
    SIRIUS_LAUNCH_CHECK();
  }
  if (q->n > 0 && q->m > 0) {
    ProbeArgs a;
    a.fk = q->fk;
    a.fk_hi = q->fk_hi;
    a.pred = q->pred;
    a.val = q->val;
    a.n = q->n;
    a.op = q->op;
    a.lit = q->literal;
    a.aggs = q->aggs;
    a.jcap = (uint32_t)L.jcap;
    a.jslots = jslots;
    a.jhdr = jhdr;
    a.tab = tab;
    a.gslots = (uint32_t)gslots;
    a.phdr = phdr;
    const int mode = choose_mode(q, L);
    const bool vec = ((uintptr_t)q->pred & 15) == 0 && ((uintptr_t)q->fk & 15) == 0 &&
                     (!q->fk_hi || ((uintptr_t)q->fk_hi & 15) == 0);
    const int threads = q->block_threads > 0 ? q->block_threads : (mode == kAggSmem ? 512 : 256);
    const size_t smem = mode == kAggSmem ? (size_t)gslots * sizeof(Agg) : 0;
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_PROBE);
    sirius_status st = L.key_width == 8 ? dispatch_probe<true>(a, mode, vec, threads, q->blocks_per_sm, smem, s)
                                        : dispatch_probe<false>(a, mode, vec, threads, q->blocks_per_sm, smem, s);
    if (st != SIRIUS_OK) return st;
  }
  {
    PhaseTimer pt(s, SIRIUS_PHASE_PIPE_FINALIZE);
    pipe_finalize_kernel<<<grid_for(gslots, 256), 256, 0, s>>>(gkeys, tab, gslots, q->aggs, out, phdr);
    SIRIUS_LAUNCH_CHECK();
  }
  return SIRIUS_OK;
}

sirius_status pipe_sync_result(const PipeLayout& L, char* base, sirius_result* r, cudaStream_t s) {
  PipeHeader h;
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, base + L.off_phdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
  r->groups = (int64_t)h.groups;
  r->status = h.status;
  if (h.status) {
    set_error("pipeline: device status %d (%s)", h.status,
              h.status == SIRIUS_ERR_TABLE_FULL ? "more distinct group keys than group_cap_hint allows"
                                                : "device error");
    return (sirius_status)h.status;
  }
  if ((int64_t)h.groups > r->out_cap) {
    r->status = SIRIUS_ERR_CAPACITY;
    set_error("pipeline: %llu groups exceed out_cap %lld", h.groups, (long long)r->out_cap);
    return SIRIUS_ERR_CAPACITY;
  }
  return SIRIUS_OK;
}

}  // namespace sirius

using namespace sirius;

extern "C" size_t sirius_pipeline_scratch_bytes(const sirius_pipeline_desc* q) {
  if (!q) return 0;
  return pipe_layout(q).total;
}

extern "C" sirius_status sirius_run_pipeline(const sirius_pipeline_desc* q, sirius_result* result,
                                             void* d_scratch, size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = validate_desc(q);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(result, "pipeline: NULL result");
  SIRIUS_REQUIRE(result->out_cap >= 0, "pipeline: negative out_cap");
  SIRIUS_REQUIRE(result->out_cap == 0 || result->keys || result->count,
                 "pipeline: no output arrays");
  const PipeLayout L = pipe_layout(q);
  Scratch sc;
  st = sc.acquire(d_scratch, scratch_bytes, L.total, s);
  if (st != SIRIUS_OK) return st;
  PipeOut out{result->keys, result->sum, result->count, result->min, result->max, result->out_cap,
              result->d_groups, result->d_status};
  st = pipe_launch(q, L, sc.base, out, s, true);
  if (st != SIRIUS_OK) return st;
  if (result->sync) return pipe_sync_result(L, sc.base, result, s);
  return SIRIUS_OK;
}
