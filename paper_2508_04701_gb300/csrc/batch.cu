// A8: many independent pipelines in one set of persistent launches (pipelines as tasks of a
// global queue, Sec. 3.2.2; batch execution, Sec. 3.4).
//
// Every query's work is cut into units per phase -- initialisation (8192 table words), build
// (2048 dim rows), probe (rows_per_unit fact rows), finalize (4096 group slots).  One kernel per
// phase runs a fixed grid whose blocks walk the concatenated units of all queries (grid-stride,
// binary search for the unit's query), so a 10K-row query and a 20M-row query share the GPU
// without a launch of their own.  Phases are ordered by the stream (no device-side waits).
// Queries whose group table fits in shared memory aggregate each probe unit there and merge
// it into the global table at the unit's end.  The task table lives in plan-owned device
// memory and is refreshed by one host-to-device copy from pinned staging, so a CUDA graph
// captured once (copy in, five kernels, copy out) serves every later batch.
#include <algorithm>
#include <new>
#include <vector>

#include "pipeline.cuh"

namespace sirius {
namespace {

constexpr int kInitUnit = 8192;
constexpr int kBuildUnit = 2048;
constexpr int kFinUnit = 4096;
constexpr int kBatchThreads = 256;
constexpr int kProbeThreads = 512;

enum : uint32_t { kQWide = 1, kQSmem = 2, kQVec = 4, kQBuild = 8 };
// Bits 0-7 of a plan's class mask: probe classes with work; this bit: some dim builds two-column keys.
constexpr uint32_t kBuildWideBit = 1u << 8;

struct BatchQuery {
  ProbeArgs a;
  DimView d;
  PipeHeader* phdr;
  PipeOut out;
  const int32_t* pk;
  const int32_t* pk_hi;
  const int32_t* grp;
  const int8_t* flag;
  DimPred dpred;   // dim-side predicate of the build
  int64_t m;
  int64_t jpairs;  // 16-byte words of join slots (0 when the dim index is prebuilt)
  int64_t dpairs;  // 16-byte words of the direct array (0 when prebuilt or hash only)
  int64_t gslots;
  unsigned long long glimit;
  uint32_t flags;
  int32_t orig;    // position of the query in the caller's arrays
  // work units of this query: kinds 0 init (words), 1 build (dim rows), 2 probe (fact rows),
  // 3 finalize (group slots), 4 table clears (words)
  int64_t u0[5];   // first unit of this query in each kind
  int64_t nu[5];   // units of this query in each kind
};

struct BatchHeader {
  int32_t nq;
  int32_t pad;
  int64_t total[5];          // units per kind, all queries
  int64_t quads_per_unit;
  int32_t cls_q0[8], cls_q1[8];  // query range of each probe class (queries sorted by class)
  int64_t cls_u0[8], cls_u1[8];  // probe-unit range of each class
  int64_t pad2[1];
  // Probe blocks claim chunks of their class's units from cls_next (zero at every run: the
  // header is copied in from the host each time); cls_chunk units per claim.
  unsigned long long cls_next[8];
  int64_t cls_chunk[8];
  int64_t pad3[16];
};
static_assert(sizeof(BatchHeader) == 512, "batch header is 512 bytes");

struct BatchStatus {
  int64_t status;
  int64_t groups;
};

template <int P>
__device__ __forceinline__ int find_query(const BatchQuery* __restrict__ Q, int nq, int64_t u) {
  int lo = 0, hi = nq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (Q[mid].u0[P] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kBatchThreads)
batch_init_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q) {
  const int nq = H->nq;
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  for (int64_t u = blockIdx.x; u < H->total[0]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<0>(Q, nq, u)];
    const int64_t local = u - b.u0[0];
    const bool build = (b.flags & kQBuild) != 0;
    if (local == 0 && threadIdx.x < 32) {
      reinterpret_cast<uint64_t*>(b.phdr)[threadIdx.x] = 0;
      if (build) {
        // word 2 of the dim header: (key_min, key_max) = (INT32_MAX, INT32_MIN); words 4 and 5:
        // the group key range = (INT64_MAX, INT64_MIN)
        reinterpret_cast<uint64_t*>(b.d.dhdr)[threadIdx.x] = threadIdx.x == 2   ? 0x800000007FFFFFFFull
                                                             : threadIdx.x == 4 ? 0x7FFFFFFFFFFFFFFFull
                                                             : threadIdx.x == 5 ? 0x8000000000000000ull
                                                                                : 0ull;
        reinterpret_cast<uint64_t*>(b.d.jhdr)[threadIdx.x] = 0;
      }
    }
    // join slots are cleared here only for hash-only dims; otherwise by the clear phases
    const int64_t jw = (build && b.d.dcap == 0) ? b.jpairs : 0;
    const int64_t end = jw + b.gslots;
    const int64_t i1 = (local + 1) * kInitUnit < end ? (local + 1) * kInitUnit : end;
    for (int64_t i = local * kInitUnit + threadIdx.x; i < i1; i += blockDim.x) {
      if (i < jw) {
        reinterpret_cast<ulonglong2*>(b.d.jslots)[i] = ones;
      } else {
        const int64_t g = i - jw;
        if (build) b.d.gkeys[g] = kEmptyKey;
        agg_identity(&b.a.tab[g]);
      }
    }
  }
}

// Key range (the direct-array decision) and group key range (the direct group-slot decision)
// of every dim the batch builds.
__global__ void __launch_bounds__(kBatchThreads)
batch_minmax_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q) {
  const int nq = H->nq;
  for (int64_t u = blockIdx.x; u < H->total[1]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<1>(Q, nq, u)];
    const int64_t r0 = (u - b.u0[1]) * kBuildUnit;
    const int64_t r1 = r0 + kBuildUnit < b.m ? r0 + kBuildUnit : b.m;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    long long glo = INT64_MAX, ghi = INT64_MIN;
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
      const int32_t k = b.pk[j];
      lo = k < lo ? k : lo;
      hi = k > hi ? k : hi;
      const long long g = group_key(b.grp[j], b.flag, j);
      glo = g < glo ? g : glo;
      ghi = g > ghi ? g : ghi;
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    glo = warp_min_i64(glo);
    ghi = warp_max_i64(ghi);
    if ((threadIdx.x & 31) == 0 && lo <= hi) {
      atomicMin(&b.d.dhdr->key_min, lo);
      atomicMax(&b.d.dhdr->key_max, hi);
      atomicMin(&b.d.dhdr->gkey_min, glo);
      atomicMax(&b.d.dhdr->gkey_max, ghi);
    }
  }
}

// Table clears of dims that may take the direct array.  Phase 0 (before the build): the
// direct array when the key range fits it, else the join slots.  Phase 1 (after the build):
// the join slots when a duplicate key turned the direct array down.
__global__ void __launch_bounds__(kBatchThreads)
batch_clear_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q, int phase) {
  const int nq = H->nq;
  const ulonglong2 ones = make_ulonglong2(kEmpty64, kEmpty64);
  for (int64_t u = blockIdx.x; u < H->total[4]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<4>(Q, nq, u)];
    const bool direct = direct_applies(b.d, b.m);
    ulonglong2* w;
    int64_t words;
    if (phase == 0) {
      w = reinterpret_cast<ulonglong2*>(direct ? (void*)b.d.dslot : b.d.jslots);
      words = direct ? b.dpairs : b.jpairs;
    } else {
      if (!(b.d.dhdr->direct && b.d.dhdr->direct_failed)) continue;
      w = reinterpret_cast<ulonglong2*>(b.d.jslots);
      words = b.jpairs;
    }
    const int64_t i0 = (u - b.u0[4]) * kInitUnit;
    const int64_t i1 = i0 + kInitUnit < words ? i0 + kInitUnit : words;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) w[i] = ones;
  }
}

// One instantiation per key width (each skips the other width's queries), so that neither
// carries the registers of both insert paths.
template <bool kWide>
__global__ void __launch_bounds__(kBatchThreads)
batch_build_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q) {
  const int nq = H->nq;
  for (int64_t u = blockIdx.x; u < H->total[1]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<1>(Q, nq, u)];
    const int64_t local = u - b.u0[1];
    const int64_t r0 = local * kBuildUnit;
    const int64_t r1 = r0 + kBuildUnit < b.m ? r0 + kBuildUnit : b.m;
    if (((b.flags & kQWide) != 0) != kWide) continue;  // block-uniform
    const DimView d = b.d;
    const BuildMode B = read_build_mode(d, b.m, b.glimit, !kWide);
    if (local == 0 && threadIdx.x == 0) d.dhdr->direct = B.direct ? 1u : 0u;
    if (B.gdirect) {  // this unit's share of the slot keys
      const int64_t units = (b.m + kBuildUnit - 1) / kBuildUnit;
      const int64_t per = (B.grange + units - 1) / units;
      const int64_t i0 = local * per;
      const int64_t i1 = i0 + per < B.grange ? i0 + per : B.grange;
      fill_direct_group_keys(d, B, i0 + threadIdx.x, i1, blockDim.x);
    }
    bool dup = false;
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
      const bool ok = dim_build_row<kWide>(b.pk, b.pk_hi, b.grp, b.flag, j, d, b.glimit, dup, b.dpred, B);
      if (!ok) set_status(&d.dhdr->status, SIRIUS_ERR_TABLE_FULL);
    }
    if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) {
      if (B.direct) d.dhdr->direct_failed = 1;
      else d.jhdr->has_dups = 1;
    }
  }
}

// Rebuild into the hash table the dims whose direct array a duplicate key turned down.
__global__ void __launch_bounds__(kBatchThreads)
batch_fallback_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q) {
  const int nq = H->nq;
  for (int64_t u = blockIdx.x; u < H->total[1]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<1>(Q, nq, u)];
    const DimView d = b.d;
    if (!(d.dhdr->direct && d.dhdr->direct_failed)) continue;
    const int64_t r0 = (u - b.u0[1]) * kBuildUnit;
    const int64_t r1 = r0 + kBuildUnit < b.m ? r0 + kBuildUnit : b.m;
    BuildMode B = read_build_mode(d, b.m, b.glimit, true);
    B.direct = false;
    bool dup = false;
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x)
      if (!dim_build_row<false>(b.pk, nullptr, b.grp, b.flag, j, d, b.glimit, dup, b.dpred, B))
        set_status(&d.dhdr->status, SIRIUS_ERR_TABLE_FULL);
    if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) d.jhdr->has_dups = 1;
  }
}

// The probe phase runs one kernel per query class (key width, aggregation mode, vector
// loads), each specialised at compile time; the host orders the task table by class, so a
// class's queries -- and their probe units -- are contiguous.  Blocks claim chunks of
// consecutive units from a per-class counter (32 claims per block when the class has at least
// 32 units per block; else one chunk each), so a block that drew expensive units (high
// selectivity) does not hold up the others, and consecutive units
// of a block mostly belong to the same query: in shared-memory mode the block keeps that
// query's aggregates on chip across them and merges them into the global table only when its
// query changes (and at the end).  One
// 512-thread block per SM, with the registers for two quads in flight per thread (one-column
// keys through the direct array): the same loads in flight as two blocks of one quad each,
// without spills, and half the blocks to merge.
template <bool kWide, int kMode, bool kVec>
__global__ void __launch_bounds__(kProbeThreads, 1)
batch_probe_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q, int cls,
                   unsigned long long* next) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int64_t s_claim;
  const int qlo = H->cls_q0[cls], qhi = H->cls_q1[cls];
  const int64_t qpu = H->quads_per_unit;
  const int64_t U0 = H->cls_u0[cls], U1 = H->cls_u1[cls];
  const int64_t chunk = H->cls_chunk[cls];
  int held = -1;  // the query whose aggregates the block's shared-memory table holds
  for (;;) {
    __syncthreads();  // every thread has read the previous claim
    if (threadIdx.x == 0) s_claim = (int64_t)atomicAdd(next, (unsigned long long)chunk);
    __syncthreads();
    const int64_t ub = U0 + s_claim;
    if (ub >= U1) break;
    const int64_t ue = ub + chunk < U1 ? ub + chunk : U1;
    for (int64_t u = ub; u < ue; ++u) {  // block-uniform
      int lo = held >= 0 ? held : qlo, hi = qhi - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (Q[mid].u0[2] <= u) lo = mid;
        else hi = mid - 1;
      }
      const BatchQuery& b = Q[lo];
      if (kMode == kAggSmem && lo != held) {
        if (held >= 0) {
          __syncthreads();
          const ProbeArgs& h = Q[held].a;
          const SmemAggs Th = smem_aggs(smem_raw, h.gslots);
          for (uint32_t i = threadIdx.x; i < h.gslots; i += blockDim.x) smem_merge(Th, i, &h.tab[i], h.aggs);
          __syncthreads();
        }
        const SmemAggs Tn = smem_aggs(smem_raw, b.a.gslots);
        for (uint32_t i = threadIdx.x; i < b.a.gslots; i += blockDim.x) smem_identity(Tn, i);
        __syncthreads();
        held = lo;
      }
      if (b.d.dhdr->status != 0) continue;  // the build failed: nothing to aggregate
      const ProbeArgs a = b.a;
      const SmemAggs T = kMode == kAggSmem ? smem_aggs(smem_raw, a.gslots) : SmemAggs{};
      const Lookup L = read_lookup(a);
      const int64_t local = u - b.u0[2];
      const int64_t nq4 = a.n >> 2;
      const int64_t q0 = local * qpu;
      const int64_t q1 = q0 + qpu < nq4 ? q0 + qpu : nq4;
      int64_t q = q0 + threadIdx.x;
      if (kVec && !kWide && L.direct)  // two quads in flight per thread (registers: one block per SM)
        for (; q + blockDim.x < q1; q += 2 * (int64_t)blockDim.x) probe_quad_pair_direct<kMode>(a, T, L, q, q + blockDim.x);
      for (; q < q1; q += blockDim.x) probe_quad<kWide, kMode, kVec, false, true>(a, T, L, q);
      if (local == b.nu[2] - 1) {
        const int64_t t0 = nq4 << 2;
        if ((int64_t)threadIdx.x < a.n - t0) probe_one<kWide, kMode>(a, T, L, t0 + threadIdx.x);
      }
    }
  }
  if (kMode == kAggSmem && held >= 0) {
    __syncthreads();
    const ProbeArgs& h = Q[held].a;
    const SmemAggs Th = smem_aggs(smem_raw, h.gslots);
    for (uint32_t i = threadIdx.x; i < h.gslots; i += blockDim.x) smem_merge(Th, i, &h.tab[i], h.aggs);
  }
}

__global__ void __launch_bounds__(kBatchThreads)
batch_finalize_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q) {
  const int nq = H->nq;
  for (int64_t u = blockIdx.x; u < H->total[3]; u += gridDim.x) {
    const BatchQuery& b = Q[find_query<3>(Q, nq, u)];
    const int64_t s0 = (u - b.u0[3]) * kFinUnit;
    const int64_t s1 = s0 + kFinUnit < b.gslots ? s0 + kFinUnit : b.gslots;
    const Agg* tab = b.a.tab;
    const PipeOut out = b.out;
    for (int64_t base = s0; base < s1; base += blockDim.x) {
      const int64_t i = base + threadIdx.x;
      const bool occ = i < s1 && tab[i].count > 0;
      const uint64_t pos = warp_append(&b.phdr->groups, occ);
      if (occ && (int64_t)pos < out.cap) {
        const Agg t = tab[i];
        if (out.keys) out.keys[pos] = b.d.gkeys[i];
        if (out.sum) out.sum[pos] = (int64_t)t.sum;
        if (out.count) out.count[pos] = (int64_t)t.count;
        if (out.min) out.min[pos] = t.min;
        if (out.max) out.max[pos] = t.max;
      }
    }
  }
}

__global__ void batch_publish_kernel(const BatchHeader* __restrict__ H, const BatchQuery* __restrict__ Q,
                                     BatchStatus* __restrict__ st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H->nq) return;
  const BatchQuery& b = Q[q];
  int32_t s = b.d.dhdr->status;
  const unsigned long long g = b.phdr->groups;
  if (s == 0 && (int64_t)g > b.out.cap) s = SIRIUS_ERR_CAPACITY;
  b.phdr->status = s;
  if (b.out.d_groups) *b.out.d_groups = (int64_t)g;
  if (b.out.d_status) *b.out.d_status = s;
  st[b.orig].status = s;
  st[b.orig].groups = (int64_t)g;
}

DimLayout layout_of_index(const sirius_dim_index* idx) { return dim_layout_of_index(idx); }
// A batch builds its dims without a Bloom filter: its dims are small enough (a join table in L2)
// that a filter would not save DRAM reads.  Prebuilt dim indexes keep theirs.
DimLayout batch_dim_layout(const sirius_pipeline_desc* q) {
  return dim_layout(q->m, q->pk_hi != nullptr || q->fk_hi != nullptr, q->group_cap_hint, q->load_factor,
                    q->join_mode == 0, false);
}

bool prebuilt(const sirius_dim_index* indexes, int i) { return indexes && indexes[i].d_mem; }

}  // namespace
}  // namespace sirius

using namespace sirius;

struct sirius_batch_plan_s {
  int32_t max_q = 0;
  size_t table_bytes = 0;      // header + queries
  char* d_buf = nullptr;       // [BatchHeader | BatchQuery[max_q] | BatchStatus[max_q]]
  char* h_buf = nullptr;       // pinned staging, same layout
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t done = nullptr;  // recorded after each run: staging is free again
  cudaGraphExec_t exec = nullptr;
  size_t graph_smem = 0;
  uint32_t graph_classes = 0;  // probe classes launched by the captured graph
  int grid_small = 0;
  int grid_build = 0;          // build-phase kernels: one block per resident slot, no second wave
  int grid_probe[8] = {};
  size_t smem_for_grid = (size_t)-1;
};

typedef void (*probe_kernel_t)(const BatchHeader*, const BatchQuery*, int, unsigned long long*);

// class bits: 1 two-column keys, 2 shared-memory aggregation, 4 16-byte column loads
static probe_kernel_t probe_kernel_for(int c) {
  switch (c) {
    case 0: return batch_probe_kernel<false, kAggGlobal, false>;
    case 1: return batch_probe_kernel<true, kAggGlobal, false>;
    case 2: return batch_probe_kernel<false, kAggSmem, false>;
    case 3: return batch_probe_kernel<true, kAggSmem, false>;
    case 4: return batch_probe_kernel<false, kAggGlobal, true>;
    case 5: return batch_probe_kernel<true, kAggGlobal, true>;
    case 6: return batch_probe_kernel<false, kAggSmem, true>;
    default: return batch_probe_kernel<true, kAggSmem, true>;
  }
}

static BatchHeader* hdr_of(char* buf) { return (BatchHeader*)buf; }
static BatchQuery* queries_of(char* buf) { return (BatchQuery*)(buf + sizeof(BatchHeader)); }
static BatchStatus* status_of(sirius_batch_plan p, char* buf) {
  return (BatchStatus*)(buf + p->table_bytes);
}

extern "C" size_t sirius_pipeline_batch_scratch_bytes(const sirius_pipeline_desc* qs, int32_t nq,
                                                      const sirius_dim_index* indexes) {
  if (!qs || nq <= 0) return 0;
  size_t off = 0;
  for (int i = 0; i < nq; ++i) {
    const sirius_pipeline_desc* q = &qs[i];
    int64_t gcap;
    if (prebuilt(indexes, i)) {
      gcap = indexes[i].group_capacity;
    } else {
      const DimLayout L = batch_dim_layout(q);
      off += L.total;
      gcap = L.gcap;
    }
    off += run_layout(gcap, 0, kAggGlobal, false).total;
  }
  return off;
}

extern "C" sirius_status sirius_batch_plan_create(int32_t max_queries, sirius_batch_plan* out) {
  clear_error();
  SIRIUS_REQUIRE(out && max_queries > 0 && max_queries <= (1 << 20), "batch plan: bad max_queries");
  sirius_batch_plan p = new (std::nothrow) sirius_batch_plan_s();
  if (!p) return SIRIUS_ERR_OOM;
  p->max_q = max_queries;
  p->table_bytes = align_up(sizeof(BatchHeader) + sizeof(BatchQuery) * (size_t)max_queries, 256);
  const size_t bytes = p->table_bytes + sizeof(BatchStatus) * (size_t)max_queries;
  cudaError_t e = cudaMalloc(&p->d_buf, bytes);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->h_buf, bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("batch plan: allocation failed: %s", cudaGetErrorString(e));
    sirius_batch_plan_destroy(p);
    return SIRIUS_ERR_OOM;
  }
  memset(p->h_buf, 0, bytes);
  *out = p;
  return SIRIUS_OK;
}

extern "C" void sirius_batch_plan_destroy(sirius_batch_plan p) {
  if (!p) return;
  if (p->done) cudaEventSynchronize(p->done);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->done) cudaEventDestroy(p->done);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->d_buf) cudaFree(p->d_buf);
  if (p->h_buf) cudaFreeHost(p->h_buf);
  delete p;
}

// Enqueue the whole batch (copy in, five phases, copy out) on stream s.
static sirius_status enqueue_batch(sirius_batch_plan p, size_t smem, uint32_t classes, cudaStream_t s,
                                   bool timed) {
  const size_t copy_in = p->table_bytes;
  BatchHeader* dH = hdr_of(p->d_buf);
  BatchQuery* dQ = queries_of(p->d_buf);
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(p->d_buf, p->h_buf, copy_in, cudaMemcpyHostToDevice, s));
  {
    PhaseTimer pt(timed ? s : nullptr, timed ? SIRIUS_PHASE_BATCH_BUILD : -1);
    batch_init_kernel<<<p->grid_small, kBatchThreads, 0, s>>>(dH, dQ);
    SIRIUS_LAUNCH_CHECK();
    batch_minmax_kernel<<<p->grid_small, kBatchThreads, 0, s>>>(dH, dQ);
    SIRIUS_LAUNCH_CHECK();
    batch_clear_kernel<<<p->grid_small, kBatchThreads, 0, s>>>(dH, dQ, 0);
    SIRIUS_LAUNCH_CHECK();
    batch_build_kernel<false><<<p->grid_build, kBatchThreads, 0, s>>>(dH, dQ);
    SIRIUS_LAUNCH_CHECK();
    if (classes & kBuildWideBit) {
      batch_build_kernel<true><<<p->grid_build, kBatchThreads, 0, s>>>(dH, dQ);
      SIRIUS_LAUNCH_CHECK();
    }
    batch_clear_kernel<<<p->grid_small, kBatchThreads, 0, s>>>(dH, dQ, 1);
    SIRIUS_LAUNCH_CHECK();
    batch_fallback_kernel<<<p->grid_build, kBatchThreads, 0, s>>>(dH, dQ);
    SIRIUS_LAUNCH_CHECK();
  }
  {
    PhaseTimer pt(timed ? s : nullptr, timed ? SIRIUS_PHASE_BATCH_PROBE : -1);
    for (int c = 0; c < 8; ++c) {
      if (!((classes >> c) & 1u)) continue;
      probe_kernel_for(c)<<<p->grid_probe[c], kProbeThreads, (c & 2) ? smem : 0, s>>>(dH, dQ, c, &dH->cls_next[c]);
      SIRIUS_LAUNCH_CHECK();
    }
  }
  {
    PhaseTimer pt(timed ? s : nullptr, timed ? SIRIUS_PHASE_BATCH_FINALIZE : -1);
    batch_finalize_kernel<<<p->grid_small, kBatchThreads, 0, s>>>(dH, dQ);
    SIRIUS_LAUNCH_CHECK();
    batch_publish_kernel<<<(p->max_q + 255) / 256, 256, 0, s>>>(dH, dQ, status_of(p, p->d_buf));
    SIRIUS_LAUNCH_CHECK();
  }
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(status_of(p, p->h_buf), status_of(p, p->d_buf),
                                  sizeof(BatchStatus) * (size_t)p->max_q, cudaMemcpyDeviceToHost, s));
  return SIRIUS_OK;
}

extern "C" sirius_status sirius_batch_plan_run(sirius_batch_plan p, const sirius_pipeline_desc* qs, int32_t nq,
                                               const sirius_dim_index* indexes, sirius_result* results,
                                               int64_t rows_per_unit, int32_t use_graph, void* d_scratch,
                                               size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(p, "batch: NULL plan");
  SIRIUS_REQUIRE(qs && results && nq > 0 && nq <= p->max_q, "batch: nq=%d outside [1, %d]", nq, p->max_q);
  SIRIUS_REQUIRE(rows_per_unit >= 0, "batch: negative rows_per_unit");
  for (int i = 0; i < nq; ++i) {
    sirius_status st = validate_fact(&qs[i]);
    if (st == SIRIUS_OK && !prebuilt(indexes, i)) st = validate_dim(&qs[i]);
    if (st == SIRIUS_OK && qs[i].nsemi != 0) {
      set_error("batch: query %d: semi-join dims are taken by sirius_run_pipeline only", i);
      st = SIRIUS_ERR_INVALID;
    }
    if (st == SIRIUS_OK && !prebuilt(indexes, i) && qs[i].n > 0 && qs[i].m > 0 &&
        (qs[i].fk_hi == nullptr) != (qs[i].pk_hi == nullptr)) {
      set_error("batch: query %d mixes one- and two-column keys", i);
      st = SIRIUS_ERR_INVALID;
    }
    if (st == SIRIUS_OK && prebuilt(indexes, i) &&
        (indexes[i].key_width != (qs[i].fk_hi ? 8 : 4) || indexes[i].group_capacity <= 0)) {
      set_error("batch: query %d's dim index does not match its keys", i);
      st = SIRIUS_ERR_INVALID;
    }
    if (st == SIRIUS_OK && (results[i].out_cap < 0 || (results[i].out_cap > 0 && !results[i].keys && !results[i].count))) {
      set_error("batch: query %d has no output arrays", i);
      st = SIRIUS_ERR_INVALID;
    }
    if (st != SIRIUS_OK) return st;
  }
  const size_t need = sirius_pipeline_batch_scratch_bytes(qs, nq, indexes);
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, need, s);
  if (st != SIRIUS_OK) return st;

  // the staging table may still feed the previous run's copy: wait for it
  SIRIUS_CUDA_TRY(cudaEventSynchronize(p->done));
  const int64_t rpu = rows_per_unit > 0 ? rows_per_unit : 65536;
  const int64_t qpu = (rpu + 3) / 4;
  BatchHeader* H = hdr_of(p->h_buf);
  BatchQuery* Q = queries_of(p->h_buf);
  memset(H, 0, sizeof(BatchHeader));
  H->nq = nq;
  H->quads_per_unit = qpu;
  // probe class of every query, then the task table in class order (stable)
  std::vector<int> cls(nq), order(nq);
  for (int i = 0; i < nq; ++i) {
    const sirius_pipeline_desc* q = &qs[i];
    const bool pre = prebuilt(indexes, i);
    const int64_t gcap = pre ? indexes[i].group_capacity : batch_dim_layout(q).gcap;
    const bool wide = pre ? indexes[i].key_width == 8 : (q->pk_hi != nullptr || q->fk_hi != nullptr);
    const bool vec = ((uintptr_t)q->pred & 15) == 0 && ((uintptr_t)q->fk & 15) == 0 &&
                     (!q->fk_hi || ((uintptr_t)q->fk_hi & 15) == 0);
    // batches aggregate per probe unit in shared memory or with reductions (no partitioned mode)
    const int am = (q->agg_mode == kAggPart || q->agg_mode == kAggHot) ? kAggGlobal : q->agg_mode;
    cls[i] = (wide ? 1 : 0) | (choose_mode(am, gcap + 1, 0) == kAggSmem ? 2 : 0) | (vec ? 4 : 0);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cls[x] < cls[y]; });
  size_t off = 0;
  int64_t max_smem_slots = 0;
  uint32_t classes = 0;
  for (int c = 0; c < 8; ++c) H->cls_q0[c] = H->cls_q1[c] = 0;
  for (int k = 0; k < nq; ++k) {
    const int i = order[k];
    const sirius_pipeline_desc* q = &qs[i];
    BatchQuery& b = Q[k];
    memset(&b, 0, sizeof(b));
    b.orig = i;
    const bool pre = prebuilt(indexes, i);
    DimLayout L;
    char* dbase;
    if (pre) {
      L = layout_of_index(&indexes[i]);
      dbase = (char*)indexes[i].d_mem;
    } else {
      L = batch_dim_layout(q);
      dbase = sc.base + off;
      off += L.total;
    }
    const RunLayout R = run_layout(L.gcap, 0, kAggGlobal, false);
    char* rbase = sc.base + off;
    off += R.total;
    b.d = dim_view(L, dbase);
    const RunView r = run_view(R, rbase);
    b.phdr = r.phdr;
    b.out = PipeOut{results[i].keys, results[i].sum, results[i].count, results[i].min, results[i].max,
                    results[i].out_cap, results[i].d_groups, results[i].d_status};
    b.a.fk = q->fk;
    b.a.fk_hi = q->fk_hi;
    b.a.pred = q->pred;
    b.a.val = q->val;
    b.a.n = q->n;
    b.a.op = q->op;
    b.a.lit = q->literal;
    b.a.aggs = q->aggs;
    b.a.jcap = b.d.jcap;
    b.a.jslots = b.d.jslots;
    b.a.jhdr = b.d.jhdr;
    b.a.dhdr = b.d.dhdr;
    b.a.dslot = b.d.dslot;
    b.a.bloom = b.d.bloom;
    b.a.bloom_mask = b.d.bloom_mask;
    b.a.tab = r.aggs;
    b.a.gslots = (uint32_t)R.gslots;
    b.pk = q->pk;
    b.pk_hi = q->pk_hi;
    b.grp = q->grp;
    b.flag = q->flag;
    b.dpred = DimPred{pre ? nullptr : q->dpred, q->dop, q->dliteral};
    b.m = pre ? 0 : q->m;
    b.gslots = R.gslots;
    b.jpairs = pre ? 0 : (L.jcap * (L.key_width == 8 ? 16 : 8) + 15) / 16;
    b.dpairs = pre ? 0 : L.dcap / 4;
    b.glimit = group_limit_for(L.gcap);
    const int c = cls[i];
    b.flags = ((c & 1) ? kQWide : 0) | ((c & 2) ? kQSmem : 0) | ((c & 4) ? kQVec : 0) | (pre ? 0 : kQBuild);
    if ((c & 2) && R.gslots > max_smem_slots) max_smem_slots = R.gslots;
    const bool probes = q->n > 0 && (pre || q->m > 0);
    const int64_t init_words = (!pre && L.dcap == 0 ? b.jpairs : 0) + b.gslots;
    b.nu[0] = (init_words + kInitUnit - 1) / kInitUnit;
    b.nu[1] = (b.m + kBuildUnit - 1) / kBuildUnit;
    const int64_t nq4 = q->n >> 2;
    b.nu[2] = probes ? ((nq4 + qpu - 1) / qpu > 0 ? (nq4 + qpu - 1) / qpu : 1) : 0;
    b.nu[3] = (b.gslots + kFinUnit - 1) / kFinUnit;
    const int64_t clear_words = (!pre && L.dcap > 0 && b.m > 0) ? (b.jpairs > b.dpairs ? b.jpairs : b.dpairs) : 0;
    b.nu[4] = (clear_words + kInitUnit - 1) / kInitUnit;
    for (int ph = 0; ph < 5; ++ph) {
      b.u0[ph] = H->total[ph];
      H->total[ph] += b.nu[ph];
    }
    if (k == 0 || cls[order[k - 1]] != c) {
      H->cls_q0[c] = k;
      H->cls_u0[c] = b.u0[2];
    }
    H->cls_q1[c] = k + 1;
    H->cls_u1[c] = H->total[2];
    if (b.nu[2] > 0) classes |= 1u << c;
    if ((c & 1) && b.nu[1] > 0) classes |= kBuildWideBit;
  }
  const size_t smem = smem_aggs_bytes((uint32_t)max_smem_slots, false);
  if (p->smem_for_grid != smem) {
    for (int c = 0; c < 8; ++c) {
      const size_t sm = (c & 2) ? smem : 0;
      if (sm > 48 * 1024)
        SIRIUS_CUDA_TRY(cudaFuncSetAttribute(probe_kernel_for(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemAggMaxBytes));
      int per = 0;
      SIRIUS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, probe_kernel_for(c), kProbeThreads, sm));
      p->grid_probe[c] = sm_count() * (per > 0 ? per : 1);
    }
    p->grid_small = sm_count() * 8;
    int per_build = 0;
    SIRIUS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_build, batch_build_kernel<false>, kBatchThreads, 0));
    p->grid_build = sm_count() * (per_build > 0 ? per_build : 1);
    p->smem_for_grid = smem;
  }
  // Claim size per class.  At least 32 units per block (large batches): 32 claims per block,
  // for a short tail.  Fewer (smaller batches, e.g. served requests): one contiguous chunk per
  // block, as a static split gives -- there a claim's round trip and the merge at every change
  // of query cost more than the imbalance they would remove (measured: a served batch of 64
  // queries, 17 units per block, lost a fifth of its peak rate with one-unit claims).
  for (int c = 0; c < 8; ++c) {
    const int64_t units = H->cls_u1[c] - H->cls_u0[c];
    const int64_t grid = p->grid_probe[c] > 0 ? p->grid_probe[c] : 1;
    const int64_t per_block = units / grid;
    const int64_t chunk = per_block >= 32 ? per_block / 32 : (units + grid - 1) / grid;
    H->cls_chunk[c] = chunk > 1 ? chunk : 1;
  }

  if (use_graph) {
    if (!p->exec || p->graph_smem != smem || p->graph_classes != classes) {
      if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      SIRIUS_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
      set_launch_counting(false);
      sirius_status est = enqueue_batch(p, smem, classes, p->cap_stream, false);
      set_launch_counting(true);
      cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
      if (est != SIRIUS_OK) {
        if (g) cudaGraphDestroy(g);
        return est;
      }
      if (ce != cudaSuccess) {
        set_error("batch: graph capture failed: %s", cudaGetErrorString(ce));
        return SIRIUS_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&p->exec, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        p->exec = nullptr;
        set_error("batch: graph instantiation failed: %s", cudaGetErrorString(ce));
        return SIRIUS_ERR_CUDA;
      }
      p->graph_smem = smem;
      p->graph_classes = classes;
    }
    PhaseTimer pt(s, SIRIUS_PHASE_BATCH_GRAPH);
    SIRIUS_CUDA_TRY(cudaGraphLaunch(p->exec, s));
    count_launch(8 + __builtin_popcount(classes));
  } else {
    st = enqueue_batch(p, smem, classes, s, true);
    if (st != SIRIUS_OK) return st;
  }
  SIRIUS_CUDA_TRY(cudaEventRecord(p->done, s));
  if (!results[0].sync) return SIRIUS_OK;
  SIRIUS_CUDA_TRY(cudaEventSynchronize(p->done));
  const BatchStatus* hs = status_of(p, p->h_buf);
  sirius_status first = SIRIUS_OK;
  for (int i = 0; i < nq; ++i) {
    results[i].groups = hs[i].groups;
    results[i].status = (int32_t)hs[i].status;
    if (first == SIRIUS_OK && hs[i].status != 0) {
      first = (sirius_status)hs[i].status;
      set_error("batch: query %d finished with status %d", i, (int)hs[i].status);
    }
  }
  return first;
}

extern "C" sirius_status sirius_run_pipeline_batch(const sirius_pipeline_desc* qs, int32_t nq,
                                                   const sirius_dim_index* indexes, sirius_result* results,
                                                   void* d_scratch, size_t scratch_bytes, sirius_stream stream) {
  sirius_batch_plan p = nullptr;
  sirius_status st = sirius_batch_plan_create(nq > 0 ? nq : 1, &p);
  if (st != SIRIUS_OK) return st;
  st = sirius_batch_plan_run(p, qs, nq, indexes, results, 0, 0, d_scratch, scratch_bytes, stream);
  sirius_batch_plan_destroy(p);  // waits for the batch: the plan's task table feeds its kernels
  return st;
}
