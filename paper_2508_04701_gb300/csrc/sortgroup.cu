// Sort-based group-by (the alternative to hashing that Sec. 4.2 weighs group-by operators
// against): the (key, value) pairs are sorted by key with a least-significant-digit radix sort,
// then each run of equal keys is reduced to its SUM / COUNT / MIN / MAX.  Groups come out in
// ascending key order.
//
// Radix sort: keys mapped to unsigned words that order like the signed keys (sign bit
// flipped); 8-bit digits, least significant first; a pass whose digit is the same in every key
// leaves the order unchanged and is skipped (decided on the device from the OR of key ^ key[0]).
// A pass: per-tile digit histograms (digit-major), their exclusive scan, and a stable scatter:
// each block takes its tile in rounds of 256 keys (one per thread, in order), ranks a key among
// the round's keys with the same digit by warp match_any plus the counts of the warps before,
// and adds the counts of the earlier rounds and tiles.
// Reduction: segment heads (key differs from the one before) counted per tile and scanned give
// every element its group index; a thread reduces its 8 consecutive elements run by run, stores
// runs that start and end within it, and combines the runs that cross thread boundaries within
// the warp before one set of atomics per run.
#include "tables.cuh"

namespace sirius {
namespace {

constexpr int kSgThreads = 256;
constexpr int kSgItems = 8;                        // keys per thread and tile
constexpr int kSgTile = kSgThreads * kSgItems;     // 2048
constexpr int kSgScanThreads = 1024;
constexpr int kSgScanSeg = 4096;                   // entries per block of the multi-block scan

struct SgHeader {
  unsigned long long diff;    // OR over keys of (key ^ key[0]): the bits that vary
  int32_t cur;                // buffer holding the current order (0 or 1)
  int32_t pad0;
  unsigned long long groups;  // G
  unsigned long long pad[29];
};
static_assert(sizeof(SgHeader) == 256, "sort group-by header is 256 bytes");

__device__ __forceinline__ uint64_t map_key(const void* keys, int width, int64_t i) {
  if (width == 4) return (uint64_t)((uint32_t)reinterpret_cast<const int32_t*>(keys)[i] ^ 0x80000000u);
  return (uint64_t)reinterpret_cast<const int64_t*>(keys)[i] ^ 0x8000000000000000ull;
}
__device__ __forceinline__ int64_t unmap_key(uint64_t u, int width) {
  if (width == 4) return (int64_t)(int32_t)((uint32_t)u ^ 0x80000000u);
  return (int64_t)(u ^ 0x8000000000000000ull);
}

__global__ void sg_load_kernel(const void* keys, int width, const int64_t* vals, int64_t n, uint64_t* k0,
                               int64_t* v0, SgHeader* h) {
  const uint64_t first = map_key(keys, width, 0);
  unsigned long long acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = map_key(keys, width, i);
    k0[i] = k;
    v0[i] = vals[i];
    acc |= k ^ first;
  }
  for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicOr(&h->diff, acc);
}

__device__ __forceinline__ bool pass_skipped(const SgHeader* h, int pass) {
  return ((h->diff >> (8 * pass)) & 0xFFull) == 0;
}

// counts[d * ntiles + t]: keys of tile t with digit d.
__global__ void __launch_bounds__(kSgThreads)
sg_hist_kernel(const uint64_t* k0, const uint64_t* k1, int64_t n, int64_t ntiles, const SgHeader* h, int pass,
               uint32_t* counts) {
  if (pass_skipped(h, pass)) return;  // block-uniform
  __shared__ uint32_t c[256];
  c[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t* src = h->cur ? k1 : k0;
  const int64_t t = blockIdx.x;
  for (int r = 0; r < kSgItems; ++r) {
    const int64_t i = t * kSgTile + r * kSgThreads + threadIdx.x;
    if (i < n) atomicAdd(&c[(src[i] >> (8 * pass)) & 0xFF], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + t] = c[threadIdx.x];
}

// Multi-block exclusive scan of m 32-bit counts in place (three launches): partial sums per
// segment, their scan in one block, then each segment scanned with its base added.
__global__ void __launch_bounds__(kSgScanThreads)
sg_scan_partials_kernel(const uint32_t* a, int64_t m, const SgHeader* h, int pass, unsigned long long* part) {
  if (pass >= 0 && pass_skipped(h, pass)) return;
  __shared__ unsigned long long s[kSgScanThreads / 32];
  unsigned long long acc = 0;
  const int64_t base = (int64_t)blockIdx.x * kSgScanSeg;
  for (int64_t i = base + threadIdx.x; i < base + kSgScanSeg && i < m; i += blockDim.x) acc += a[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kSgScanThreads / 32; ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kSgScanThreads)
sg_scan_top_kernel(unsigned long long* part, int64_t nb, const SgHeader* h, int pass, unsigned long long* total) {
  if (pass >= 0 && pass_skipped(h, pass)) return;
  __shared__ unsigned long long s[kSgScanThreads];
  unsigned long long carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kSgScanThreads) {
    const int64_t i = b0 + threadIdx.x;
    const unsigned long long v = i < nb ? part[i] : 0ull;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kSgScanThreads; o <<= 1) {
      const unsigned long long x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
      __syncthreads();
      s[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) part[i] = carry + s[threadIdx.x] - v;  // exclusive
    const unsigned long long blk = s[kSgScanThreads - 1];
    __syncthreads();
    carry += blk;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kSgScanThreads)
sg_scan_apply_kernel(uint32_t* a, int64_t m, const unsigned long long* part, const SgHeader* h, int pass,
                     unsigned long long* out64) {
  if (pass >= 0 && pass_skipped(h, pass)) return;
  // segment of kSgScanSeg entries: 4 per thread, thread-local sums, block scan of those
  __shared__ unsigned long long s[kSgScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kSgScanSeg + (int64_t)threadIdx.x * 4;
  uint32_t v[4];
  unsigned long long loc = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < m ? a[base + j] : 0u;
    loc += v[j];
  }
  s[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < kSgScanThreads; o <<= 1) {
    const unsigned long long x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  unsigned long long run = part[blockIdx.x] + s[threadIdx.x] - loc;
  for (int j = 0; j < 4; ++j) {
    if (base + j < m) {
      if (out64) out64[base + j] = run;
      else a[base + j] = (uint32_t)run;
    }
    run += v[j];
  }
}

// Stable scatter of one pass: src buffer cur -> the other one.
__global__ void __launch_bounds__(kSgThreads)
sg_scatter_kernel(uint64_t* k0, uint64_t* k1, int64_t* v0, int64_t* v1, int64_t n, int64_t ntiles,
                  const SgHeader* h, int pass, const uint32_t* offs) {
  if (pass_skipped(h, pass)) return;  // block-uniform
  __shared__ uint32_t base[256];      // next free position of each digit for this tile
  __shared__ uint32_t wcnt[kSgThreads / 32][256];
  const int cur = h->cur;
  const uint64_t* ks = cur ? k1 : k0;
  const int64_t* vs = cur ? v1 : v0;
  uint64_t* kd = cur ? k0 : k1;
  int64_t* vd = cur ? v0 : v1;
  const int64_t t = blockIdx.x;
  base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + t];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSgItems; ++r) {
    for (int w = 0; w < kSgThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = t * kSgTile + r * kSgThreads + threadIdx.x;
    const bool has = i < n;
    uint64_t k = 0;
    int64_t v = 0;
    uint32_t d = 256;  // no key: a digit no real key has
    if (has) {
      k = ks[i];
      v = vs[i];
      d = (uint32_t)(k >> (8 * pass)) & 0xFFu;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank_w = __popc(peers & lt);
    if (has && rank_w == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t before = 0;  // keys of this digit in the earlier warps of the round
    if (has)
      for (int w = 0; w < warp; ++w) before += wcnt[w][d];
    if (has) {
      const uint32_t pos = base[d] + before + rank_w;
      kd[pos] = k;
      vd[pos] = v;
    }
    __syncthreads();
    // advance each digit's base by the round's count
    uint32_t tot = 0;
    for (int w = 0; w < kSgThreads / 32; ++w) tot += wcnt[w][threadIdx.x];
    base[threadIdx.x] += tot;
    __syncthreads();
  }
}

__global__ void sg_flip_kernel(SgHeader* h, int pass) {
  if (!pass_skipped(h, pass)) h->cur ^= 1;
}

// ------------------------------------------------------------------ reduction of the runs
// th[t]: segment heads (a key differing from the one before it) among tile t's elements.
__global__ void __launch_bounds__(kSgThreads)
sg_heads_kernel(const uint64_t* k0, const uint64_t* k1, int64_t n, const SgHeader* h, uint32_t* th) {
  __shared__ uint32_t s[kSgThreads / 32];
  const uint64_t* ks = h->cur ? k1 : k0;
  const int64_t t = blockIdx.x;
  uint32_t c = 0;
  for (int j = 0; j < kSgItems; ++j) {
    const int64_t i = t * kSgTile + (int64_t)threadIdx.x * kSgItems + j;
    if (i < n && (i == 0 || ks[i] != ks[i - 1])) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kSgThreads / 32; ++w) tot += s[w];
    th[t] = tot;
  }
}

struct SgOut {
  int64_t* keys;
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t cap;
};

// Identity aggregates for the groups that will be written (the ones below out_cap).
__global__ void sg_init_out_kernel(SgOut o, const SgHeader* h) {
  const int64_t g = (int64_t)h->groups < o.cap ? (int64_t)h->groups : o.cap;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
    if (o.sum) o.sum[i] = 0;
    if (o.count) o.count[i] = 0;
    if (o.min) o.min[i] = INT64_MAX;
    if (o.max) o.max[i] = INT64_MIN;
  }
}

struct SgPart {
  long long sum, cnt, mn, mx;
  int64_t g;  // -1: none
  uint64_t key;
};

__device__ __forceinline__ void sg_store(const SgOut& o, int64_t g, uint64_t key, int width, const SgPart& p) {
  if (g >= o.cap) return;
  if (o.keys) o.keys[g] = unmap_key(key, width);
  if (o.sum) o.sum[g] = p.sum;
  if (o.count) o.count[g] = p.cnt;
  if (o.min) o.min[g] = p.mn;
  if (o.max) o.max[g] = p.mx;
}

__device__ __forceinline__ void sg_merge(const SgOut& o, int64_t g, uint64_t key, int width, const SgPart& p) {
  if (g >= o.cap) return;
  if (o.keys) o.keys[g] = unmap_key(key, width);  // every contributor stores the same key
  if (o.sum) atomicAdd(reinterpret_cast<unsigned long long*>(&o.sum[g]), (unsigned long long)p.sum);
  if (o.count) atomicAdd(reinterpret_cast<unsigned long long*>(&o.count[g]), (unsigned long long)p.cnt);
  if (o.min) atomicMin(reinterpret_cast<long long*>(&o.min[g]), p.mn);
  if (o.max) atomicMax(reinterpret_cast<long long*>(&o.max[g]), p.mx);
}

// Warp-level combine of the runs that cross thread boundaries (lanes holding the same group
// are contiguous), then one set of atomics per group by its lowest lane.
__device__ __forceinline__ void sg_merge_warp(const SgOut& o, int width, SgPart p, SgPart* stage) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)p.g);
  stage[lane] = p;
  __syncwarp();
  if (p.g >= 0 && (peers & ((1u << lane) - 1u)) == 0) {
    SgPart acc = p;
    for (unsigned m = peers & ~(1u << lane); m; m &= m - 1) {
      const SgPart& q = stage[__ffs(m) - 1];
      acc.sum += q.sum;
      acc.cnt += q.cnt;
      acc.mn = q.mn < acc.mn ? q.mn : acc.mn;
      acc.mx = q.mx > acc.mx ? q.mx : acc.mx;
    }
    sg_merge(o, acc.g, acc.key, width, acc);
  }
  __syncwarp();
}

// Each thread reduces its kSgItems consecutive elements (th: the tiles' exclusive group bases).
__global__ void __launch_bounds__(kSgThreads)
sg_reduce_kernel(const uint64_t* k0, const uint64_t* k1, const int64_t* v0, const int64_t* v1, int64_t n,
                 int width, const SgHeader* h, const uint32_t* th, SgOut o) {
  __shared__ uint32_t scan[kSgThreads];
  __shared__ SgPart stage[kSgThreads];
  const int cur = h->cur;
  const uint64_t* ks = cur ? k1 : k0;
  const int64_t* vs = cur ? v1 : v0;
  const int64_t t = blockIdx.x;
  const int64_t e0 = t * kSgTile + (int64_t)threadIdx.x * kSgItems;
  uint32_t heads = 0;
  for (int j = 0; j < kSgItems; ++j) {
    const int64_t i = e0 + j;
    if (i < n && (i == 0 || ks[i] != ks[i - 1])) ++heads;
  }
  // exclusive scan of the threads' head counts within the tile
  scan[threadIdx.x] = heads;
  __syncthreads();
  for (int off = 1; off < kSgThreads; off <<= 1) {
    const uint32_t x = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0u;
    __syncthreads();
    scan[threadIdx.x] += x;
    __syncthreads();
  }
  // group of the element before the thread's first one: th[t] + heads before this thread - 1
  int64_t g = (int64_t)th[t] + (int64_t)(scan[threadIdx.x] - heads) - 1;
  SgPart first{0, 0, INT64_MAX, INT64_MIN, -1, 0}, last{0, 0, INT64_MAX, INT64_MIN, -1, 0};
  SgPart run{0, 0, INT64_MAX, INT64_MIN, -1, 0};
  bool run_from_head = false;  // the current run began at a head inside this thread
  bool first_done = false;
  int64_t i_end = e0 + kSgItems < n ? e0 + kSgItems : n;
  for (int64_t i = e0; i < i_end; ++i) {
    const uint64_t k = ks[i];
    const bool head = i == 0 || k != ks[i - 1];
    if (head) {
      if (run.g >= 0) {
        // the run ended before this head inside the thread
        if (run_from_head) sg_store(o, run.g, run.key, width, run);
        else { first = run; first_done = true; }
      }
      ++g;
      run = SgPart{0, 0, INT64_MAX, INT64_MIN, g, k};
      run_from_head = true;
    } else if (run.g < 0) {
      run = SgPart{0, 0, INT64_MAX, INT64_MIN, g, k};  // continues a run from the thread before
      run_from_head = false;
    }
    const long long v = vs[i];
    run.sum += v;
    run.cnt += 1;
    run.mn = v < run.mn ? v : run.mn;
    run.mx = v > run.mx ? v : run.mx;
  }
  if (run.g >= 0) {
    // the last run is complete if it began at a head here and the next element starts a new key
    const bool next_head = i_end >= n || ks[i_end] != ks[i_end - 1];
    if (run_from_head && next_head) sg_store(o, run.g, run.key, width, run);
    else if (!run_from_head && !first_done) first = run;  // one run spanning the whole thread
    else last = run;
  }
  (void)first_done;
  SgPart* st = stage + (threadIdx.x & ~31);
  sg_merge_warp(o, width, first, st);
  sg_merge_warp(o, width, last, st);
}

size_t sg_layout(int64_t n, size_t* off_k1, size_t* off_v0, size_t* off_v1, size_t* off_cnt, size_t* off_part) {
  const int64_t nn = n > 0 ? n : 1;
  const int64_t ntiles = (nn + kSgTile - 1) / kSgTile;
  const int64_t m = 256 * ntiles;
  const int64_t nb = (m + kSgScanSeg - 1) / kSgScanSeg;
  size_t off = 256;  // header
  const size_t k0 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  *off_k1 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  *off_v0 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  *off_v1 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  *off_cnt = off;
  off = align_up(off + (size_t)m * 4, 256);
  *off_part = off;
  off = align_up(off + (size_t)nb * 8, 256);
  (void)k0;
  return off;
}

sirius_status sg_scan(uint32_t* a, int64_t m, unsigned long long* part, const SgHeader* h, int pass,
                      unsigned long long* total, cudaStream_t s) {
  const int64_t nb = (m + kSgScanSeg - 1) / kSgScanSeg;
  sg_scan_partials_kernel<<<(unsigned)nb, kSgScanThreads, 0, s>>>(a, m, h, pass, part);
  SIRIUS_LAUNCH_CHECK();
  sg_scan_top_kernel<<<1, kSgScanThreads, 0, s>>>(part, nb, h, pass, total);
  SIRIUS_LAUNCH_CHECK();
  sg_scan_apply_kernel<<<(unsigned)nb, kSgScanThreads, 0, s>>>(a, m, part, h, pass, nullptr);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

__global__ void sg_copy_groups_kernel(const SgHeader* h, int64_t* d_groups) { *d_groups = (int64_t)h->groups; }

}  // namespace
}  // namespace sirius

using namespace sirius;

extern "C" size_t sirius_groupby_sort_scratch_bytes(int64_t n) {
  size_t a, b, c, d, e;
  return sg_layout(n, &a, &b, &c, &d, &e);
}

extern "C" sirius_status sirius_groupby_sort(const void* d_keys, int32_t key_width, const int64_t* d_vals,
                                             int64_t n, uint32_t aggs, int64_t* d_out_keys, int64_t* d_sum,
                                             int64_t* d_count, int64_t* d_min, int64_t* d_max, int64_t out_cap,
                                             int64_t* d_groups, int64_t* h_groups, void* d_scratch,
                                             size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(key_width == 4 || key_width == 8, "groupby_sort: key_width must be 4 or 8");
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "groupby_sort: n out of range");
  SIRIUS_REQUIRE(n == 0 || (d_keys && d_vals), "groupby_sort: NULL input");
  SIRIUS_REQUIRE(out_cap >= 0, "groupby_sort: negative out_cap");
  SIRIUS_REQUIRE(aggs <= SIRIUS_AGG_ALL, "groupby_sort: bad aggregate mask");
  size_t off_k1, off_v0, off_v1, off_cnt, off_part;
  const size_t need = sg_layout(n, &off_k1, &off_v0, &off_v1, &off_cnt, &off_part);
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, need, s);
  if (st != SIRIUS_OK) return st;
  SgHeader* hdr = (SgHeader*)sc.base;
  uint64_t* k0 = (uint64_t*)(sc.base + 256);
  uint64_t* k1 = (uint64_t*)(sc.base + off_k1);
  int64_t* v0 = (int64_t*)(sc.base + off_v0);
  int64_t* v1 = (int64_t*)(sc.base + off_v1);
  uint32_t* cnt = (uint32_t*)(sc.base + off_cnt);
  unsigned long long* part = (unsigned long long*)(sc.base + off_part);
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256, s));
  const SgOut o{d_out_keys, (aggs & SIRIUS_AGG_SUM) ? d_sum : nullptr, d_count,
                (aggs & SIRIUS_AGG_MIN) ? d_min : nullptr, (aggs & SIRIUS_AGG_MAX) ? d_max : nullptr, out_cap};
  PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
  if (n > 0) {
    const int64_t ntiles = (n + kSgTile - 1) / kSgTile;
    sg_load_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_keys, key_width, d_vals, n, k0, v0, hdr);
    SIRIUS_LAUNCH_CHECK();
    const int passes = key_width == 4 ? 4 : 8;
    for (int pass = 0; pass < passes; ++pass) {
      sg_hist_kernel<<<(unsigned)ntiles, kSgThreads, 0, s>>>(k0, k1, n, ntiles, hdr, pass, cnt);
      SIRIUS_LAUNCH_CHECK();
      if ((st = sg_scan(cnt, 256 * ntiles, part, hdr, pass, nullptr, s)) != SIRIUS_OK) return st;
      sg_scatter_kernel<<<(unsigned)ntiles, kSgThreads, 0, s>>>(k0, k1, v0, v1, n, ntiles, hdr, pass, cnt);
      SIRIUS_LAUNCH_CHECK();
      sg_flip_kernel<<<1, 1, 0, s>>>(hdr, pass);
      SIRIUS_LAUNCH_CHECK();
    }
    sg_heads_kernel<<<(unsigned)ntiles, kSgThreads, 0, s>>>(k0, k1, n, hdr, cnt);
    SIRIUS_LAUNCH_CHECK();
    if ((st = sg_scan(cnt, ntiles, part, hdr, -1, &hdr->groups, s)) != SIRIUS_OK) return st;
    sg_init_out_kernel<<<grid_for(out_cap > 0 ? out_cap : 1, 256), 256, 0, s>>>(o, hdr);
    SIRIUS_LAUNCH_CHECK();
    sg_reduce_kernel<<<(unsigned)ntiles, kSgThreads, 0, s>>>(k0, k1, v0, v1, n, key_width, hdr, cnt, o);
    SIRIUS_LAUNCH_CHECK();
  }
  if (d_groups) {
    sg_copy_groups_kernel<<<1, 1, 0, s>>>(hdr, d_groups);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_groups) {
    SgHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_groups = (int64_t)h.groups;
    if ((int64_t)h.groups > out_cap) {
      set_error("groupby_sort: %lld groups exceed out_cap %lld", (long long)h.groups, (long long)out_cap);
      return SIRIUS_ERR_CAPACITY;
    }
  }
  return SIRIUS_OK;
}
