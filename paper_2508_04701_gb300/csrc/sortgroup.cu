// Sort-based group-by (the alternative to hashing that Sec. 4.2 weighs group-by operators
// against): the (key, value) pairs are sorted by key with a least-significant-digit radix sort,
// then each run of equal keys is reduced to its SUM / COUNT / MIN / MAX.  Groups come out in
// ascending key order.
//
// Radix sort: keys as unsigned words of their own width (32 bits for int32 keys) that order like
// the signed keys (sign bit flipped); 8-bit digits, least significant first; a pass whose digit
// is the same in every key leaves the order unchanged and is skipped (decided on the device
// from the OR of key ^ key[0], formed while the first histogram is taken).  The first pass that
// runs reads the caller's columns directly; later ones ping-pong between two buffers.
// The digit counts of every pass are taken in one read of the keys up front.  A pass is one
// sweep over tiles of 4096 keys: the scatter ranks the tile's keys stably (each warp ranks its
// 512 consecutive keys with ballots and warp-private digit counters), finds each digit's output
// offset from the digit's base and a decoupled look-back over the earlier tiles' counts, places
// the keys in shared memory in digit order and writes each digit's run out contiguously, every
// key with its value (the tile's values arrive by a bulk copy).
// Reduction: segment heads (key differs from the one before) counted per tile and scanned give
// every element its group index; a thread reduces its 16 consecutive elements (staged in shared
// memory) run by run, stores runs that start and end within it, and combines the runs that
// cross thread boundaries within the warp before one set of atomics per run.
#include "scan.cuh"

namespace sirius {
namespace {

constexpr int kSgThreads = 256;
constexpr int kSgWarps = kSgThreads / 32;
constexpr int kSgItems = 16;                       // keys per thread and tile
constexpr int kSgTile = kSgThreads * kSgItems;     // 4096
constexpr int kSgWarpSpan = kSgTile / kSgWarps;    // 512 consecutive keys ranked by one warp

struct SgHeader {
  unsigned long long diff;       // OR over keys of (key ^ key[0]): the bits that vary
  int32_t src;                   // where the current order lives: 0 the input, 1 / 2 buffer 0 / 1
  int32_t status;                // SIRIUS_OK, or SIRIUS_ERR_TIMEOUT when a bounded wait ran out
  unsigned long long groups;     // G
  unsigned long long ticket[8];  // per pass: tiles handed out so far
  unsigned long long pad[21];
};
static_assert(sizeof(SgHeader) == 256, "sort group-by header is 256 bytes");

template <typename K>
struct SgBufs {
  const K* in_k;         // the caller's keys read as unsigned words (sign bit not flipped)
  const int64_t* in_v;
  K* k0;
  K* k1;
  int64_t* v0;
  int64_t* v1;
  int in_v_aligned;      // the caller's values start on a 16-byte boundary (bulk copies allowed)
};

template <typename K>
struct SgSrc {
  const K* k;
  const int64_t* v;
  K flip;  // XOR that maps a stored word to its ordered form
};

template <typename K>
__device__ __forceinline__ SgSrc<K> sg_src(const SgBufs<K>& b, int src) {
  if (src == 0) return SgSrc<K>{b.in_k, b.in_v, (K)((K)1 << (8 * sizeof(K) - 1))};
  if (src == 1) return SgSrc<K>{b.k0, b.v0, (K)0};
  return SgSrc<K>{b.k1, b.v1, (K)0};
}

template <typename K>
__device__ __forceinline__ uint32_t sg_digit(K k, int pass) {
  return (uint32_t)(k >> (8 * pass)) & 0xFFu;
}

template <typename K>
__device__ __forceinline__ int64_t unmap_key(K u) {
  if (sizeof(K) == 4) return (int64_t)(int32_t)((uint32_t)u ^ 0x80000000u);
  return (int64_t)((unsigned long long)u ^ 0x8000000000000000ull);
}

// Lanes of the warp whose valid key has the same 8-bit digit as this lane's: the digit's bits
// compared by eight ballots (a fixed cost, whatever the number of distinct digits in the warp).
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool valid) {
  unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned v = __ballot_sync(0xffffffffu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

__device__ __forceinline__ bool pass_skipped(const SgHeader* h, int pass) {
  return ((h->diff >> (8 * pass)) & 0xFFull) == 0;
}

// Global digit counts of every pass in one read of the keys (gcount[pass * 256 + digit]), and
// the bits that vary.  A warp whose keys share a digit adds once; otherwise each lane adds to
// one of kSgCopies copies of the histogram (by lane), so that a digit with few values does not
// serialise the adds.
template <typename K>
__host__ __device__ constexpr int sg_copies() { return sizeof(K) == 4 ? 8 : 4; }

template <typename K>
__global__ void __launch_bounds__(kSgThreads)
sg_upfront_kernel(const K* __restrict__ in, int64_t n, SgHeader* h, unsigned long long* gcount) {
  constexpr int kP = (int)sizeof(K);
  constexpr int kC = sg_copies<K>();
  constexpr int kU = 8;  // keys per thread and step, loaded together
  extern __shared__ __align__(16) unsigned char sg_smem[];
  uint32_t* hs = reinterpret_cast<uint32_t*>(sg_smem);  // [pass][copy][digit]
  for (int i = threadIdx.x; i < kP * kC * 256; i += kSgThreads) hs[i] = 0;
  __syncthreads();
  const K sign = (K)((K)1 << (8 * sizeof(K) - 1));
  const K first = in[0] ^ sign;
  const int lane = threadIdx.x & 31;
  const int copy = lane & (kC - 1);
  K acc = 0;
  for (int64_t base = (int64_t)blockIdx.x * kSgThreads * kU; base < n; base += (int64_t)gridDim.x * kSgThreads * kU) {
    K k[kU];
    bool v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = base + u * kSgThreads + threadIdx.x;
      v[u] = i < n;
      k[u] = v[u] ? (K)(in[i] ^ sign) : first;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      acc |= k[u] ^ first;
      // the bytes in which the warp's keys differ from lane 0's
      K x = k[u] ^ __shfl_sync(0xffffffffu, k[u], 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
      const unsigned vm = __ballot_sync(0xffffffffu, v[u]);
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        uint32_t* hp = hs + (p * kC + copy) * 256;
        if (sg_digit(x, p) == 0) {  // warp-uniform: one digit for the whole warp
          if (lane == 0 && vm) atomicAdd(&hp[sg_digit(k[u], p)], (uint32_t)__popc(vm));
        } else if (v[u]) {
          atomicAdd(&hp[sg_digit(k[u], p)], 1u);
        }
      }
    }
  }
  unsigned long long a = (unsigned long long)acc;
  for (int o = 16; o > 0; o >>= 1) a |= __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0 && a) atomicOr(&h->diff, a);
  __syncthreads();
  for (int p = 0; p < kP; ++p) {
    uint32_t c = 0;
    for (int q = 0; q < kC; ++q) c += hs[(p * kC + q) * 256 + threadIdx.x];
    if (c) atomicAdd(&gcount[p * 256 + threadIdx.x], (unsigned long long)c);
  }
}

// Exclusive scan of one value per thread over a block of kSgThreads (warp shuffles, then the
// warp totals).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  return before + inc - x;
}

// One block: each pass's digit counts -> exclusive digit bases, in place.
__global__ void __launch_bounds__(kSgThreads) sg_digit_base_kernel(unsigned long long* gcount, int passes) {
  __shared__ uint32_t wsum[kSgWarps];
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = (uint32_t)gcount[p * 256 + threadIdx.x];  // totals are at most n < 2^32
    const uint32_t e = block_excl_scan(c, wsum);
    gcount[p * 256 + threadIdx.x] = e;
    __syncthreads();  // wsum is reused by the next pass
  }
}

// Tile status words of the one-sweep scatter: (epoch << 56) | (count << 2) | flag, the epoch
// being the pass + 1 so that words of an earlier pass read as not ready.
constexpr uint64_t kSgAgg = 1, kSgPrefix = 2;
constexpr int kSgLookSpin = 1 << 21;

__device__ __forceinline__ uint64_t sg_word(uint32_t epoch, uint64_t count, uint64_t flag) {
  return ((uint64_t)epoch << 56) | (count << 2) | flag;
}

// Exclusive prefix of digit d over the tiles before `tile` (decoupled look-back): aggregates
// of earlier tiles are summed until a tile with its inclusive prefix is met.  The words of
// kSgWindow predecessors are read together; bounded waits.
constexpr int kSgWindow = 8;

__device__ __forceinline__ uint64_t sg_look_back(uint64_t* status, int64_t tile, int d, uint32_t epoch,
                                                 bool* timed_out) {
  uint64_t excl = 0;
  int64_t j = tile - 1;
  int spins = 0;
  while (j >= 0) {
    uint64_t w[kSgWindow];
#pragma unroll
    for (int q = 0; q < kSgWindow; ++q)
      w[q] = j - q >= 0 ? ld_relaxed_u64(&status[(j - q) * 256 + d]) : sg_word(epoch, 0, kSgPrefix);
    int q = 0;
    bool done = false;
#pragma unroll
    for (; q < kSgWindow; ++q) {  // in order, up to the first word not ready
      const uint64_t x = w[q];
      if ((uint32_t)(x >> 56) != epoch || (x & 3) == 0) break;
      excl += (x & ((1ull << 56) - 1)) >> 2;
      if ((x & 3) == kSgPrefix) {
        done = true;
        break;
      }
    }
    if (done) break;
    j -= q;
    if (q == 0) {
      if (++spins > kSgLookSpin) {
        *timed_out = true;
        return excl;
      }
      if (spins > 32) __nanosleep(128);
    }
  }
  return excl;
}

constexpr int kSgSpin = 1 << 22;  // bound of the bulk copy wait (far above its latency)

template <typename K>
constexpr size_t sg_scatter_smem() {
  return (size_t)kSgTile * 8 + (size_t)kSgTile * sizeof(K) + (size_t)kSgTile * 2 + (size_t)kSgWarps * 256 * 4 +
         2 * 256 * 4 + 64;
}

// Stable scatter of one pass from the current order to the other buffer (one sweep: the tile's
// output offsets come from the digit bases and a look-back over earlier tiles).  Tiles are
// handed out in launch order by a ticket, so every tile looked back at belongs to a block that
// is already running.  The tile's values arrive in shared memory by one bulk copy issued
// first, while the keys are ranked.
template <typename K>
__global__ void __launch_bounds__(kSgThreads, 3)
sg_scatter_kernel(SgBufs<K> b, int64_t n, SgHeader* h, int pass, const unsigned long long* dbase,
                  uint64_t* status) {
  if (pass_skipped(h, pass)) return;  // block-uniform
  __shared__ int64_t s_tile;
  __shared__ int s_bad;
  extern __shared__ __align__(16) unsigned char sg_smem[];
  int64_t* sv = reinterpret_cast<int64_t*>(sg_smem);                       // values, tile order
  K* sk = reinterpret_cast<K*>(sv + kSgTile);                              // keys, digit order
  uint16_t* inv = reinterpret_cast<uint16_t*>(sk + kSgTile);               // tile index of sk[p]
  uint32_t* wh = reinterpret_cast<uint32_t*>(inv + kSgTile);               // [warp][digit]
  uint32_t* lstart = wh + kSgWarps * 256;   // tile-local start of each digit
  uint32_t* gbase = lstart + 256;           // output offset of each digit's run
  uint32_t* wsum = gbase + 256;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wsum + kSgWarps);
  const int src = h->src;
  const SgSrc<K> s = sg_src(b, src);
  K* kd = src == 1 ? b.k1 : b.k0;
  int64_t* vd = src == 1 ? b.v1 : b.v0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) {
    s_tile = (int64_t)atomicAdd(&h->ticket[pass], 1ull);
    s_bad = 0;
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kSgWarps * 256; i += kSgThreads) wh[i] = 0;
  __syncthreads();
  const int64_t t = s_tile;
  const int64_t tile0 = t * kSgTile;
  const int tn = (int)(n - tile0 < kSgTile ? n - tile0 : kSgTile);
  // values: a bulk copy of the even-length prefix (16-byte multiple), the odd last one by a load
  const bool bulk = (src != 0 || b.in_v_aligned) && tn >= 2;
  const int nbulk = bulk ? (tn & ~1) : 0;
  if (threadIdx.x == 0 && bulk) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, (uint32_t)nbulk * 8u);
    tma_load_1d(sv, s.v + tile0, (uint32_t)nbulk * 8u, bar);
  }
  for (int j = nbulk + threadIdx.x; j < tn; j += kSgThreads) sv[j] = s.v[tile0 + j];
  // keys of this warp's span, in rounds of 32 consecutive ones
  K k[kSgItems];
#pragma unroll
  for (int r = 0; r < kSgItems; ++r) {
    const int j = warp * kSgWarpSpan + r * 32 + lane;
    k[r] = j < tn ? (K)(s.k[tile0 + j] ^ s.flip) : (K)0;
  }
  // rank within the warp's span: digit counters of this warp before the key, plus lower lanes
  uint32_t pos[kSgItems];
  uint32_t* myh = wh + warp * 256;
#pragma unroll
  for (int r = 0; r < kSgItems; ++r) {
    const int j = warp * kSgWarpSpan + r * 32 + lane;
    const bool has = j < tn;
    const uint32_t d = sg_digit(k[r], pass);
    const unsigned peers = digit_peers(d, has);
    pos[r] = has ? myh[d] + __popc(peers & lt) : 0u;
    __syncwarp();
    if (has && (peers & lt) == 0) myh[d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: the counts of the warps before (in place), the tile's count published, scanned
  // within the tile, and the earlier tiles' counts looked back at
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kSgWarps; ++w) {
      const uint32_t x = wh[w * 256 + d];
      wh[w * 256 + d] = run;
      run += x;
    }
    st_relaxed_u64(&status[t * 256 + d], sg_word((uint32_t)pass + 1, run, t == 0 ? kSgPrefix : kSgAgg));
    lstart[d] = block_excl_scan(run, wsum);
    gbase[d] = run;  // the tile's count, until the look-back below
  }
  __syncthreads();
  // keys into shared memory in digit order while the earlier tiles finish publishing
#pragma unroll
  for (int r = 0; r < kSgItems; ++r) {
    const int j = warp * kSgWarpSpan + r * 32 + lane;
    if (j < tn) {
      const uint32_t d = sg_digit(k[r], pass);
      const uint32_t p = pos[r] + lstart[d] + wh[warp * 256 + d];
      sk[p] = k[r];
      inv[p] = (uint16_t)j;
    }
  }
  {
    const int d = threadIdx.x;
    const uint32_t epoch = (uint32_t)pass + 1;
    const uint32_t run = gbase[d];
    uint64_t excl = 0;
    if (t > 0) {
      bool timed_out = false;
      excl = sg_look_back(status, t, d, epoch, &timed_out);
      if (timed_out) s_bad = 1;
      st_relaxed_u64(&status[t * 256 + d], sg_word(epoch, excl + run, kSgPrefix));
    }
    gbase[d] = (uint32_t)(dbase[pass * 256 + d] + excl);  // only thread d touches gbase[d]
  }
  bool ok = s_bad == 0;
  if (bulk && !mbar_wait(bar, 0, kSgSpin)) {
    ok = false;
    mbar_wait(bar, 0, kSgSpin);  // the copy may still be landing: wait once more before leaving
  }
  if (!ok) set_status(&h->status, SIRIUS_ERR_TIMEOUT);
  // a block whose offsets or values are not all known writes nothing (no write out of bounds)
  if (__syncthreads_or(!ok)) return;
  // out in digit order: each digit's run is consecutive here and in the output
#pragma unroll 4
  for (int r = 0; r < kSgItems; ++r) {
    const int j = r * kSgThreads + threadIdx.x;
    if (j < tn) {
      const K kk = sk[j];
      const uint32_t d = sg_digit(kk, pass);
      const uint32_t g = gbase[d] + (uint32_t)j - lstart[d];
      kd[g] = kk;
      vd[g] = sv[inv[j]];
    }
  }
}

__global__ void sg_flip_kernel(SgHeader* h, int pass) {
  if (!pass_skipped(h, pass)) h->src = h->src == 1 ? 2 : 1;
}

// ------------------------------------------------------------------ reduction of the runs
// th[t]: segment heads (a key differing from the one before it) among tile t's elements.
template <typename K>
__global__ void __launch_bounds__(kSgThreads)
sg_heads_kernel(SgBufs<K> b, int64_t n, const SgHeader* h, uint32_t* th) {
  __shared__ uint32_t s[kSgWarps];
  const SgSrc<K> src = sg_src(b, h->src);
  const int64_t t = blockIdx.x;
  uint32_t c = 0;
  for (int r = 0; r < kSgItems; ++r) {
    const int64_t i = t * kSgTile + r * kSgThreads + threadIdx.x;
    if (i < n && (i == 0 || src.k[i] != src.k[i - 1])) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kSgWarps; ++w) tot += s[w];
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
  int64_t key;
};

__device__ __forceinline__ void sg_store(const SgOut& o, const SgPart& p) {
  if (p.g >= o.cap) return;
  if (o.keys) o.keys[p.g] = p.key;
  if (o.sum) o.sum[p.g] = p.sum;
  if (o.count) o.count[p.g] = p.cnt;
  if (o.min) o.min[p.g] = p.mn;
  if (o.max) o.max[p.g] = p.mx;
}

__device__ __forceinline__ void sg_merge(const SgOut& o, const SgPart& p) {
  if (p.g >= o.cap) return;
  if (o.keys) o.keys[p.g] = p.key;  // every contributor stores the same key
  if (o.sum) atomicAdd(reinterpret_cast<unsigned long long*>(&o.sum[p.g]), (unsigned long long)p.sum);
  if (o.count) atomicAdd(reinterpret_cast<unsigned long long*>(&o.count[p.g]), (unsigned long long)p.cnt);
  if (o.min) atomicMin(reinterpret_cast<long long*>(&o.min[p.g]), p.mn);
  if (o.max) atomicMax(reinterpret_cast<long long*>(&o.max[p.g]), p.mx);
}

// Warp-level combine of the runs that cross thread boundaries (lanes holding the same group
// are contiguous), then one set of atomics per group by its lowest lane.
__device__ __forceinline__ void sg_merge_warp(const SgOut& o, SgPart p, SgPart* stage) {
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
    sg_merge(o, acc);
  }
  __syncwarp();
}

// Shared-memory index of staged element i with one pad slot after every 16: a thread's 16
// consecutive elements then start in different banks (stride 17).
__device__ __forceinline__ int sg_pad(int i) { return i + (i >> 4); }

constexpr size_t kSgReduceSmem(size_t key_bytes) {
  return (size_t)(kSgTile + kSgTile / 16 + 4) * key_bytes + (size_t)(kSgTile + kSgTile / 16) * 8 +
         (size_t)kSgThreads * sizeof(SgPart) + 64;
}

// Each thread reduces its kSgItems consecutive elements of the tile, staged in shared memory
// (th: the tiles' exclusive group bases).
template <typename K>
__global__ void __launch_bounds__(kSgThreads)
sg_reduce_kernel(SgBufs<K> b, int64_t n, const SgHeader* h, const uint32_t* th, SgOut o) {
  extern __shared__ __align__(16) unsigned char sg_smem[];
  int64_t* sv = reinterpret_cast<int64_t*>(sg_smem);                     // values, padded
  SgPart* stage = reinterpret_cast<SgPart*>(sv + kSgTile + kSgTile / 16);  // kSgThreads parts
  K* sk = reinterpret_cast<K*>(stage + kSgThreads);  // padded: key before, the tile's, key after
  __shared__ uint32_t wsum[kSgWarps];
  const SgSrc<K> s = sg_src(b, h->src);
  const int64_t t = blockIdx.x;
  const int64_t tile0 = t * kSgTile;
  const int tn = (int)(n - tile0 < kSgTile ? n - tile0 : kSgTile);
  for (int j = threadIdx.x; j < tn; j += kSgThreads) {
    sk[sg_pad(j + 1)] = s.k[tile0 + j];
    sv[sg_pad(j)] = s.v[tile0 + j];
  }
  if (threadIdx.x == 0) sk[0] = tile0 > 0 ? s.k[tile0 - 1] : (K)0;
  if (threadIdx.x == 1) sk[sg_pad(tn + 1)] = tile0 + tn < n ? s.k[tile0 + tn] : (K)0;
  __syncthreads();
  // element e of the tile (0-based) is a head iff it is the first row or differs from e - 1
  const int e0 = threadIdx.x * kSgItems;
  const int e_end = e0 + kSgItems < tn ? e0 + kSgItems : tn;
  uint32_t heads = 0;
  for (int e = e0; e < e_end; ++e)
    if ((tile0 + e == 0) || sk[sg_pad(e + 1)] != sk[sg_pad(e)]) ++heads;
  // group of the element before the thread's first one: th[t] + heads before this thread - 1
  int64_t g = (int64_t)th[t] + (int64_t)block_excl_scan(heads, wsum) - 1;
  SgPart first{0, 0, INT64_MAX, INT64_MIN, -1, 0}, last{0, 0, INT64_MAX, INT64_MIN, -1, 0};
  SgPart run{0, 0, INT64_MAX, INT64_MIN, -1, 0};
  bool run_from_head = false;  // the current run began at a head inside this thread
  bool first_done = false;
  for (int e = e0; e < e_end; ++e) {
    const K k = sk[sg_pad(e + 1)];
    const bool head = (tile0 + e == 0) || k != sk[sg_pad(e)];
    if (head) {
      if (run.g >= 0) {
        // the run ended before this head inside the thread
        if (run_from_head) sg_store(o, run);
        else { first = run; first_done = true; }
      }
      ++g;
      run = SgPart{0, 0, INT64_MAX, INT64_MIN, g, unmap_key<K>(k ^ s.flip)};
      run_from_head = true;
    } else if (run.g < 0) {
      run = SgPart{0, 0, INT64_MAX, INT64_MIN, g, unmap_key<K>(k ^ s.flip)};  // continues a run
      run_from_head = false;
    }
    const long long v = sv[sg_pad(e)];
    run.sum += v;
    run.cnt += 1;
    run.mn = v < run.mn ? v : run.mn;
    run.mx = v > run.mx ? v : run.mx;
  }
  if (run.g >= 0) {
    // the last run is complete if it began at a head here and the next element starts a new key
    const bool next_head = tile0 + e_end >= n || sk[sg_pad(e_end + 1)] != sk[sg_pad(e_end)];
    if (run_from_head && next_head) sg_store(o, run);
    else if (!run_from_head && !first_done) first = run;  // one run spanning the whole thread
    else last = run;
  }
  SgPart* st = stage + (threadIdx.x & ~31);
  sg_merge_warp(o, first, st);
  sg_merge_warp(o, last, st);
}

struct SgLayout {
  size_t k1, v0, v1, dbase, status, cnt, part, total;
};

SgLayout sg_layout(int64_t n, int key_width) {
  const int64_t nn = n > 0 ? n : 1;
  const int64_t ntiles = (nn + kSgTile - 1) / kSgTile;
  const int64_t nb = scan_part_entries(ntiles);
  SgLayout L;
  size_t off = align_up(256 + (size_t)nn * key_width, 256);  // header, keys buffer 0
  L.k1 = off;
  off = align_up(off + (size_t)nn * key_width, 256);
  L.v0 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  L.v1 = off;
  off = align_up(off + (size_t)nn * 8, 256);
  L.dbase = off;                                  // 8 passes x 256 digit counts, then bases
  off = align_up(off + (size_t)8 * 256 * 8, 256);
  L.status = off;                                 // tile status words, 256 per tile
  off = align_up(off + (size_t)ntiles * 256 * 8, 256);
  L.cnt = off;                                    // segment heads per tile, then group bases
  off = align_up(off + (size_t)ntiles * 4, 256);
  L.part = off;
  L.total = align_up(off + (size_t)nb * 8, 256);
  return L;
}

__global__ void sg_copy_groups_kernel(const SgHeader* h, int64_t* d_groups) {
  *d_groups = h->status == SIRIUS_OK ? (int64_t)h->groups : -1;
}

template <typename K>
sirius_status sg_run(const void* d_keys, const int64_t* d_vals, int64_t n, const SgOut& o, char* base,
                     const SgLayout& L, SgHeader* hdr, cudaStream_t s) {
  static std::atomic<uint64_t> smem_set0{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(sg_scatter_kernel<K>, (int)sg_scatter_smem<K>(), smem_set0));
  static std::atomic<uint64_t> smem_set1{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(sg_reduce_kernel<K>, (int)kSgReduceSmem(sizeof(K)), smem_set1));
  static std::atomic<uint64_t> smem_set2{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(sg_upfront_kernel<K>, (int)(sizeof(K) * sg_copies<K>() * 256 * 4), smem_set2));
  SgBufs<K> b;
  b.in_k = reinterpret_cast<const K*>(d_keys);
  b.in_v = d_vals;
  b.k0 = reinterpret_cast<K*>(base + 256);
  b.k1 = reinterpret_cast<K*>(base + L.k1);
  b.v0 = reinterpret_cast<int64_t*>(base + L.v0);
  b.v1 = reinterpret_cast<int64_t*>(base + L.v1);
  b.in_v_aligned = ((uintptr_t)d_vals & 15) == 0;
  unsigned long long* dbase = reinterpret_cast<unsigned long long*>(base + L.dbase);
  uint64_t* status = reinterpret_cast<uint64_t*>(base + L.status);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + L.cnt);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(base + L.part);
  const int64_t ntiles = (n + kSgTile - 1) / kSgTile;
  constexpr int kPasses = (int)sizeof(K);
  SIRIUS_CUDA_TRY(cudaMemsetAsync(dbase, 0, (size_t)kPasses * 256 * 8, s));
  SIRIUS_CUDA_TRY(cudaMemsetAsync(status, 0, (size_t)ntiles * 256 * 8, s));
  const int64_t up_grid_want = (n + kSgThreads * 8 - 1) / (kSgThreads * 8);
  const int up_grid = (int)(up_grid_want < (int64_t)sm_count() * 8 ? up_grid_want : (int64_t)sm_count() * 8);
  sg_upfront_kernel<K><<<up_grid, kSgThreads, (size_t)sizeof(K) * sg_copies<K>() * 256 * 4, s>>>(b.in_k, n, hdr,
                                                                                                 dbase);
  SIRIUS_LAUNCH_CHECK();
  sg_digit_base_kernel<<<1, kSgThreads, 0, s>>>(dbase, kPasses);
  SIRIUS_LAUNCH_CHECK();
  sirius_status st;
  for (int pass = 0; pass < kPasses; ++pass) {
    sg_scatter_kernel<K><<<(unsigned)ntiles, kSgThreads, sg_scatter_smem<K>(), s>>>(b, n, hdr, pass, dbase, status);
    SIRIUS_LAUNCH_CHECK();
    sg_flip_kernel<<<1, 1, 0, s>>>(hdr, pass);
    SIRIUS_LAUNCH_CHECK();
  }
  sg_heads_kernel<K><<<(unsigned)ntiles, kSgThreads, 0, s>>>(b, n, hdr, cnt);
  SIRIUS_LAUNCH_CHECK();
  if ((st = exclusive_scan_u32(cnt, ntiles, part, &hdr->groups, s)) != SIRIUS_OK) return st;
  sg_init_out_kernel<<<grid_for(o.cap > 0 ? o.cap : 1, 256), 256, 0, s>>>(o, hdr);
  SIRIUS_LAUNCH_CHECK();
  sg_reduce_kernel<K><<<(unsigned)ntiles, kSgThreads, kSgReduceSmem(sizeof(K)), s>>>(b, n, hdr, cnt, o);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

}  // namespace
}  // namespace sirius

using namespace sirius;

extern "C" size_t sirius_groupby_sort_scratch_bytes(int64_t n) { return sg_layout(n, 8).total; }

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
  const SgLayout L = sg_layout(n, key_width);
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, L.total, s);
  if (st != SIRIUS_OK) return st;
  SgHeader* hdr = (SgHeader*)sc.base;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256, s));
  const SgOut o{d_out_keys, (aggs & SIRIUS_AGG_SUM) ? d_sum : nullptr, d_count,
                (aggs & SIRIUS_AGG_MIN) ? d_min : nullptr, (aggs & SIRIUS_AGG_MAX) ? d_max : nullptr, out_cap};
  PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
  if (n > 0) {
    st = key_width == 4 ? sg_run<uint32_t>(d_keys, d_vals, n, o, sc.base, L, hdr, s)
                        : sg_run<unsigned long long>(d_keys, d_vals, n, o, sc.base, L, hdr, s);
    if (st != SIRIUS_OK) return st;
  }
  if (d_groups) {
    sg_copy_groups_kernel<<<1, 1, 0, s>>>(hdr, d_groups);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_groups) {
    SgHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.status != SIRIUS_OK) {
      set_error("groupby_sort: a bounded wait for a bulk copy ran out");
      return (sirius_status)h.status;
    }
    *h_groups = (int64_t)h.groups;
    if ((int64_t)h.groups > out_cap) {
      set_error("groupby_sort: %lld groups exceed out_cap %lld", (long long)h.groups, (long long)out_cap);
      return SIRIUS_ERR_CAPACITY;
    }
  }
  return SIRIUS_OK;
}
