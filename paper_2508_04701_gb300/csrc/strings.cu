// String keys (Sec. 4.2: group-by on string keys is among the measured bottlenecks, the
// library path grouping them by sorting).  The GB300 path hashes each string once into a
// dictionary of dense int32 codes; GROUP BY a string column aggregates each row's value into its
// string's slot in the same pass, and lists the groups in code order.
//
// Dictionary encoding, exact: a string's 32-bit hash (below) selects a slot of an
// open-addressing table; a slot holds (hash, where the representative's bytes are) and is
// claimed by a 128-bit compare-and-swap, so the pair is never seen half written.  A row whose
// hash equals a slot's compares its bytes with the representative's: equal -> the same string;
// different -> a hash collision, and the probe goes on to the next slot.  Each slot also keeps the smallest
// row holding its string.  Codes number the distinct strings in order of first occurrence:
// the first rows are marked in a bitmap over the rows, and a string's code is the number of
// marks before its first row (an exclusive scan of the bitmap words' popcounts).
//
// String hash (32 bits; the table settles equality by bytes, so the hash only picks the slot
// and filters): the bytes as 8-byte little-endian words, the tail zero-padded; each word's two
// halves, offset by its position, go through MurmurHash3's finalizer fmix32 (Austin Appleby,
// public domain); the sum of those and of the length, finalized once more, is the hash.  A sum
// does not depend on the order the words are taken in, so a warp hashes its 32 strings word by
// word across its lanes.  The home slot is the hash scaled to the table by a multiply-high.
//
// Work per warp: 32 consecutive rows, whose bytes are contiguous.  Their words are dealt out to
// the lanes in rounds of 32 (consecutive lanes read consecutive words), each word's mix added
// to its string's sum in shared memory; then every lane probes the table for its own string,
// and the byte comparison with a slot's representative is dealt out the same way.  A warp
// whose strings hold more than kWarpWords words in all works string by string per lane.
#include "scan.cuh"

namespace sirius {
namespace {

constexpr int kDictThreads = 256;

struct DictHeader {
  int32_t status;
  uint32_t pad0;
  unsigned long long pad1;
  unsigned long long ndict;    // D, the number of distinct strings
  unsigned long long groups;   // string group-by: G (= D)
  unsigned long long pad[28];
};
static_assert(sizeof(DictHeader) == 256, "dictionary header is 256 bytes");

// A slot: lo = hash (0 = empty); hi = the representative's length << 32 | (its first byte's
// offset + 1) (0 = not yet written).
struct __align__(16) DictSlot {
  unsigned long long hash;
  unsigned long long rep;
};


// Word j of a string: its bytes 8j .. 8j+7 as a little-endian word, zero past the end.  Read
// as the one or two aligned 8-byte words that hold those bytes -- only words holding at least
// one byte of the string, so no read leaves the pages the column occupies.
// Aggregates of one string for GROUP BY a string column (32 bytes: one sector).
struct __align__(32) SlotAgg {
  unsigned long long sum;    // two's-complement sum (exact while the true sum fits int64)
  unsigned long long count;
  long long mn, mx;
};

__global__ void slot_agg_init_kernel(SlotAgg* agg, int64_t cap) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap; s += (int64_t)gridDim.x * blockDim.x)
    agg[s] = SlotAgg{0ull, 0ull, INT64_MAX, INT64_MIN};
}

__device__ __forceinline__ uint64_t str_word(const uint8_t* p, int len, int j) {
  const int nb = len - 8 * j < 8 ? len - 8 * j : 8;  // 1..8
  const uintptr_t ua = (uintptr_t)(p + 8 * j);
  const uint64_t* aw = reinterpret_cast<const uint64_t*>(ua & ~(uintptr_t)7);
  const int sh = (int)(ua & 7);
  uint64_t v = __ldg(aw) >> (8 * sh);
  if (sh + nb > 8) v |= __ldg(aw + 1) << (64 - 8 * sh);
  if (nb < 8) v &= (1ull << (8 * nb)) - 1;
  return v;
}

// Word j's contribution: its two halves, each offset by a constant times the word's position,
// through MurmurHash3's fmix32.  A string's hash is the finalized sum of its words'
// contributions plus its length, so the words can be mixed in any order (by different lanes).
__device__ __forceinline__ uint32_t mixw(uint64_t w, int j) {
  return fmix32((uint32_t)w + 0x9e3779b9u * (uint32_t)(2 * j + 1)) +
         fmix32((uint32_t)(w >> 32) + 0x85ebca6bu * (uint32_t)(2 * j + 2));
}

__device__ __forceinline__ uint32_t hash_finish(uint32_t acc, int len, bool weak) {
  uint32_t h = fmix32(acc + 0xc2b2ae35u * (uint32_t)len);
  if (weak) h = (h & 0xFFu) + 1u;  // 256 values: distinct strings share hashes (tests)
  return h ? h : 1u;
}

__device__ uint32_t str_hash(const uint8_t* p, int len, bool weak) {
  uint32_t acc = 0;
  const int words = (len + 7) >> 3;
  for (int j = 0; j < words; ++j) acc += mixw(str_word(p, len, j), j);
  return hash_finish(acc, len, weak);
}

__device__ __forceinline__ bool str_equal(const uint8_t* a, const uint8_t* b, int len) {
  const int words = (len + 7) >> 3;
  for (int j = 0; j < words; ++j)
    if (str_word(a, len, j) != str_word(b, len, j)) return false;
  return true;
}

struct StrCol {
  const int32_t* off;
  const uint8_t* chars;
  int64_t n;
  int64_t n_chars;
};

// Bounds of row i's bytes; false (and INVALID) when the offsets leave [0, n_chars] or decrease.
__device__ __forceinline__ bool str_bounds(const StrCol& c, int64_t i, int32_t* a, int32_t* len, int32_t* status) {
  const int32_t lo = c.off[i], hi = c.off[i + 1];
  if (lo < 0 || hi < lo || (int64_t)hi > c.n_chars) {
    set_status(status, SIRIUS_ERR_INVALID);
    return false;
  }
  *a = lo;
  *len = hi - lo;
  return true;
}

constexpr int kWarpWords = 256;  // words of a warp's 32 strings dealt out across its lanes

// Probe for a string from slot s with `left` slots still unvisited: the first slot that is empty
// (claimed by compare-and-swap) or holds the same string (same hash, equal bytes).
__device__ uint32_t probe_lane(DictSlot* slots, uint64_t mask, uint64_t s, int64_t left, uint64_t h,
                               const uint8_t* chars, int32_t a, int32_t len) {
  while (left > 0) {
    // scan to the first slot that is empty or carries this hash (a short, tight loop)
    unsigned long long hs = __ldcg(&slots[s].hash);
    while (hs != 0 && hs != h && --left > 0) {
      s = (s + 1) & mask;
      hs = __ldcg(&slots[s].hash);
    }
    if (left == 0) break;
    DictSlot* sl = &slots[s];
    // read through L2 (slots change while the kernel runs); a torn or stale read can only show
    // "empty" or "not yet written", which the compare-and-swap settles
    unsigned long long rep = __ldcg(&sl->rep);
    if (hs == 0 || rep == 0) {
      unsigned long long olo, ohi;
      const unsigned long long mine = ((unsigned long long)(uint32_t)len << 32) | (unsigned long long)(a + 1);
      cas128(reinterpret_cast<unsigned long long*>(sl), 0ull, 0ull, h, mine, olo, ohi);
      if (olo == 0) return (uint32_t)s;  // claimed: this row represents its string
      hs = olo;
      rep = ohi;
    }
    if (hs == h) {
      const int32_t ra = (int32_t)(uint32_t)rep - 1, rlen = (int32_t)(rep >> 32);
      if (rlen == len && str_equal(chars + a, chars + ra, len)) return (uint32_t)s;
    }
    s = (s + 1) & mask;  // another string here (same hash, or claimed just before us)
    --left;
  }
  return 0xFFFFFFFFu;
}

__global__ void __launch_bounds__(kDictThreads, 6)
dict_insert_kernel(StrCol c, DictSlot* slots, uint32_t* smin, int64_t cap, uint32_t* row_slot, DictHeader* hdr,
                   int weak, const int64_t* __restrict__ vals, SlotAgg* agg, uint32_t aggs) {
  __shared__ uint8_t s_map[kDictThreads / 32][kWarpWords];  // word -> lane of its string
  __shared__ uint32_t s_acc[kDictThreads / 32][32];          // hash sums, then "bytes differ" flags
  const uint64_t mask = (uint64_t)cap - 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* map = s_map[wib];
  uint32_t* acc = s_acc[wib];
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < c.n; base += warps * 32) {
    const int64_t i = base + lane;
    int32_t a = 0, len = 0;
    const bool valid = i < c.n && str_bounds(c, i, &a, &len, &hdr->status);
    if (!valid) len = 0;
    const int words = (len + 7) >> 3;
    int P = words;  // exclusive prefix of the words over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, P, o);
      if (lane >= o) P += y;
    }
    const int W = __shfl_sync(0xffffffffu, P, 31);
    P -= words;
    uint32_t found = 0xFFFFFFFFu;
    if (W > kWarpWords) {  // long strings: each lane on its own (warp-uniform branch)
      if (valid) {
        const uint64_t h = str_hash(c.chars + a, len, weak != 0);
        found = probe_lane(slots, mask, (h * (uint64_t)cap) >> 32, cap, h, c.chars, a, len);
      }
    } else {
      // hash: the warp's words dealt out across the lanes
      acc[lane] = 0;
      for (int k = 0; k < words; ++k) map[P + k] = (uint8_t)lane;
      __syncwarp();
      for (int q0 = 0; q0 < W; q0 += 32) {
        const int q = q0 + lane;
        const int sl = q < W ? map[q] : 0;
        const int ps = __shfl_sync(0xffffffffu, P, sl);
        const int as = __shfl_sync(0xffffffffu, a, sl);
        const int ls = __shfl_sync(0xffffffffu, len, sl);
        if (q < W) atomicAdd(&acc[sl], mixw(str_word(c.chars + as, ls, q - ps), q - ps));
      }
      __syncwarp();
      const uint64_t h = hash_finish(acc[lane], len, weak != 0);
      // probe: the first slot that is empty (claim it) or carries this hash (compare below)
      uint64_t s = (h * (uint64_t)cap) >> 32;
      int64_t left = cap;
      bool cmp = false;
      int32_t ra = 0;
      if (valid) {
        unsigned long long hs = __ldcg(&slots[s].hash);
        while (hs != 0 && hs != h && --left > 0) {
          s = (s + 1) & mask;
          hs = __ldcg(&slots[s].hash);
        }
        if (left > 0) {
          DictSlot* sl = &slots[s];
          unsigned long long rep = __ldcg(&sl->rep);
          if (hs == 0 || rep == 0) {
            unsigned long long olo, ohi;
            const unsigned long long mine = ((unsigned long long)(uint32_t)len << 32) | (unsigned long long)(a + 1);
            cas128(reinterpret_cast<unsigned long long*>(sl), 0ull, 0ull, h, mine, olo, ohi);
            if (olo == 0) found = (uint32_t)s;
            hs = olo;
            rep = ohi;
          }
          if (found == 0xFFFFFFFFu && hs == h && (int32_t)(rep >> 32) == len) {
            cmp = true;
            ra = (int32_t)(uint32_t)rep - 1;
          }
        }
      }
      // byte comparison with the representative, dealt out the same way (acc: 1 = differ)
      __syncwarp();
      acc[lane] = 0;
      __syncwarp();
      for (int q0 = 0; q0 < W; q0 += 32) {
        const int q = q0 + lane;
        const int sl = q < W ? map[q] : 0;
        const int ps = __shfl_sync(0xffffffffu, P, sl);
        const int as = __shfl_sync(0xffffffffu, a, sl);
        const int ls = __shfl_sync(0xffffffffu, len, sl);
        const int rs = __shfl_sync(0xffffffffu, ra, sl);
        const bool cs = __shfl_sync(0xffffffffu, cmp, sl);
        if (q < W && cs && str_word(c.chars + as, ls, q - ps) != str_word(c.chars + rs, ls, q - ps)) acc[sl] = 1;
      }
      __syncwarp();
      if (cmp && acc[lane] == 0) found = (uint32_t)s;
      // the rest (a different string at this slot: hash collision, other length, or a claim
      // lost to another string) probes on by itself
      if (valid && found == 0xFFFFFFFFu && left > 0)
        found = probe_lane(slots, mask, (s + 1) & mask, left - 1, h, c.chars, a, len);
      __syncwarp();
    }
    if (valid && found == 0xFFFFFFFFu) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
    if (i < c.n) row_slot[i] = found;
    // the smallest row of each string, and for GROUP BY the row's value into its string's
    // aggregates: reductions whose results nobody waits for
    if (found != 0xFFFFFFFFu) {
      atomicMin(&smin[found], (uint32_t)i);
      if (agg) {
        const long long v = vals[i];
        SlotAgg* g = &agg[found];
        atomicAdd(&g->count, 1ull);
        if (aggs & SIRIUS_AGG_SUM) atomicAdd(&g->sum, (unsigned long long)v);
        if (aggs & SIRIUS_AGG_MIN) atomicMin(&g->mn, v);
        if (aggs & SIRIUS_AGG_MAX) atomicMax(&g->mx, v);
      }
    }
  }
}

// The first row of each string marked in the row bitmap.
__global__ void dict_mark_kernel(const DictSlot* slots, const uint32_t* smin, int64_t cap, uint32_t* bits) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap; s += (int64_t)gridDim.x * blockDim.x) {
    if (slots[s].hash == 0) continue;
    const uint32_t r = smin[s];
    atomicOr(&bits[r >> 5], 1u << (r & 31));
  }
}

__global__ void dict_popc_kernel(const uint32_t* bits, int64_t words, uint32_t* cnt) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(bits[w]);
}

// Code of each slot: marks before its first row; the dictionary lists first rows by code.
__global__ void dict_code_kernel(const DictSlot* slots, const uint32_t* smin, int64_t cap, const uint32_t* bits,
                                 const uint32_t* base, uint32_t* slot_code, int64_t* dict_rows, int64_t dict_cap) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap; s += (int64_t)gridDim.x * blockDim.x) {
    if (slots[s].hash == 0) continue;
    const uint32_t r = smin[s];
    const uint32_t code = base[r >> 5] + __popc(bits[r >> 5] & ((1u << (r & 31)) - 1u));
    slot_code[s] = code;
    if (dict_rows && (int64_t)code < dict_cap) dict_rows[code] = r;
  }
}

// More distinct strings than the table's load limit -> TABLE_FULL (as for the group table).
__global__ void dict_check_kernel(DictHeader* hdr, unsigned long long limit) {
  if (hdr->ndict > limit) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
}

__global__ void dict_assign_kernel(const uint32_t* row_slot, int64_t n, const uint32_t* slot_code, int32_t* codes) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = row_slot[i];
    codes[i] = s == 0xFFFFFFFFu ? -1 : (int32_t)slot_code[s];
  }
}

struct DictLayout {
  int64_t cap, words;
  size_t slots, smin, slot_code, row_slot, bits, cnt, part, total;
};

DictLayout dict_layout(int64_t n, int64_t hint) {
  DictLayout L;
  L.cap = group_capacity_for(hint);
  const int64_t nn = n > 0 ? n : 1;
  L.words = (nn + 31) / 32;
  size_t off = 256;  // header
  L.slots = off;
  off = align_up(off + (size_t)L.cap * sizeof(DictSlot), 256);
  L.smin = off;
  off = align_up(off + (size_t)L.cap * 4, 256);
  L.slot_code = off;
  off = align_up(off + (size_t)L.cap * 4, 256);
  L.row_slot = off;
  off = align_up(off + (size_t)nn * 4, 256);
  L.bits = off;
  off = align_up(off + (size_t)L.words * 4, 256);
  L.cnt = off;
  off = align_up(off + (size_t)L.words * 4, 256);
  L.part = off;
  L.total = align_up(off + (size_t)scan_part_entries(L.words) * 8, 256);
  return L;
}

// The encoding proper, into a scratch region laid out by dict_layout; D goes to hdr->ndict.
// With agg (GROUP BY), each row's value is aggregated into its string's slot during the insert.
sirius_status dict_run(const StrCol& c, int64_t hint, uint32_t flags, int32_t* d_codes, int64_t* d_dict_rows,
                       int64_t dict_cap, char* base, const DictLayout& L, cudaStream_t s,
                       const int64_t* vals = nullptr, SlotAgg* agg = nullptr, uint32_t aggs = 0) {
  DictHeader* hdr = (DictHeader*)base;
  DictSlot* slots = (DictSlot*)(base + L.slots);
  uint32_t* smin = (uint32_t*)(base + L.smin);
  uint32_t* slot_code = (uint32_t*)(base + L.slot_code);
  uint32_t* row_slot = (uint32_t*)(base + L.row_slot);
  uint32_t* bits = (uint32_t*)(base + L.bits);
  uint32_t* cnt = (uint32_t*)(base + L.cnt);
  unsigned long long* part = (unsigned long long*)(base + L.part);
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256, s));
  SIRIUS_CUDA_TRY(cudaMemsetAsync(slots, 0, (size_t)L.cap * sizeof(DictSlot), s));
  SIRIUS_CUDA_TRY(cudaMemsetAsync(smin, 0xFF, (size_t)L.cap * 4, s));
  SIRIUS_CUDA_TRY(cudaMemsetAsync(bits, 0, (size_t)L.words * 4, s));
  if (agg) {
    slot_agg_init_kernel<<<grid_for(L.cap, 256), 256, 0, s>>>(agg, L.cap);
    SIRIUS_LAUNCH_CHECK();
  }
  if (c.n == 0) return SIRIUS_OK;
  dict_insert_kernel<<<grid_for(c.n, kDictThreads), kDictThreads, 0, s>>>(
      c, slots, smin, L.cap, row_slot, hdr, (flags & SIRIUS_DICT_WEAK_HASH) ? 1 : 0, vals, agg, aggs);
  SIRIUS_LAUNCH_CHECK();
  dict_mark_kernel<<<grid_for(L.cap, 256), 256, 0, s>>>(slots, smin, L.cap, bits);
  SIRIUS_LAUNCH_CHECK();
  dict_popc_kernel<<<grid_for(L.words, 256), 256, 0, s>>>(bits, L.words, cnt);
  SIRIUS_LAUNCH_CHECK();
  sirius_status st = exclusive_scan_u32(cnt, L.words, part, &hdr->ndict, s);
  if (st != SIRIUS_OK) return st;
  dict_check_kernel<<<1, 1, 0, s>>>(hdr, group_limit_for(L.cap));
  SIRIUS_LAUNCH_CHECK();
  dict_code_kernel<<<grid_for(L.cap, 256), 256, 0, s>>>(slots, smin, L.cap, bits, cnt, slot_code, d_dict_rows,
                                                        dict_cap);
  SIRIUS_LAUNCH_CHECK();
  if (d_codes) {
    dict_assign_kernel<<<grid_for(c.n, 256), 256, 0, s>>>(row_slot, c.n, slot_code, d_codes);
    SIRIUS_LAUNCH_CHECK();
  }
  return SIRIUS_OK;
}

sirius_status check_strcol(const int32_t* d_offsets, const uint8_t* d_chars, int64_t n, int64_t n_chars) {
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows - 1, "strings: n=%lld out of range", (long long)n);
  SIRIUS_REQUIRE(n_chars >= 0 && n_chars <= 0x7FFFFFFFll, "strings: n_chars=%lld out of range (int32 offsets)",
                 (long long)n_chars);
  SIRIUS_REQUIRE(n == 0 || d_offsets, "strings: NULL offsets");
  SIRIUS_REQUIRE(n_chars == 0 || d_chars, "strings: NULL chars");
  return SIRIUS_OK;
}

// Host read of the header after a synchronize: the device status, then D against a capacity.
sirius_status dict_finish(const DictHeader* hdr, int64_t cap, int64_t* h_count, const char* what,
                          cudaStream_t s) {
  DictHeader h;
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.status == SIRIUS_ERR_TABLE_FULL) {
    set_error("%s: more distinct strings than the table takes (hint too small)", what);
    return SIRIUS_ERR_TABLE_FULL;
  }
  if (h.status != SIRIUS_OK) {
    set_error("%s: offsets outside [0, n_chars] or decreasing", what);
    return (sirius_status)h.status;
  }
  *h_count = (int64_t)h.ndict;
  if ((int64_t)h.ndict > cap) {
    set_error("%s: %lld distinct strings exceed the output capacity %lld", what, (long long)h.ndict,
              (long long)cap);
    return SIRIUS_ERR_CAPACITY;
  }
  return SIRIUS_OK;
}

__global__ void dict_copy_count_kernel(const DictHeader* h, int64_t* d_out) {
  *d_out = h->status == SIRIUS_OK ? (int64_t)h->ndict : -1;
}

// GROUP BY outputs: each string's aggregates moved from its slot to its code's position.
struct StrGroupOut {
  int64_t* rows;
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t cap;
};

__global__ void strgroup_place_kernel(const DictSlot* slots, const uint32_t* smin, const uint32_t* slot_code,
                                      const SlotAgg* agg, int64_t cap, StrGroupOut o) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap; s += (int64_t)gridDim.x * blockDim.x) {
    if (slots[s].hash == 0) continue;
    const int64_t code = slot_code[s];
    if (code >= o.cap) continue;
    const SlotAgg g = agg[s];
    if (o.rows) o.rows[code] = smin[s];
    if (o.sum) o.sum[code] = (int64_t)g.sum;
    o.count[code] = (int64_t)g.count;
    if (o.min) o.min[code] = g.mn;
    if (o.max) o.max[code] = g.mx;
  }
}

struct StrGroupLayout {
  DictLayout d;
  size_t agg, total;
};

StrGroupLayout strgroup_layout(int64_t n, int64_t hint) {
  StrGroupLayout L;
  L.d = dict_layout(n, hint);
  L.agg = L.d.total;
  L.total = align_up(L.agg + (size_t)L.d.cap * sizeof(SlotAgg), 256);
  return L;
}

}  // namespace
}  // namespace sirius

using namespace sirius;

extern "C" int64_t sirius_dict_capacity(int64_t distinct_hint) {
  return (int64_t)group_limit_for(group_capacity_for(distinct_hint));
}

extern "C" size_t sirius_dict_scratch_bytes(int64_t n, int64_t distinct_hint) {
  return dict_layout(n, distinct_hint).total;
}

extern "C" sirius_status sirius_dict_encode(const int32_t* d_offsets, const uint8_t* d_chars, int64_t n_chars,
                                            int64_t n, int64_t distinct_hint, uint32_t flags, int32_t* d_codes,
                                            int64_t* d_dict_rows, int64_t dict_cap, int64_t* d_ndict,
                                            int64_t* h_ndict, void* d_scratch, size_t scratch_bytes,
                                            sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = check_strcol(d_offsets, d_chars, n, n_chars);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(n == 0 || d_codes, "dict_encode: NULL codes");
  SIRIUS_REQUIRE(dict_cap >= 0, "dict_encode: negative dict_cap");
  SIRIUS_REQUIRE(distinct_hint <= (1ll << 31), "dict_encode: distinct_hint above 2^31");
  SIRIUS_REQUIRE((flags & ~(uint32_t)SIRIUS_DICT_WEAK_HASH) == 0, "dict_encode: unknown flags 0x%x", flags);
  const DictLayout L = dict_layout(n, distinct_hint);
  Scratch sc;
  if ((st = sc.acquire(d_scratch, scratch_bytes, L.total, s)) != SIRIUS_OK) return st;
  PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
  const StrCol c{d_offsets, d_chars, n, n_chars};
  if ((st = dict_run(c, distinct_hint, flags, d_codes, d_dict_rows, dict_cap, sc.base, L, s)) != SIRIUS_OK)
    return st;
  if (d_ndict) {
    dict_copy_count_kernel<<<1, 1, 0, s>>>((const DictHeader*)sc.base, d_ndict);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_ndict) return dict_finish((const DictHeader*)sc.base, dict_cap, h_ndict, "dict_encode", s);
  return SIRIUS_OK;
}

extern "C" size_t sirius_groupby_string_scratch_bytes(int64_t n, int64_t distinct_hint) {
  return strgroup_layout(n, distinct_hint).total;
}

extern "C" sirius_status sirius_groupby_string(const int32_t* d_offsets, const uint8_t* d_chars, int64_t n_chars,
                                               const int64_t* d_vals, int64_t n, int64_t distinct_hint,
                                               uint32_t flags, uint32_t aggs, int64_t* d_out_rows, int64_t* d_sum,
                                               int64_t* d_count, int64_t* d_min, int64_t* d_max, int64_t out_cap,
                                               int64_t* d_groups, int64_t* h_groups, void* d_scratch,
                                               size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  sirius_status st = check_strcol(d_offsets, d_chars, n, n_chars);
  if (st != SIRIUS_OK) return st;
  SIRIUS_REQUIRE(n == 0 || d_vals, "groupby_string: NULL values");
  SIRIUS_REQUIRE(d_count, "groupby_string: NULL count output");
  SIRIUS_REQUIRE(out_cap >= 0, "groupby_string: negative out_cap");
  SIRIUS_REQUIRE(aggs <= SIRIUS_AGG_ALL, "groupby_string: bad aggregate mask");
  SIRIUS_REQUIRE(distinct_hint <= (1ll << 31), "groupby_string: distinct_hint above 2^31");
  SIRIUS_REQUIRE((flags & ~(uint32_t)SIRIUS_DICT_WEAK_HASH) == 0, "groupby_string: unknown flags 0x%x", flags);
  const StrGroupLayout L = strgroup_layout(n, distinct_hint);
  Scratch sc;
  if ((st = sc.acquire(d_scratch, scratch_bytes, L.total, s)) != SIRIUS_OK) return st;
  char* base = sc.base;
  DictHeader* hdr = (DictHeader*)base;
  SlotAgg* agg = (SlotAgg*)(base + L.agg);
  {
    PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
    const StrCol c{d_offsets, d_chars, n, n_chars};
    if ((st = dict_run(c, distinct_hint, flags, nullptr, nullptr, 0, base, L.d, s, d_vals, agg, aggs)) !=
        SIRIUS_OK)
      return st;
    if (n > 0) {
      const StrGroupOut o{d_out_rows, (aggs & SIRIUS_AGG_SUM) ? d_sum : nullptr, d_count,
                          (aggs & SIRIUS_AGG_MIN) ? d_min : nullptr, (aggs & SIRIUS_AGG_MAX) ? d_max : nullptr,
                          out_cap};
      strgroup_place_kernel<<<grid_for(L.d.cap, 256), 256, 0, s>>>(
          (const DictSlot*)(base + L.d.slots), (const uint32_t*)(base + L.d.smin),
          (const uint32_t*)(base + L.d.slot_code), agg, L.d.cap, o);
      SIRIUS_LAUNCH_CHECK();
    }
  }
  if (d_groups) {
    dict_copy_count_kernel<<<1, 1, 0, s>>>(hdr, d_groups);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_groups) return dict_finish(hdr, out_cap, h_groups, "groupby_string", s);
  return SIRIUS_OK;
}
