// String keys (Sec. 4.2: group-by on string keys is among the measured bottlenecks, the
// library path grouping them by sorting).  The GB300 path hashes each string once into a
// dictionary of dense int32 codes and groups the codes with the integer group-by.
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
// and filters): the bytes as 4-byte little-endian words, the tail zero-padded, each mixed in by
// the body round of MurmurHash3_x86_32 (Austin Appleby, public domain); the length and that
// hash's finalizer close it.  The home slot is the hash scaled to the table by a multiply-high.
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

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

__device__ __forceinline__ uint32_t mm3_round(uint32_t h, uint32_t k) {
  k *= 0xcc9e2d51u;
  k = rotl32(k, 15);
  k *= 0x1b873593u;
  h ^= k;
  h = rotl32(h, 13);
  return h * 5u + 0xe6546b64u;
}

// Word j of a string: its bytes 8j .. 8j+7 as a little-endian word, zero past the end.  Read
// as the one or two aligned 8-byte words that hold those bytes -- only words holding at least
// one byte of the string, so no read leaves the pages the column occupies.
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

__device__ uint32_t str_hash(const uint8_t* p, int len, bool weak) {
  uint32_t h = 0x9747b28cu;
  const int words = (len + 7) >> 3;
  for (int j = 0; j < words; ++j) {
    const uint64_t w = str_word(p, len, j);
    h = mm3_round(h, (uint32_t)w);
    if (8 * j + 4 < len) h = mm3_round(h, (uint32_t)(w >> 32));
  }
  h = fmix32(h ^ (uint32_t)len);
  if (weak) h = (h & 0xFFu) + 1u;  // 256 values: distinct strings share hashes (tests)
  return h ? h : 1u;
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

__global__ void __launch_bounds__(kDictThreads)
dict_insert_kernel(StrCol c, DictSlot* slots, uint32_t* smin, int64_t cap, uint32_t* row_slot, DictHeader* hdr,
                   int weak) {
  const uint64_t mask = (uint64_t)cap - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a, len;
    uint32_t found = 0xFFFFFFFFu;
    if (str_bounds(c, i, &a, &len, &hdr->status)) {
      const uint8_t* p = c.chars + a;
      const uint64_t h = str_hash(p, len, weak != 0);
      uint64_t s = (h * (uint64_t)cap) >> 32;  // cap <= 2^32
      int64_t left = cap;  // slots not yet visited
      while (left > 0) {
        // scan to the first slot that is empty or carries this hash (a short, tight loop)
        unsigned long long hs = __ldcg(&slots[s].hash);
        while (hs != 0 && hs != h && --left > 0) {
          s = (s + 1) & mask;
          hs = __ldcg(&slots[s].hash);
        }
        if (left == 0) break;
        DictSlot* sl = &slots[s];
        // read through L2 (slots change while the kernel runs); a torn or stale read can only
        // show "empty" or "not yet written", which the compare-and-swap settles
        unsigned long long rep = __ldcg(&sl->rep);
        if (hs == 0 || rep == 0) {
          unsigned long long olo, ohi;
          const unsigned long long mine = ((unsigned long long)(uint32_t)len << 32) | (unsigned long long)(a + 1);
          cas128(reinterpret_cast<unsigned long long*>(sl), 0ull, 0ull, h, mine, olo, ohi);
          if (olo == 0) {  // claimed: this row represents its string
            found = (uint32_t)s;
            break;
          }
          hs = olo;
          rep = ohi;
        }
        if (hs == h) {
          const int32_t ra = (int32_t)(uint32_t)rep - 1, rlen = (int32_t)(rep >> 32);
          if (rlen == len && str_equal(p, c.chars + ra, len)) {
            found = (uint32_t)s;
            break;
          }
        }
        s = (s + 1) & mask;  // another string here (same hash, or claimed just before us)
        --left;
      }
      if (found == 0xFFFFFFFFu) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
    }
    row_slot[i] = found;
    if (found != 0xFFFFFFFFu && (uint32_t)i < __ldcg(&smin[found])) atomicMin(&smin[found], (uint32_t)i);
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
sirius_status dict_run(const StrCol& c, int64_t hint, uint32_t flags, int32_t* d_codes, int64_t* d_dict_rows,
                       int64_t dict_cap, char* base, const DictLayout& L, cudaStream_t s) {
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
  if (c.n == 0) return SIRIUS_OK;
  dict_insert_kernel<<<grid_for(c.n, kDictThreads), kDictThreads, 0, s>>>(
      c, slots, smin, L.cap, row_slot, hdr, (flags & SIRIUS_DICT_WEAK_HASH) ? 1 : 0);
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
  dict_assign_kernel<<<grid_for(c.n, 256), 256, 0, s>>>(row_slot, c.n, slot_code, d_codes);
  SIRIUS_LAUNCH_CHECK();
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

// Group-by outputs of the codes (in table order) moved to their code's position.
struct StrGroupOut {
  int64_t* rows;
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t cap;
};

__global__ void strgroup_place_kernel(const int64_t* gkey, const int64_t* gsum, const int64_t* gcount,
                                      const int64_t* gmin, const int64_t* gmax, const int64_t* d_groups,
                                      const int64_t* dict_rows, StrGroupOut o) {
  const int64_t g = *d_groups;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t code = gkey[i];
    if (code < 0 || code >= o.cap) continue;
    if (o.rows) o.rows[code] = dict_rows[code];
    if (o.sum) o.sum[code] = gsum[i];
    o.count[code] = gcount[i];
    if (o.min) o.min[code] = gmin[i];
    if (o.max) o.max[code] = gmax[i];
  }
}

struct StrGroupLayout {
  DictLayout d;
  size_t codes, dict_rows, gout, gcount, gb, total;
};

StrGroupLayout strgroup_layout(int64_t n, int64_t hint) {
  StrGroupLayout L;
  L.d = dict_layout(n, hint);
  const int64_t nn = n > 0 ? n : 1;
  size_t off = L.d.total;
  L.codes = off;
  off = align_up(off + (size_t)nn * 4, 256);
  L.dict_rows = off;
  off = align_up(off + (size_t)L.d.cap * 8, 256);
  L.gout = off;  // five columns of cap entries
  off = align_up(off + (size_t)L.d.cap * 8 * 5, 256);
  L.gcount = off;
  off = align_up(off + 8, 256);
  L.gb = off;
  L.total = align_up(off + sirius_groupby_scratch_bytes(hint), 256);
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
  int32_t* codes = (int32_t*)(base + L.codes);
  int64_t* dict_rows = (int64_t*)(base + L.dict_rows);
  int64_t* gout = (int64_t*)(base + L.gout);
  int64_t* gcount_dev = (int64_t*)(base + L.gcount);
  const int64_t cap = L.d.cap;
  {
    PhaseTimer pt(s, SIRIUS_PHASE_GROUPBY);
    const StrCol c{d_offsets, d_chars, n, n_chars};
    if ((st = dict_run(c, distinct_hint, flags, codes, dict_rows, cap, base, L.d, s)) != SIRIUS_OK) return st;
  }
  // the codes grouped by the hash group-by (a dictionary that accepted D strings has at most
  // as many as a group table of the same hint takes), then moved to code order
  if (n > 0) {
    if ((st = sirius_groupby_agg(codes, 4, d_vals, n, aggs, distinct_hint, gout, gout + cap, gout + 2 * cap,
                                 gout + 3 * cap, gout + 4 * cap, cap, gcount_dev, nullptr, base + L.gb,
                                 L.total - L.gb, stream)) != SIRIUS_OK)
      return st;
    const StrGroupOut o{d_out_rows, (aggs & SIRIUS_AGG_SUM) ? d_sum : nullptr, d_count,
                        (aggs & SIRIUS_AGG_MIN) ? d_min : nullptr, (aggs & SIRIUS_AGG_MAX) ? d_max : nullptr,
                        out_cap};
    strgroup_place_kernel<<<grid_for(cap, 256), 256, 0, s>>>(gout, gout + cap, gout + 2 * cap, gout + 3 * cap,
                                                             gout + 4 * cap, gcount_dev, dict_rows, o);
    SIRIUS_LAUNCH_CHECK();
  }
  if (d_groups) {
    dict_copy_count_kernel<<<1, 1, 0, s>>>(hdr, d_groups);
    SIRIUS_LAUNCH_CHECK();
  }
  if (h_groups) return dict_finish(hdr, out_cap, h_groups, "groupby_string", s);
  return SIRIUS_OK;
}
