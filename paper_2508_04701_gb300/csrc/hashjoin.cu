// A1 / A3 / A4: hash join build and probe, and late materialisation by row id
// (Sec. 3.2.2 join and materialisation operators; Sec. 4.2: joins dominate query time).
//
// Table layout in caller memory: a 256-byte header (has_dups flag, status) followed by
// `capacity` slots.  4-byte keys: one uint64 slot = key (low word) | payload << 32.
// 8-byte keys: a 16-byte slot {uint64 key, uint32 payload, uint32 pad}.  A slot is empty when
// its payload is 0xFFFFFFFF, which no row id takes (row counts stay below 2^32 - 1), so every
// key value -- including all-ones -- can be stored.  Inserts walk linearly from the key's home
// slot and claim the first empty slot with a single compare-and-swap of the whole slot; a walk
// that passes a slot holding the same key records a duplicate.  Two inserts of equal keys walk
// the same sequence, so the later one always passes the earlier one's slot: the flag is exact.
#include "pipeline.cuh"

namespace sirius {
namespace {

constexpr int kThreads = 256;

__global__ void join_build32_kernel(const int32_t* __restrict__ keys, int64_t m,
                                    uint64_t* __restrict__ slots, uint32_t cap, JoinHeader* hdr) {
  bool dup = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = (uint32_t)keys[j];
    const uint64_t desired = (uint64_t)key | ((uint64_t)(uint32_t)j << 32);
    if (!join_insert32(slots, cap, key, desired, dup)) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) hdr->has_dups = 1;
}

__global__ void join_build64_kernel(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                    int64_t m, ulonglong2* __restrict__ slots, uint32_t cap,
                                    JoinHeader* hdr) {
  bool dup = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = pack_key64(hi[j], lo[j]);
    if (!join_insert64(slots, cap, key, (uint32_t)j, dup)) set_status(&hdr->status, SIRIUS_ERR_TABLE_FULL);
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) hdr->has_dups = 1;
}

// Probe of a table holding duplicate keys: one probe row per lane per round; a round ends when
// every lane of the warp has finished its walk.  Matches are appended with one atomic per warp
// and step.
template <bool kWide>
__device__ __forceinline__ void probe_walk_all(const void* __restrict__ slots_v, uint32_t cap, bool dups,
                                               const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                               const uint32_t* __restrict__ sel, int64_t n,
                                               uint32_t* __restrict__ out_probe, uint32_t* __restrict__ out_build,
                                               int64_t out_cap, unsigned long long* __restrict__ counter) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); w * 32 < n; w += warps) {
    const int64_t i = w * 32 + lane;
    bool walking = i < n;
    uint32_t row = 0, s = 0;
    uint64_t key = 0;
    if (walking) {
      row = sel ? sel[i] : (uint32_t)i;
      key = kWide ? pack_key64(hi[row], lo[row]) : (uint64_t)(uint32_t)lo[row];
      s = kWide ? home_slot64(key, cap) : home_slot32((uint32_t)key, cap);
    }
    uint32_t steps = 0;
    while (__any_sync(0xffffffffu, walking)) {
      bool match = false;
      uint32_t payload = kEmpty32;
      if (walking) {
        uint64_t skey;
        if (kWide) {
          const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(slots_v) + s);
          skey = v.x;
          payload = (uint32_t)v.y;
        } else {
          const uint64_t v = __ldg(reinterpret_cast<const uint64_t*>(slots_v) + s);
          skey = (uint32_t)v;
          payload = (uint32_t)(v >> 32);
        }
        if (payload == kEmpty32 || ++steps > cap) {
          walking = false;
        } else {
          match = skey == key;
          if (match && !dups) walking = false;
          s = (s + 1 == cap) ? 0 : s + 1;
        }
      }
      const uint64_t pos = warp_append(counter, match);
      if (match && (int64_t)pos < out_cap) {
        out_probe[pos] = row;
        out_build[pos] = payload;
      }
    }
  }
}

// Appends this lane's `cnt` pairs (probe rows row[r], build rows pay[r] for the bits of `found`)
// at consecutive positions: one atomic per warp.  Every lane of the warp calls it.
__device__ __forceinline__ void append_pairs(unsigned long long* counter, uint32_t found, const uint32_t (&row)[4],
                                             const uint32_t (&pay)[4], uint32_t* out_probe, uint32_t* out_build,
                                             int64_t out_cap) {
  const int lane = threadIdx.x & 31;
  const uint32_t cnt = __popc(found);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 0 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 0);
  int64_t pos = (int64_t)(base + incl - cnt);
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if ((found >> r) & 1u) {
      if (pos < out_cap) {
        out_probe[pos] = row[r];
        out_build[pos] = pay[r];
      }
      ++pos;
    }
}

// The probe rows of quad q (rows 4q .. 4q+3 of the probe sequence, those below n): their row
// ids (through the selection vector when there is one; a 16-byte load when it allows) and keys.
template <bool kWide>
__device__ __forceinline__ uint32_t probe_quad_rows(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    const uint32_t* __restrict__ sel, int64_t n, int64_t q,
                                                    uint32_t (&row)[4], uint64_t (&key)[4]) {
  const int64_t i0 = q << 2;
  uint32_t bits = 0;
  if (sel && i0 + 3 < n && ((uintptr_t)sel & 15) == 0) {
    const uint4 s4 = __ldcs(reinterpret_cast<const uint4*>(sel) + q);
    row[0] = s4.x, row[1] = s4.y, row[2] = s4.z, row[3] = s4.w;
    bits = 15u;
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool in = i0 + r < n;
      row[r] = in ? (sel ? sel[i0 + r] : (uint32_t)(i0 + r)) : 0u;
      bits |= (uint32_t)in << r;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
    key[r] = ((bits >> r) & 1u) ? (kWide ? pack_key64(hi[row[r]], lo[row[r]]) : (uint64_t)(uint32_t)lo[row[r]]) : 0;
  return bits;
}

// Probe (no duplicate keys in the table): four probe rows per thread, every home bucket (32 bytes:
// four narrow or two wide slots) requested before any is examined; a walk continues only past a
// full bucket.  A table with duplicate keys takes probe_walk_all.
template <bool kWide>
__global__ void __launch_bounds__(kThreads, 4)
join_probe_kernel(const void* __restrict__ slots_v, uint32_t cap, const JoinHeader* __restrict__ hdr,
                  const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                  const uint32_t* __restrict__ sel, int64_t n, uint32_t* __restrict__ out_probe,
                  uint32_t* __restrict__ out_build, int64_t out_cap,
                  unsigned long long* __restrict__ counter) {
  if (hdr->has_dups) {
    probe_walk_all<kWide>(slots_v, cap, true, lo, hi, sel, n, out_probe, out_build, out_cap, counter);
    return;
  }
  ProbeArgs a{};
  a.jslots = slots_v;
  a.jcap = cap;
  Lookup L{};  // hash table, no duplicates, no Bloom filter
  const int64_t nq = (n + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of rounds (append_pairs is warp-wide)
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31);
  for (int64_t q0 = first; q0 < nq; q0 += stride) {
    const int64_t q = q0 + (threadIdx.x & 31);
    uint32_t row[4], pay[4] = {kEmpty32, kEmpty32, kEmpty32, kEmpty32};
    uint64_t key[4];
    const uint32_t bits = q < nq ? probe_quad_rows<kWide>(lo, hi, sel, n, q, row, key) : 0u;
    const int64_t zero[4] = {0, 0, 0, 0};
    if (bits) probe_rows_emit<kWide, false>(a, L, bits, key, zero, [&](int r, uint32_t p, int64_t) { pay[r] = p; });
    uint32_t found = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) found |= (uint32_t)(pay[r] != kEmpty32) << r;
    append_pairs(counter, found, row, pay, out_probe, out_build, out_cap);
  }
}

// Warp-cooperative probe (no duplicate keys): four lanes per probe key, each reading one of
// four consecutive buckets of the key's probe sequence (16 narrow or 8 wide slots per step, a
// 128-byte span); the first slot in probe order that is empty or holds the key decides.
template <bool kWide>
__global__ void __launch_bounds__(kThreads, 4)
join_probe_coop_kernel(const void* __restrict__ slots_v, uint32_t cap, const JoinHeader* __restrict__ hdr,
                       const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                       const uint32_t* __restrict__ sel, int64_t n, uint32_t* __restrict__ out_probe,
                       uint32_t* __restrict__ out_build, int64_t out_cap,
                       unsigned long long* __restrict__ counter) {
  if (hdr->has_dups) {
    probe_walk_all<kWide>(slots_v, cap, true, lo, hi, sel, n, out_probe, out_build, out_cap, counter);
    return;
  }
  constexpr int kPer = kWide ? 2 : 4;  // slots per bucket
  const uint32_t nb = cap / kPer;      // buckets
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, j = lane & 3;          // key group of four lanes, bucket offset
  const unsigned gmask = 0xFu << (g * 4);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x / 4;  // keys per grid round
  const int64_t first = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) / 4;
  for (int64_t k0 = first; k0 < n; k0 += stride) {
    const int64_t i = k0 + g;                     // this group's probe row index
    const bool in = i < n;
    uint32_t row = 0;
    uint64_t key = 0;
    if (in) {
      row = sel ? sel[i] : (uint32_t)i;
      key = kWide ? pack_key64(hi[row], lo[row]) : (uint64_t)(uint32_t)lo[row];
    }
    uint32_t b = in ? (kWide ? home_slot64(key, cap) : home_slot32((uint32_t)key, cap)) / kPer : 0u;
    bool done = !in;
    uint32_t pay = kEmpty32;
    for (uint32_t step = 0; step < nb; step += 4) {
      if (!__any_sync(0xffffffffu, !done)) break;
      // this lane's bucket: the first slot in it that is empty or holds the key
      int ev = kPer;        // slot index of the event, kPer = none
      bool hit = false;
      uint32_t p = kEmpty32;
      if (!done) {
        uint32_t bb = b + j;
        if (bb >= nb) bb -= nb;
        uint64_t w[4];
        load_bucket<kWide>(slots_v, bb * kPer, w);
#pragma unroll
        for (int t = kPer - 1; t >= 0; --t) {
          const uint64_t sk = kWide ? w[2 * t] : (uint64_t)(uint32_t)w[t];
          const uint32_t sp = kWide ? (uint32_t)w[2 * t + 1] : (uint32_t)(w[t] >> 32);
          if (sp == kEmpty32 || sk == key) {
            ev = t;
            hit = sp != kEmpty32;
            p = sp;
          }
        }
      }
      // the lowest lane of the group with an event decides for the key
      const unsigned evm = __ballot_sync(0xffffffffu, ev < kPer) & gmask;
      if (!done && evm) {
        const int src = __ffs(evm) - 1;
        const bool h = __shfl_sync(gmask, (int)hit, src) != 0;
        const uint32_t sp = __shfl_sync(gmask, p, src);
        if (h) pay = sp;
        done = true;
      } else if (!done) {
        b += 4;
        if (b >= nb) b -= nb;
      }
    }
    // lane 0 of each group appends its key's pair
    uint32_t rows4[4] = {row, 0, 0, 0}, pays4[4] = {pay, 0, 0, 0};
    append_pairs(counter, (j == 0 && pay != kEmpty32) ? 1u : 0u, rows4, pays4, out_probe, out_build, out_cap);
  }
}

// dst[i] = src[idx[i]]: four rows per thread (a 16-byte index load when the indexes are 16-byte
// aligned), the four source reads in flight together.
// Four consecutive outputs: 16-byte stores when the destination allows, so that a warp's
// stores fill whole sectors.
__device__ __forceinline__ void store4(int32_t* p, const int32_t (&x)[4], bool vec) {
  if (vec) __stcs(reinterpret_cast<int4*>(p), make_int4(x[0], x[1], x[2], x[3]));
  else
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = x[k];
}
__device__ __forceinline__ void store4(int64_t* p, const int64_t (&x)[4], bool vec) {
  if (vec) {
    __stcs(reinterpret_cast<longlong2*>(p), make_longlong2(x[0], x[1]));
    __stcs(reinterpret_cast<longlong2*>(p) + 1, make_longlong2(x[2], x[3]));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = x[k];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
gather_kernel(const T* __restrict__ src, const uint32_t* __restrict__ idx, int64_t n, T* __restrict__ dst) {
  const int64_t nq = n >> 2;
  const bool vec = ((uintptr_t)idx & 15) == 0;
  const bool vec_out = ((uintptr_t)dst & 15) == 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t r[4];
    if (vec) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(idx) + q);
      r[0] = v.x, r[1] = v.y, r[2] = v.z, r[3] = v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = idx[4 * q + k];
    }
    T x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = src[r[k]];
    store4(dst + 4 * q, x, vec_out);
  }
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < n - (nq << 2)) {
    const int64_t i = (nq << 2) + threadIdx.x;
    dst[i] = src[idx[i]];
  }
}

__global__ void __launch_bounds__(kThreads)
gather_group_key_kernel(const int32_t* __restrict__ grp, const int8_t* __restrict__ flag,
                        const uint32_t* __restrict__ idx, int64_t n, int64_t* __restrict__ dst) {
  const int64_t nq = n >> 2;
  const bool vec = ((uintptr_t)idx & 15) == 0;
  const bool vec_out = ((uintptr_t)dst & 15) == 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t r[4];
    if (vec) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(idx) + q);
      r[0] = v.x, r[1] = v.y, r[2] = v.z, r[3] = v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = idx[4 * q + k];
    }
    int64_t x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = group_key(grp[r[k]], flag, r[k]);
    store4(dst + 4 * q, x, vec_out);
  }
  if (blockIdx.x == 0 && (int64_t)threadIdx.x < n - (nq << 2)) {
    const int64_t i = (nq << 2) + threadIdx.x;
    const uint32_t r = idx[i];
    dst[i] = group_key(grp[r], flag, r);
  }
}

}  // namespace

int grid_for(int64_t n, int threads) {
  const int64_t want = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

sirius_status join_build(const int32_t* lo, const int32_t* hi, int64_t m, void* mem, int64_t capacity,
                         cudaStream_t s, bool clear) {
  JoinHeader* hdr = (JoinHeader*)mem;
  void* slots = (char*)mem + 256;
  const size_t slot_bytes = hi ? 16 : 8;
  if (clear) SIRIUS_CUDA_TRY(cudaMemsetAsync(mem, 0, 256, s));
  if (clear) SIRIUS_CUDA_TRY(cudaMemsetAsync(slots, 0xFF, (size_t)capacity * slot_bytes, s));
  if (m == 0) return SIRIUS_OK;
  const int g = grid_for(m, kThreads);
  PhaseTimer pt(s, SIRIUS_PHASE_JOIN_BUILD);
  if (hi)
    join_build64_kernel<<<g, kThreads, 0, s>>>(lo, hi, m, (ulonglong2*)slots, (uint32_t)capacity, hdr);
  else
    join_build32_kernel<<<g, kThreads, 0, s>>>(lo, m, (uint64_t*)slots, (uint32_t)capacity, hdr);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

}  // namespace sirius

using namespace sirius;

extern "C" int64_t sirius_join_table_capacity(int64_t m, double load_factor) {
  if (m < 0) return 0;
  if (!(load_factor > 0.0) || load_factor > 0.95) load_factor = 0.5;
  int64_t c = (int64_t)((double)m / load_factor) + 1;
  if (c <= m) c = m + 1;
  if (c < 16) c = 16;
  return (c + 3) & ~(int64_t)3;  // whole 32-byte buckets
}

extern "C" size_t sirius_join_table_bytes(int64_t capacity, int32_t key_width) {
  if (capacity <= 0 || (key_width != 4 && key_width != 8)) return 0;
  return 256 + (size_t)capacity * (key_width == 8 ? 16 : 8);
}

extern "C" sirius_status sirius_hash_join_build(const int32_t* d_keys, const int32_t* d_keys_hi,
                                                int64_t m, sirius_join_table* table,
                                                int32_t* h_has_dups, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(table && table->d_mem, "join build: NULL table");
  SIRIUS_REQUIRE(table->key_width == (d_keys_hi ? 8 : 4),
                 "join build: key_width %d does not match the key columns", table->key_width);
  SIRIUS_REQUIRE(m >= 0 && m <= kMaxRows && m < table->capacity && table->capacity < (1ll << 32),
                 "join build: m=%lld needs capacity > m (< 2^32), have %lld", (long long)m,
                 (long long)table->capacity);
  SIRIUS_REQUIRE(table->capacity % 4 == 0, "join build: capacity must be a multiple of 4");
  SIRIUS_REQUIRE(m == 0 || d_keys, "join build: NULL keys");
  SIRIUS_REQUIRE(((uintptr_t)table->d_mem & 255) == 0, "join build: table memory must be 256-byte aligned");
  sirius_status st = join_build(d_keys, d_keys_hi, m, table->d_mem, table->capacity, s, true);
  if (st != SIRIUS_OK) return st;
  if (h_has_dups) {
    JoinHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, table->d_mem, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_has_dups = h.has_dups ? 1 : 0;
    if (h.status) {
      set_error("join build: device status %d", h.status);
      return (sirius_status)h.status;
    }
  }
  return SIRIUS_OK;
}

extern "C" sirius_status sirius_hash_join_probe(const sirius_join_table* table, const int32_t* d_keys,
                                                const int32_t* d_keys_hi, const uint32_t* d_sel,
                                                int64_t n, uint32_t* d_out_probe,
                                                uint32_t* d_out_build, int64_t out_cap,
                                                int64_t* d_out_count, int64_t* h_out_count,
                                                sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(table && table->d_mem, "join probe: NULL table");
  SIRIUS_REQUIRE(table->key_width == (d_keys_hi ? 8 : 4), "join probe: key width mismatch");
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "join probe: n=%lld out of range", (long long)n);
  SIRIUS_REQUIRE(out_cap >= 0 && (out_cap == 0 || (d_out_probe && d_out_build)),
                 "join probe: NULL outputs");
  SIRIUS_REQUIRE(n == 0 || d_keys, "join probe: NULL keys");
  SIRIUS_REQUIRE(d_out_count || h_out_count, "join probe: no place for the pair count");
  SIRIUS_REQUIRE(table->probe_variant >= 0 && table->probe_variant <= 2, "join probe: bad probe_variant %d",
                 table->probe_variant);
  // the pair counter lives in the table header's spare word (reset here, stream-ordered)
  JoinHeader* hdr = (JoinHeader*)table->d_mem;
  unsigned long long* counter = (unsigned long long*)&hdr->pairs;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(counter, 0, 8, s));
  if (n > 0) {
    const void* slots = (const char*)table->d_mem + 256;
    const uint32_t cap = (uint32_t)table->capacity;
    // resident blocks (four per SM) loop over the probe rows: four rows per thread, or one key
    // per four lanes (warp-cooperative)
    const bool coop = table->probe_variant == 2;
    const int64_t units = coop ? (n + 7) / 8 * 32 : (n + 3) / 4;
    int64_t g = (units + kThreads - 1) / kThreads;
    const int64_t most = (int64_t)sm_count() * 4;
    g = g < 1 ? 1 : (g > most ? most : g);
    PhaseTimer pt(s, SIRIUS_PHASE_JOIN_PROBE);
    auto k = d_keys_hi ? (coop ? join_probe_coop_kernel<true> : join_probe_kernel<true>)
                       : (coop ? join_probe_coop_kernel<false> : join_probe_kernel<false>);
    k<<<(unsigned)g, kThreads, 0, s>>>(slots, cap, hdr, d_keys, d_keys_hi, d_sel, n, d_out_probe, d_out_build,
                                       out_cap, counter);
    SIRIUS_LAUNCH_CHECK();
  }
  if (d_out_count)
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(d_out_count, counter, 8, cudaMemcpyDeviceToDevice, s));
  if (h_out_count) {
    unsigned long long c = 0;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&c, counter, 8, cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_out_count = (int64_t)c;
    if ((int64_t)c > out_cap) {
      set_error("join probe: %llu pairs exceed out_cap %lld", c, (long long)out_cap);
      return SIRIUS_ERR_CAPACITY;
    }
  }
  return SIRIUS_OK;
}

template <typename T>
static sirius_status gather_any(const T* src, const uint32_t* idx, int64_t n, T* dst, cudaStream_t s) {
  clear_error();
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "gather: n out of range");
  SIRIUS_REQUIRE(n == 0 || (src && idx && dst), "gather: NULL pointer");
  if (n == 0) return SIRIUS_OK;
  PhaseTimer pt(s, SIRIUS_PHASE_GATHER);
  gather_kernel<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(src, idx, n, dst);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

extern "C" sirius_status sirius_gather_i32(const int32_t* d_src, const uint32_t* d_idx, int64_t n,
                                           int32_t* d_dst, sirius_stream stream) {
  return gather_any<int32_t>(d_src, d_idx, n, d_dst, (cudaStream_t)stream);
}

extern "C" sirius_status sirius_gather_i64(const int64_t* d_src, const uint32_t* d_idx, int64_t n,
                                           int64_t* d_dst, sirius_stream stream) {
  return gather_any<int64_t>(d_src, d_idx, n, d_dst, (cudaStream_t)stream);
}

extern "C" sirius_status sirius_gather_group_key(const int32_t* d_grp, const int8_t* d_flag,
                                                 const uint32_t* d_idx, int64_t n, int64_t* d_dst,
                                                 sirius_stream stream) {
  clear_error();
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "gather_group_key: n out of range");
  SIRIUS_REQUIRE(n == 0 || (d_grp && d_idx && d_dst), "gather_group_key: NULL pointer");
  if (n == 0) return SIRIUS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  gather_group_key_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(d_grp, d_flag, d_idx, n, d_dst);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}
