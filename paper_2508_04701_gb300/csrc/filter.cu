// A2: predicate filter with stable stream compaction (Sec. 3.2.2 predicate pushdown; Sec. 4.2).
//
// One pass over the column.  A thread block owns a tile of 32768 rows (8 warps x 4096 rows; a
// lane reads thirty-two 16-byte vectors, rows 4*(lane + 32k) .. +3 of its warp's slice, in two
// phases of sixteen loads in flight together).  Each warp counts its selected rows; the block
// scans its 8 warp totals and publishes the tile's count at once; ballots and popcounts rank
// the selected rows, whose offsets in the tile (16-bit) are placed in shared memory in row
// order while warp 0 finds the tile's output offset with a decoupled look-back over the tiles
// before it (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back",
// NVIDIA technical report NVR-2016-002); then the block writes its ids out as one contiguous,
// coalesced run.  Large tiles spread each block's fixed costs (two barriers, the look-back's
// L2 round trip) over 128 KB of input; 8192-row tiles ran at 0.52 of the copy rate, these at
// 0.79 (600M rows, 30 % selected).  The tile is the block index: blocks are dispatched in index
// order, so every tile a look-back waits on has been dispatched; each wait is still bounded and
// reports TIMEOUT.
#include <mutex>

#include "common.cuh"

namespace sirius {
namespace {

constexpr int kFilterThreads = 256;
constexpr int kFilterK = 32;                                 // 16-byte vectors per lane
constexpr int kFilterPhase = 16;                             // vectors per load phase
constexpr int kWarpRows = 32 * 4 * kFilterK;                 // 4096
constexpr int kTileRows = kWarpRows * (kFilterThreads / 32);  // 32768 (offsets fit 16 bits)
static_assert(kTileRows <= 65536, "tile offsets are 16-bit");
constexpr uint64_t kFlagAgg = 1, kFlagPrefix = 2;
// Bound of one look-back wait: 2^21 polls, the later ones 256 ns apart (about half a second).
// A predecessor tile that is running publishes its count within microseconds, so only a
// predecessor that cannot run -- its GPU time-sliced away to another context for longer than the
// bound, or a fault -- turns into SIRIUS_ERR_TIMEOUT; the caller may then simply retry the call.
constexpr int kSpinLimit = 1 << 21;

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Publishes this tile's selected count: as its inclusive prefix for tile 0, else as an
// aggregate that successors can add up before this tile's own prefix is known.
__device__ __forceinline__ void publish_count(uint64_t* status, int64_t tile, uint64_t total) {
  st_relaxed_u64(&status[tile], (total << 2) | (tile == 0 ? kFlagPrefix : kFlagAgg));
}

// Exclusive prefix of this tile (its count already published): the sum of all earlier tiles'
// selected counts.  Run by one whole warp, which reads the status words of the 32 tiles before
// the current position and adds their counts back to the nearest published inclusive prefix
// (only the words nearer than that prefix need to be ready); returns the same value in every
// lane.
__device__ uint64_t look_back_published(uint64_t* status, int64_t tile, uint64_t total, int32_t* err) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t j0 = tile - 1;
  bool timed_out = false;
  while (true) {
    const int64_t j = j0 - lane;
    uint64_t w = 0;
    int spins = 0;
    while (true) {
      w = (j >= 0) ? ld_relaxed_u64(&status[j]) : kFlagPrefix;
      // done when every word nearer than the nearest published prefix is ready
      const unsigned nr = __ballot_sync(0xffffffffu, (w & 3) == 0);
      const unsigned pr = __ballot_sync(0xffffffffu, (w & 3) == kFlagPrefix);
      if (nr == 0 || (pr != 0 && (pr & (0u - pr)) < (nr & (0u - nr)))) break;
      if (++spins > kSpinLimit) {
        timed_out = true;
        break;
      }
      if (spins > 64) __nanosleep(256);
    }
    if (timed_out) break;
    const unsigned pm = __ballot_sync(0xffffffffu, (w & 3) == kFlagPrefix);
    const int stop = pm ? __ffs(pm) - 1 : 31;
    excl += warp_sum_u64(lane <= stop ? (w >> 2) : 0);
    if (pm) break;
    j0 -= 32;
  }
  if (timed_out && lane == 0) set_status(err, SIRIUS_ERR_TIMEOUT);
  if (lane == 0) st_relaxed_u64(&status[tile], ((excl + total) << 2) | kFlagPrefix);
  return excl;
}

__device__ uint64_t look_back(uint64_t* status, int64_t tile, uint64_t total, int32_t* err) {
  if ((threadIdx.x & 31) == 0) publish_count(status, tile, total);
  return look_back_published(status, tile, total, err);
}

// Self-test of the look-back's bounded wait: one warp plays tile 1, whose predecessor (tile 0)
// never publishes, so the wait runs out and records SIRIUS_ERR_TIMEOUT in *err.
__global__ void lookback_selftest_kernel(uint64_t* status, int32_t* err) { look_back(status, 1, 7, err); }

// Three blocks per SM (64 KB of shared memory and up to 85 registers each).
template <bool kVec>
__global__ void __launch_bounds__(kFilterThreads, 3)
filter_compact_kernel(const int32_t* __restrict__ col, int64_t n, int op, int32_t lit,
                      uint32_t* __restrict__ out, int64_t* __restrict__ d_count,
                      DevHeader* hdr, uint64_t* status, int64_t num_tiles) {
  __shared__ uint32_t s_warp_total[kFilterThreads / 32];
  __shared__ uint32_t s_warp_excl[kFilterThreads / 32];
  __shared__ uint32_t s_total;
  __shared__ uint64_t s_tile_excl;
  extern __shared__ uint16_t s_ids[];   // [kTileRows] the tile's selected rows (offsets in the tile), in row order

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t tile = blockIdx.x;
  const int64_t warp_row0 = tile * kTileRows + (int64_t)warp * kWarpRows;

  // ---- load + evaluate: bits of vector k of this lane at 4k .. 4k+3 (two phases of loads)
  uint32_t bits[kFilterK / 8] = {};  // vector k at bits[k / 8], bits 4 (k % 8) .. +3
  const bool full_tile = (tile + 1) * (int64_t)kTileRows <= n;
  if (kVec && full_tile) {
    const int4* p = reinterpret_cast<const int4*>(col + warp_row0);
#pragma unroll
    for (int h = 0; h < kFilterK; h += kFilterPhase) {
      int4 v[kFilterPhase];
#pragma unroll
      for (int k = 0; k < kFilterPhase; ++k) v[k] = __ldcs(p + lane + 32 * (h + k));
#pragma unroll
      for (int k = 0; k < kFilterPhase; ++k)
        bits[(h + k) / 8] |= ((uint32_t)cmp_op(v[k].x, lit, op) | ((uint32_t)cmp_op(v[k].y, lit, op) << 1) |
                              ((uint32_t)cmp_op(v[k].z, lit, op) << 2) | ((uint32_t)cmp_op(v[k].w, lit, op) << 3))
                             << (4 * ((h + k) % 8));
    }
  } else {
#pragma unroll
    for (int k = 0; k < kFilterK; ++k) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t r = warp_row0 + 4 * (lane + 32 * k) + j;
        if (r < n && cmp_op(col[r], lit, op)) bits[k / 8] |= 1u << (4 * (k % 8) + j);
      }
    }
  }

  // ---- warp total of selected rows
  const unsigned lt = lanemask_lt();
  uint32_t running = 0;
#pragma unroll
  for (int i = 0; i < kFilterK / 8; ++i) running += __popc(bits[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) running += __shfl_xor_sync(0xffffffffu, running, o);
  if (lane == 0) s_warp_total[warp] = running;
  __syncthreads();

  // ---- block scan of warp totals; the tile's count is published at once
  if (warp == 0) {
    const uint32_t v = lane < kFilterThreads / 32 ? s_warp_total[lane] : 0;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane < kFilterThreads / 32) s_warp_excl[lane] = incl - v;
    if (lane == 31) {
      s_total = incl;
      publish_count(status, tile, incl);
    }
  }
  __syncthreads();

  // ---- the selected row ids into shared memory in row order (tile-local positions): per
  // vector k the ballots rank this lane's rows among the warp's
  uint32_t pos = s_warp_excl[warp];
#pragma unroll
  for (int k = 0; k < kFilterK; ++k) {
    const uint32_t b = (bits[k / 8] >> (4 * (k % 8))) & 15u;
    const uint32_t off0 = (uint32_t)(warp * kWarpRows + 4 * (lane + 32 * k));
    uint32_t m[4], below = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m[j] = __ballot_sync(0xffffffffu, (b >> j) & 1u);
      below += __popc(m[j] & lt);
      tot += __popc(m[j]);
    }
    uint32_t q = pos + below;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((b >> j) & 1u) s_ids[q++] = (uint16_t)(off0 + j);
    pos += tot;
  }
  // ---- the tile's output offset (warp 0)
  const uint32_t total = s_total;
  if (warp == 0) {
    const uint64_t excl = look_back_published(status, tile, total, &hdr->status);
    if (lane == 0) {
      s_tile_excl = excl;
      if (tile == num_tiles - 1) {
        hdr->count = excl + total;
        if (d_count) *d_count = (int64_t)(excl + total);
      }
    }
  }
  __syncthreads();

  // ---- one contiguous run of ids out
  uint32_t* dst = out + s_tile_excl;
  const uint32_t tile_row0 = (uint32_t)(tile * kTileRows);
  for (uint32_t i = threadIdx.x; i < total; i += kFilterThreads) dst[i] = tile_row0 + s_ids[i];
}

}  // namespace

size_t filter_scratch_bytes(int64_t n) {
  const int64_t tiles = n > 0 ? (n + kTileRows - 1) / kTileRows : 0;
  return 256 + align_up((size_t)tiles * 8, 256);
}

sirius_status filter_launch(const int32_t* d_col, int64_t n, int32_t op, int32_t literal,
                            uint32_t* d_row_ids, int64_t* d_count, DevHeader* hdr,
                            uint64_t* status, cudaStream_t s) {
  const int64_t tiles = (n + kTileRows - 1) / kTileRows;
  SIRIUS_CUDA_TRY(cudaMemsetAsync(hdr, 0, 256 + (size_t)tiles * 8, s));
  const bool vec = ((uintptr_t)d_col & 15) == 0;
  PhaseTimer pt(s, SIRIUS_PHASE_FILTER);
  static std::atomic<uint64_t> smem_set[2] = {};  // per kernel: devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(filter_compact_kernel<true>, kTileRows * 2, smem_set[0]));
  SIRIUS_CUDA_TRY(ensure_smem_limit(filter_compact_kernel<false>, kTileRows * 2, smem_set[1]));
  if (vec)
    filter_compact_kernel<true><<<(unsigned)tiles, kFilterThreads, kTileRows * 2, s>>>(
        d_col, n, op, literal, d_row_ids, d_count, hdr, status, tiles);
  else
    filter_compact_kernel<false><<<(unsigned)tiles, kFilterThreads, kTileRows * 2, s>>>(
        d_col, n, op, literal, d_row_ids, d_count, hdr, status, tiles);
  SIRIUS_LAUNCH_CHECK();
  return SIRIUS_OK;
}

}  // namespace sirius

using namespace sirius;

extern "C" size_t sirius_filter_scratch_bytes(int64_t n) { return filter_scratch_bytes(n); }

extern "C" sirius_status sirius_filter(const int32_t* d_col, int64_t n, int32_t op,
                                       int32_t literal, uint32_t* d_row_ids, int64_t* d_count,
                                       int64_t* h_count, void* d_scratch, size_t scratch_bytes,
                                       sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(n >= 0 && n <= kMaxRows, "filter: n=%lld out of range", (long long)n);
  SIRIUS_REQUIRE(op >= SIRIUS_LT && op <= SIRIUS_NE, "filter: bad comparison %d", op);
  SIRIUS_REQUIRE(n == 0 || (d_col && d_row_ids), "filter: NULL column or output");
  if (n == 0) {
    if (d_count) SIRIUS_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
    if (h_count) *h_count = 0;
    return SIRIUS_OK;
  }
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, filter_scratch_bytes(n), s);
  if (st != SIRIUS_OK) return st;
  DevHeader* hdr = (DevHeader*)sc.take(256);
  uint64_t* status = (uint64_t*)(sc.base + 256);
  st = filter_launch(d_col, n, op, literal, d_row_ids, d_count, hdr, status, s);
  if (st != SIRIUS_OK) return st;
  if (h_count) {
    DevHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_count = (int64_t)h.count;
    if (h.status != 0) {
      set_error("filter: device status %d", h.status);
      return (sirius_status)h.status;
    }
  }
  return SIRIUS_OK;
}

// ------------------------------------------------------------------ filter without allocation
// sirius_filter_static: the same filter for callers that cannot allocate device memory at
// all -- code running where cudaMalloc / cudaMallocAsync are unavailable or must not be called
// (a host callback or another latency-critical path where an allocation could block the
// device or fail, or a process whose device memory is entirely owned by another allocator and
// that passes only its own inputs and outputs).  Its look-back scratch (the 256-byte header and
// one status word per 32768-row tile) lives in the file-scope device array below, which every
// GPU that loads this library holds until the process exits.
namespace {
constexpr int64_t kStaticFilterMaxRows = 1ll << 28;  // 268 435 456 rows
constexpr int64_t kStaticFilterMaxTiles = (kStaticFilterMaxRows + kTileRows - 1) / kTileRows;
static __device__ __align__(256) uint64_t g_filter_static_scratch[32 + kStaticFilterMaxTiles];

std::mutex g_static_mu;
void* g_static_addr[64] = {};  // device address of the array, per device ordinal

// Host code cannot use the array's name as a device address; look the address up once per
// device, with that device current.
sirius_status static_scratch_addr(void** out) {
  int dev = 0;
  SIRIUS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("filter_static: device ordinal %d beyond 63", dev);
    return SIRIUS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_filter_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("filter_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return SIRIUS_ERR_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return SIRIUS_OK;
}
}  // namespace

extern "C" int64_t sirius_filter_static_max_rows(void) { return kStaticFilterMaxRows; }

extern "C" sirius_status sirius_filter_static(const int32_t* d_col, int64_t n, int32_t op, int32_t literal,
                                              uint32_t* d_row_ids, int64_t* d_count, int64_t* h_count,
                                              sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(n >= 0 && n <= kStaticFilterMaxRows,
                 "filter_static: n=%lld exceeds the static scratch limit of %lld rows (use sirius_filter)",
                 (long long)n, (long long)kStaticFilterMaxRows);
  SIRIUS_REQUIRE(op >= SIRIUS_LT && op <= SIRIUS_NE, "filter_static: bad comparison %d", op);
  SIRIUS_REQUIRE(n == 0 || (d_col && d_row_ids), "filter_static: NULL column or output");
  if (n == 0) {
    if (d_count) SIRIUS_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
    if (h_count) *h_count = 0;
    return SIRIUS_OK;
  }
  void* base = nullptr;
  sirius_status st = static_scratch_addr(&base);
  if (st != SIRIUS_OK) return st;
  DevHeader* hdr = (DevHeader*)base;
  uint64_t* status = (uint64_t*)((char*)base + 256);
  // filter_launch clears the header and the status words this call uses before its kernel
  st = filter_launch(d_col, n, op, literal, d_row_ids, d_count, hdr, status, s);
  if (st != SIRIUS_OK) return st;
  if (h_count) {
    DevHeader h;
    SIRIUS_CUDA_TRY(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_count = (int64_t)h.count;
    if (h.status != 0) {
      set_error("filter_static: device status %d", h.status);
      return (sirius_status)h.status;
    }
  }
  return SIRIUS_OK;
}

// ------------------------------------------------------------------ self-test of the look-back wait
extern "C" sirius_status sirius_selftest_lookback_timeout(void* d_mem, size_t bytes, int32_t* h_status,
                                                         sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(d_mem && bytes >= 256 && ((uintptr_t)d_mem & 255) == 0,
                 "selftest: need 256 bytes of 256-byte aligned device memory");
  SIRIUS_REQUIRE(h_status, "selftest: NULL host result");
  int32_t* err = (int32_t*)d_mem;
  uint64_t* status = (uint64_t*)((char*)d_mem + 64);  // two tile words, both "not ready"
  SIRIUS_CUDA_TRY(cudaMemsetAsync(d_mem, 0, 256, s));
  lookback_selftest_kernel<<<1, 32, 0, s>>>(status, err);
  SIRIUS_LAUNCH_CHECK();
  SIRIUS_CUDA_TRY(cudaMemcpyAsync(h_status, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
  return SIRIUS_OK;
}
