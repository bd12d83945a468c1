// Top N groups of a group-by result: ORDER BY <column> [DESC], key LIMIT N (Sec. 4.2 names
// top-N among the operators whose cost follows the data, and TPC-H's join-heavy queries end in
// one).  Each group i has a 128-bit sort word C_i = (its order value mapped to an unsigned
// integer that grows with the wanted order, its key mapped likewise), unique because keys are.
// The N-th smallest word T is found by radix selection, 8 bits per pass from the top (each
// pass histograms the digit of the words that still match the selected prefix; one block
// then picks the digit where the running count reaches the rank left).  The groups with
// C_i <= T -- exactly min(N, G) of them -- are compacted and sorted in one block (bitonic
// sort in shared memory), and their positions written out best first.
#include "tables.cuh"

namespace sirius {
namespace {

constexpr int kTopThreads = 256;
constexpr int kTopPasses = 16;  // 128-bit words, 8 bits per pass
constexpr int64_t kTopMax = 8192;

struct TopState {
  unsigned long long prefix_hi, prefix_lo;  // digits selected so far
  unsigned long long remaining;            // rank still to be found among the matching words
  unsigned long long count;                // compacted words
  unsigned long long pad[28];
};
static_assert(sizeof(TopState) == 256, "top-N state is 256 bytes");

struct Word {
  unsigned long long hi, lo;
  uint32_t idx;
  uint32_t pad;
};

// Order-preserving maps of int64 to uint64 (flip the sign bit); descending order complements.
__device__ __forceinline__ Word word_of(const int64_t* order, const int64_t* keys, int64_t i, bool desc) {
  const unsigned long long u = (unsigned long long)order[i] ^ 0x8000000000000000ull;
  Word w;
  w.hi = desc ? ~u : u;
  w.lo = (unsigned long long)keys[i] ^ 0x8000000000000000ull;
  w.idx = (uint32_t)i;
  w.pad = 0;
  return w;
}

__device__ __forceinline__ bool matches_prefix(const Word& w, const TopState* st, int pass) {
  // words agree with the prefix on the digits of passes 0 .. pass-1 (the top 8 * pass bits)
  const int bits = 8 * pass;
  if (bits == 0) return true;
  if (bits <= 64) {
    const unsigned long long m = bits == 64 ? ~0ull : ~0ull << (64 - bits);
    return (w.hi & m) == (st->prefix_hi & m);
  }
  const int lb = bits - 64;
  const unsigned long long m = lb == 64 ? ~0ull : ~0ull << (64 - lb);
  return w.hi == st->prefix_hi && (w.lo & m) == (st->prefix_lo & m);
}

__device__ __forceinline__ uint32_t digit_of(const Word& w, int pass) {
  return pass < 8 ? (uint32_t)(w.hi >> (56 - 8 * pass)) & 255u : (uint32_t)(w.lo >> (56 - 8 * (pass - 8))) & 255u;
}

__global__ void top_init_kernel(TopState* st, unsigned int* hist, unsigned long long rank) {
  if (threadIdx.x == 0) {
    st->prefix_hi = st->prefix_lo = 0;
    st->remaining = rank;
    st->count = 0;
  }
  hist[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(kTopThreads)
top_hist_kernel(const int64_t* __restrict__ order, const int64_t* __restrict__ keys, int64_t g, int desc,
                const TopState* st, unsigned int* hist, int pass) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
    const Word w = word_of(order, keys, i, desc != 0);
    if (matches_prefix(w, st, pass)) atomicAdd(&h[digit_of(w, pass)], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// One block of 256 threads: the digit whose bin holds the remaining rank; clears the histogram.
__global__ void top_select_kernel(TopState* st, unsigned int* hist, int pass) {
  __shared__ unsigned long long incl[256];
  const unsigned int c = hist[threadIdx.x];
  incl[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {  // inclusive scan (Hillis-Steele)
    const unsigned long long v = threadIdx.x >= (unsigned)o ? incl[threadIdx.x - o] : 0ull;
    __syncthreads();
    incl[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned long long rem = st->remaining;
  const unsigned long long before = incl[threadIdx.x] - c;
  __syncthreads();
  if (c > 0 && before < rem && rem <= incl[threadIdx.x]) {
    st->remaining = rem - before;
    const unsigned long long d = threadIdx.x;
    if (pass < 8) st->prefix_hi |= d << (56 - 8 * pass);
    else st->prefix_lo |= d << (56 - 8 * (pass - 8));
  }
  hist[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(kTopThreads)
top_compact_kernel(const int64_t* __restrict__ order, const int64_t* __restrict__ keys, int64_t g, int desc,
                   TopState* st, Word* out, int64_t cap) {
  const unsigned long long th = st->prefix_hi, tl = st->prefix_lo;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
    const Word w = word_of(order, keys, i, desc != 0);
    if (w.hi < th || (w.hi == th && w.lo <= tl)) {
      const unsigned long long p = atomicAdd(&st->count, 1ull);
      if ((int64_t)p < cap) out[p] = w;
    }
  }
}

__device__ __forceinline__ bool word_less(const Word& a, const Word& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// One block: bitonic sort of the (at most kTopMax) compacted words in shared memory, padded
// to a power of two with words that sort last; positions out best first.
__global__ void __launch_bounds__(1024)
top_sort_kernel(const Word* __restrict__ in, const TopState* st, int64_t n_top, uint32_t* out_idx,
                int64_t* d_count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Word* w = reinterpret_cast<Word*>(smem_raw);
  const int64_t n = (int64_t)st->count < n_top ? (int64_t)st->count : n_top;
  int64_t p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (int64_t i = threadIdx.x; i < p2; i += blockDim.x) {
    if (i < n) w[i] = in[i];
    else w[i] = Word{~0ull, ~0ull, 0xFFFFFFFFu, 0u};
  }
  __syncthreads();
  for (int64_t k = 2; k <= p2; k <<= 1) {
    for (int64_t j = k >> 1; j > 0; j >>= 1) {
      for (int64_t i = threadIdx.x; i < p2; i += blockDim.x) {
        const int64_t l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool swap = up ? word_less(w[l], w[i]) : word_less(w[i], w[l]);
          if (swap) {
            const Word t = w[i];
            w[i] = w[l];
            w[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) out_idx[i] = w[i].idx;
  if (threadIdx.x == 0 && d_count) *d_count = n;
}

size_t top_layout(int64_t n_top, size_t* off_hist, size_t* off_words) {
  *off_hist = 256;
  *off_words = 256 + 256 * 4 + 256;
  return *off_words + (size_t)(n_top > 0 ? n_top : 1) * sizeof(Word);
}

}  // namespace
}  // namespace sirius

using namespace sirius;

extern "C" size_t sirius_topn_scratch_bytes(int64_t n_top) {
  size_t a, b;
  return top_layout(n_top, &a, &b);
}

extern "C" sirius_status sirius_topn_groups(const int64_t* d_keys, const int64_t* d_order, int64_t g,
                                            int32_t descending, int64_t n_top, uint32_t* d_out_idx,
                                            int64_t* d_count, int64_t* h_count, void* d_scratch,
                                            size_t scratch_bytes, sirius_stream stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  SIRIUS_REQUIRE(g >= 0 && g < (int64_t)0xFFFFFFFFll, "topn: g=%lld out of range", (long long)g);
  SIRIUS_REQUIRE(n_top >= 1 && n_top <= kTopMax, "topn: n_top=%lld outside [1, %lld]", (long long)n_top,
                 (long long)kTopMax);
  SIRIUS_REQUIRE(g == 0 || (d_keys && d_order), "topn: NULL input");
  SIRIUS_REQUIRE(d_out_idx, "topn: NULL output");
  size_t off_hist, off_words;
  const size_t need = top_layout(n_top, &off_hist, &off_words);
  Scratch sc;
  sirius_status st = sc.acquire(d_scratch, scratch_bytes, need, s);
  if (st != SIRIUS_OK) return st;
  TopState* state = (TopState*)sc.base;
  unsigned int* hist = (unsigned int*)(sc.base + off_hist);
  Word* words = (Word*)(sc.base + off_words);
  const int64_t rank = g < n_top ? g : n_top;
  if (rank == 0) {
    if (d_count) SIRIUS_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
    if (h_count) *h_count = 0;
    return SIRIUS_OK;
  }
  top_init_kernel<<<1, 256, 0, s>>>(state, hist, (unsigned long long)rank);
  SIRIUS_LAUNCH_CHECK();
  const int grid = grid_for(g, kTopThreads);
  for (int pass = 0; pass < kTopPasses; ++pass) {
    top_hist_kernel<<<grid, kTopThreads, 0, s>>>(d_order, d_keys, g, descending != 0, state, hist, pass);
    SIRIUS_LAUNCH_CHECK();
    top_select_kernel<<<1, 256, 0, s>>>(state, hist, pass);
    SIRIUS_LAUNCH_CHECK();
  }
  top_compact_kernel<<<grid, kTopThreads, 0, s>>>(d_order, d_keys, g, descending != 0, state, words, rank);
  SIRIUS_LAUNCH_CHECK();
  int64_t p2 = 1;
  while (p2 < rank) p2 <<= 1;
  const size_t smem = (size_t)p2 * sizeof(Word);
  static std::atomic<uint64_t> smem_set{0};  // devices with the limit raised
  SIRIUS_CUDA_TRY(ensure_smem_limit(top_sort_kernel, (int)(kTopMax * sizeof(Word)), smem_set));
  top_sort_kernel<<<1, 1024, smem, s>>>(words, state, rank, d_out_idx, d_count);
  SIRIUS_LAUNCH_CHECK();
  if (h_count) {
    SIRIUS_CUDA_TRY(cudaStreamSynchronize(s));
    *h_count = rank;
  }
  return SIRIUS_OK;
}
