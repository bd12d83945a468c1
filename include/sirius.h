/*
 * sirius.h -- C ABI of the GB300 (sm_103a) relational hot path.
 *
 * The operators are the physical operators of a GPU-native SQL engine's pipeline (Sec. 3.2.2):
 * a predicate filter that yields row ids, an inner hash join (build, probe) that yields row-id
 * pairs, late materialisation of columns by row id (gather), and a hash group-by computing
 * SUM / COUNT / MIN / MAX.  Operators are stateless; the caller (the executor) owns every
 * buffer and pushes columns through them (push-based model, Sec. 3.2.2).  Columns are plain
 * contiguous device arrays without validity bitmaps, passed by pointer as in an Arrow-derived
 * columnar format (Sec. 3.2.3).  sirius_run_pipeline fuses one whole pipeline -- filter, probe,
 * materialisation and aggregation in one pass over the fact table -- after a build over the dim
 * table; sirius_run_pipeline_batch runs many independent pipelines in one set of launches
 * (pipelines as tasks of a global queue, Sec. 3.2.2; batch execution, Sec. 3.4).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are device memory, h_* host memory.  The library never frees caller
 *    memory and keeps no pointer after a call returns (hash tables live in caller memory).
 *  - Every call is ordered on `stream` (a cudaStream_t; NULL is the legacy default stream) and
 *    is asynchronous unless it takes a non-NULL h_* output, in which case it synchronises
 *    `stream` before returning.
 *  - Scratch: calls that need temporary device memory take (d_scratch, scratch_bytes).  Pass a
 *    buffer of at least the size the matching *_scratch_bytes() query returns, 256-byte
 *    aligned; or pass NULL to let the call allocate and free it stream-ordered
 *    (cudaMallocAsync / cudaFreeAsync).  Two calls in flight at once must not share scratch.
 *  - Row ids are uint32: every row count must be below 2^32 - 1 (the paper's engine uses 64-bit
 *    row ids, Sec. 3.2.3; this library narrows them and checks the bound).
 *  - Arithmetic is exact integer arithmetic.  SUM wraps modulo 2^64 if the true sum does not fit
 *    int64 (the caller guarantees it fits).
 *  - Errors: the return value is authoritative.  A call never traps or aborts the device; device
 *    failures are reported through a status word.  sirius_last_error() returns a message for the
 *    last failing call on the calling thread.
 */
#ifndef SIRIUS_H
#define SIRIUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* sirius_stream; /* a cudaStream_t */

typedef enum {
  SIRIUS_OK = 0,
  SIRIUS_ERR_INVALID = 1,    /* bad argument: NULL column, negative or too large size, bad enum */
  SIRIUS_ERR_OOM = 2,        /* the call's own scratch allocation failed */
  SIRIUS_ERR_CAPACITY = 3,   /* an output buffer is too small; the needed size is reported */
  SIRIUS_ERR_TABLE_FULL = 4, /* a hash table ran out of slots; retry with a larger capacity */
  SIRIUS_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (results undefined) */
  SIRIUS_ERR_CUDA = 6,       /* a CUDA runtime call failed; see sirius_last_error() */
  SIRIUS_ERR_SCRATCH = 7     /* scratch buffer smaller than the *_scratch_bytes() query */
} sirius_status;

typedef enum { SIRIUS_LT = 0, SIRIUS_LE = 1, SIRIUS_GT = 2, SIRIUS_GE = 3, SIRIUS_EQ = 4,
               SIRIUS_NE = 5 } sirius_cmp;

enum { SIRIUS_AGG_SUM = 1, SIRIUS_AGG_COUNT = 2, SIRIUS_AGG_MIN = 4, SIRIUS_AGG_MAX = 8,
       SIRIUS_AGG_ALL = 15 };

/* ------------------------------------------------------------------ library */
int32_t sirius_version(void);
const char* sirius_last_error(void);        /* thread-local; "" when the last call succeeded */
uint64_t sirius_launch_count(void);         /* kernels this library has launched (all threads) */
int32_t sirius_device_sm_count(void);       /* SMs of the current device */

/* Phase timing: while enabled, the library records a pair of CUDA events on the launching
 * stream around each of its kernels, by phase.  sirius_profile_start() clears the record and
 * enables it; sirius_profile_stop() waits for the recorded events, writes per phase the summed
 * milliseconds (ms[p]) and launch counts (launches[p]) for p < nphases, disables recording and
 * returns SIRIUS_OK (or SIRIUS_ERR_CUDA).  Not for use inside CUDA graph capture. */
enum { SIRIUS_PHASE_FILTER = 0, SIRIUS_PHASE_JOIN_BUILD = 1, SIRIUS_PHASE_JOIN_PROBE = 2,
       SIRIUS_PHASE_GATHER = 3, SIRIUS_PHASE_GROUPBY = 4, SIRIUS_PHASE_PIPE_INIT = 5,
       SIRIUS_PHASE_PIPE_BUILD = 6, SIRIUS_PHASE_PIPE_PROBE = 7, SIRIUS_PHASE_PIPE_FINALIZE = 8,
       SIRIUS_PHASE_BATCH_GRAPH = 9, SIRIUS_PHASE_BATCH_BUILD = 10, SIRIUS_PHASE_BATCH_PROBE = 11,
       SIRIUS_PHASE_BATCH_FINALIZE = 12, SIRIUS_PHASE_COPY = 13, SIRIUS_PHASE_PIPE_AGGREGATE = 14,
       SIRIUS_PHASE_PIPE_SINGLE = 15, SIRIUS_PHASES = 16 };
void sirius_profile_start(void);
sirius_status sirius_profile_stop(double* ms, int64_t* launches, int32_t nphases);

/* ------------------------------------------------------------------ A2: filter
 * Predicate filter with stream compaction (Sec. 3.2.2: predicate pushdown; Sec. 4.2: filter
 * operator).  Writes the row ids i of d_col[0..n) with `d_col[i] <op> literal`, in ascending
 * order (stable), to d_row_ids (capacity n), and their number to *d_count (device, nullable)
 * and *h_count (host, nullable; synchronises).  One pass: each warp ranks its rows with
 * ballots and popcounts, each tile finds its output offset by a decoupled look-back over the
 * tiles before it.  Scratch: sirius_filter_scratch_bytes(n) (tile status words, zeroed by the
 * call).  Errors: INVALID (NULL pointers with n > 0, n < 0, n >= 2^32 - 1, bad op), SCRATCH,
 * OOM, CUDA, TIMEOUT (a look-back wait exceeded its bound). */
size_t sirius_filter_scratch_bytes(int64_t n);
sirius_status sirius_filter(const int32_t* d_col, int64_t n, int32_t op, int32_t literal,
                            uint32_t* d_row_ids, int64_t* d_count, int64_t* h_count,
                            void* d_scratch, size_t scratch_bytes, sirius_stream stream);

/* Failure injection for tests of callers' error handling (Sec. 3.2.3's buffer manager sizes
 * and acquires the processing region; this exercises the path where that acquisition fails):
 * the next `count` scratch allocations the library itself makes -- calls given d_scratch NULL
 * -- fail with SIRIUS_ERR_OOM and a message, without calling the allocator and before any
 * device work; calls given caller scratch are unaffected.  count 0 cancels pending failures.
 * Process-wide and thread-safe; returns the number of failures still pending before the call.
 * No device memory is touched, so the GPU and every later call stay usable. */
int32_t sirius_inject_alloc_failures(int32_t count);

/* sirius_filter_static: sirius_filter for callers that cannot allocate device memory at all.
 * The paper has no counterpart; it exists for code that must not call cudaMalloc or
 * cudaMallocAsync -- a host callback or another latency-critical path where an allocation
 * could block the device or fail, or a process whose device memory is entirely owned by
 * another allocator -- and so can pass neither scratch nor NULL.  The caller still passes the
 * input column and the outputs (d_row_ids with room for n ids; d_count / h_count as in
 * sirius_filter, same results).  The look-back scratch lives instead in one file-scope device
 * array of the library, sized for at most sirius_filter_static_max_rows() = 2^28 rows (about
 * 64 KB: one word per 32768-row tile); every GPU that loads the library holds that array until the process exits.  Larger
 * n is rejected with SIRIUS_ERR_INVALID and a message.  The call allocates nothing: it clears
 * the part of the array it uses (stream-ordered) before its kernel.  The first call on each
 * device looks up the array's device address (with that device current) and caches it; make
 * that first call before any stream capture.  All calls share the one array, which keeps the
 * last call's contents: two calls that may overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.  The cached address belongs to the device's
 * current context: after cudaDeviceReset (or any teardown of the primary context) it is stale,
 * so a process that resets a device must not call this function on that device again.  A
 * device-side failure (a look-back wait that ran out: SIRIUS_ERR_TIMEOUT) is returned only
 * when h_count is given -- the call then reads the status back; with h_count NULL the call is
 * asynchronous, returns SIRIUS_OK after the launch, and the status stays in the library's
 * array until the next call clears it. */
int64_t sirius_filter_static_max_rows(void);
sirius_status sirius_filter_static(const int32_t* d_col, int64_t n, int32_t op, int32_t literal,
                                   uint32_t* d_row_ids, int64_t* d_count, int64_t* h_count,
                                   sirius_stream stream);

/* ------------------------------------------------------------------ A1 / A3: hash join
 * An open-addressing hash table of the build side (Sec. 3.2.2 join operator; Sec. 4.2: joins
 * dominate).  Keys are one int32 column or a two-column (hi, lo) int32 key compared as one
 * 64-bit value.  Slots hold (key, build row id); linear probing from a hashed home slot;
 * inserts claim an empty slot with one 64-bit (4-byte keys) or 128-bit (two-column keys)
 * compare-and-swap.  Duplicate build keys are kept (a multimap) and detected during the build;
 * a table without duplicates lets probes stop at the first match.
 * The table lives in caller memory: d_mem of sirius_join_table_bytes(capacity, key_width)
 * bytes, 256-byte aligned; capacity from sirius_join_table_capacity(m, load_factor) (> m). */
typedef struct {
  void* d_mem;         /* caller-owned device memory */
  int64_t capacity;    /* slots; must exceed the number of build rows */
  int32_t key_width;   /* 4 or 8 */
  int32_t probe_variant; /* how sirius_hash_join_probe walks the table when it holds no duplicate
                            keys: 0 or 1, four probe rows per thread, each reading its key's
                            32-byte home bucket (all four requested together); 2, warp-cooperative,
                            four lanes per probe key reading four consecutive buckets per step.
                            A table with duplicate keys is walked one row per lane. */
} sirius_join_table;

int64_t sirius_join_table_capacity(int64_t m, double load_factor); /* load_factor in (0, 0.95] */
size_t sirius_join_table_bytes(int64_t capacity, int32_t key_width);

/* Build: inserts rows 0..m-1 of d_keys (low words; d_keys_hi = NULL for 4-byte keys, else the
 * high words) with payload = row id.  Clears the table first.  Errors: INVALID (m >= capacity,
 * key width not matching d_keys_hi, NULL memory), TABLE_FULL (cannot happen when
 * m < capacity; reported defensively), CUDA.  h_has_dups (nullable; synchronises) receives 1
 * if some key occurs twice. */
sirius_status sirius_hash_join_build(const int32_t* d_keys, const int32_t* d_keys_hi, int64_t m,
                                     sirius_join_table* table, int32_t* h_has_dups,
                                     sirius_stream stream);

/* Probe: for each i in [0, n) the probe row r = d_sel ? d_sel[i] : i with key
 * (d_keys_hi[r], d_keys[r]) is matched against the table; every match appends the pair
 * (r, build row id) to (d_out_probe, d_out_build) in unspecified order.  The number of pairs
 * goes to *d_out_count / *h_out_count (synchronises).  When it exceeds out_cap only the first
 * out_cap pairs are written and the call returns CAPACITY (h_out_count holds the size
 * needed; with h_out_count NULL the caller checks *d_out_count > out_cap itself). */
sirius_status sirius_hash_join_probe(const sirius_join_table* table, const int32_t* d_keys,
                                     const int32_t* d_keys_hi, const uint32_t* d_sel, int64_t n,
                                     uint32_t* d_out_probe, uint32_t* d_out_build, int64_t out_cap,
                                     int64_t* d_out_count, int64_t* h_out_count,
                                     sirius_stream stream);

/* ------------------------------------------------------------------ A4: gather
 * Late materialisation (Sec. 3.2.2 materialisation kernel): d_dst[i] = d_src[d_idx[i]].
 * sirius_gather_group_key builds the int64 group key of build rows d_idx[i]: grp, or
 * (grp, flag) packed as grp * 256 + (uint8)flag when d_flag is not NULL. */
sirius_status sirius_gather_i32(const int32_t* d_src, const uint32_t* d_idx, int64_t n,
                                int32_t* d_dst, sirius_stream stream);
sirius_status sirius_gather_i64(const int64_t* d_src, const uint32_t* d_idx, int64_t n,
                                int64_t* d_dst, sirius_stream stream);
sirius_status sirius_gather_group_key(const int32_t* d_grp, const int8_t* d_flag,
                                      const uint32_t* d_idx, int64_t n, int64_t* d_dst,
                                      sirius_stream stream);

/* ------------------------------------------------------------------ A5 / A6: group-by
 * Hash group-by aggregation (Sec. 3.2.2; Sec. 4.2: few groups contend on memory).  Keys are
 * int32 (key_width 4) or int64 (key_width 8); values int64.  For each distinct key: SUM,
 * COUNT(*), MIN, MAX (those selected by `aggs`; COUNT is always computed).  A first pass
 * records the key range; when it spans at most the table's limit of distinct keys (7/8 of its
 * slots), a key's slot is its offset from the smallest key (no hashing; only those slots are
 * cleared and scanned), else keys are hashed.  Small tables are pre-aggregated per thread block
 * in shared memory; large ones aggregate with global atomics, behind a per-block cache of hot
 * groups (direct slots) or after a warp-level combine of equal keys (hashed keys).  With direct
 * slots, MIN or MAX asked for, at least 2^24 rows and at least 256 rows per table slot, the
 * pass is split: the first 1/16 of the rows aggregate in full, then the smallest MAX and the
 * largest MIN over the groups seen (and which groups those were) let the other rows skip the
 * MIN / MAX updates they cannot change (exact).  The table holds sirius_groupby_capacity(hint)
 * slots; more distinct keys than it can take -> TABLE_FULL (retry with a larger hint).
 * Outputs (device, out_cap each, NULL for aggregates not requested): keys, sums, counts, mins,
 * maxs, in unspecified order; the group count G goes to *d_groups / *h_groups
 * (synchronises).  G > out_cap -> CAPACITY with the needed G in *h_groups. */
int64_t sirius_groupby_capacity(int64_t group_cap_hint);
size_t sirius_groupby_scratch_bytes(int64_t group_cap_hint);
sirius_status sirius_groupby_agg(const void* d_keys, int32_t key_width, const int64_t* d_vals,
                                 int64_t n, uint32_t aggs, int64_t group_cap_hint,
                                 int64_t* d_out_keys, int64_t* d_sum, int64_t* d_count,
                                 int64_t* d_min, int64_t* d_max, int64_t out_cap,
                                 int64_t* d_groups, int64_t* h_groups, void* d_scratch,
                                 size_t scratch_bytes, sirius_stream stream);

/* Sort-based group-by (Sec. 4.2 sets hash against sort group-by): the same inputs, aggregates,
 * outputs and errors as sirius_groupby_agg, without a hash table -- the (key, value) pairs are
 * sorted by key (least-significant-digit radix sort, 8-bit digits; a digit that no two keys
 * differ in is skipped), then each run of equal keys is reduced.  Groups come out in ascending
 * key order.  No table limit, so no TABLE_FULL; G > out_cap -> CAPACITY (with h_groups).
 * d_vals needs only 8-byte alignment (16-byte aligned values are fetched by bulk copies).
 * Scratch: sirius_groupby_sort_scratch_bytes(n) (about 32 bytes per row, for either key width).
 * A bounded device wait that runs out gives TIMEOUT through h_groups and -1 in *d_groups. */
size_t sirius_groupby_sort_scratch_bytes(int64_t n);
sirius_status sirius_groupby_sort(const void* d_keys, int32_t key_width, const int64_t* d_vals, int64_t n,
                                  uint32_t aggs, int64_t* d_out_keys, int64_t* d_sum, int64_t* d_count,
                                  int64_t* d_min, int64_t* d_max, int64_t out_cap, int64_t* d_groups,
                                  int64_t* h_groups, void* d_scratch, size_t scratch_bytes, sirius_stream stream);

/* ------------------------------------------------------------------ string keys
 * A string column in the Arrow layout: row i is the bytes d_chars[off[i] .. off[i+1]) with
 * int32 offsets (n + 1 of them, non-decreasing, within [0, n_chars]); strings compare by bytes.
 * Rows whose offsets break that rule are skipped and the call returns INVALID (code -1).
 *
 * Dictionary encoding (Sec. 4.2: group-by on string keys is a measured bottleneck; the library
 * path groups them by sorting): codes[i] = c when row i holds the c-th distinct string in
 * order of first occurrence; d_dict_rows[c] = the first row holding string c (so the rows
 * come out ascending).  Exact: strings are hashed (32 bits) into an open-addressing table of
 * sirius_dict_capacity(distinct_hint) strings, and equal hashes are settled by comparing the
 * bytes.  More distinct strings than that -> TABLE_FULL (retry with a larger hint).
 * distinct_hint <= 2^31.
 * D = the number of distinct strings goes to *d_ndict (-1 after an error) and *h_ndict
 * (synchronises); D > dict_cap -> CAPACITY with D in *h_ndict.
 * flags: 0, or SIRIUS_DICT_WEAK_HASH, for tests: an 8-bit hash, so that many distinct strings
 * share a hash and the byte comparison decides.  Errors: INVALID, TABLE_FULL, CAPACITY,
 * SCRATCH, OOM, CUDA. */
#define SIRIUS_DICT_WEAK_HASH 1u
int64_t sirius_dict_capacity(int64_t distinct_hint);
size_t sirius_dict_scratch_bytes(int64_t n, int64_t distinct_hint);
sirius_status sirius_dict_encode(const int32_t* d_offsets, const uint8_t* d_chars, int64_t n_chars, int64_t n,
                                 int64_t distinct_hint, uint32_t flags, int32_t* d_codes, int64_t* d_dict_rows,
                                 int64_t dict_cap, int64_t* d_ndict, int64_t* h_ndict, void* d_scratch,
                                 size_t scratch_bytes, sirius_stream stream);

/* GROUP BY a string column: per distinct string s, SUM / COUNT(*) / MIN / MAX of d_vals (those
 * in `aggs`; COUNT always), the groups in code order (first occurrence, as sirius_dict_encode
 * numbers them): d_out_rows[c] = the first row holding string c, d_sum[c] ... its aggregates.
 * The strings are dictionary-encoded and, in the same pass, each row's value is aggregated into
 * its string's table slot (COUNT and the selected aggregates); the groups are then listed in code
 * order.  G = D goes to *d_groups / *h_groups (synchronises); G > out_cap -> CAPACITY with G in
 * *h_groups.
 * Scratch: sirius_groupby_string_scratch_bytes(n, distinct_hint).  Errors as sirius_dict_encode. */
size_t sirius_groupby_string_scratch_bytes(int64_t n, int64_t distinct_hint);
sirius_status sirius_groupby_string(const int32_t* d_offsets, const uint8_t* d_chars, int64_t n_chars,
                                    const int64_t* d_vals, int64_t n, int64_t distinct_hint, uint32_t flags,
                                    uint32_t aggs, int64_t* d_out_rows, int64_t* d_sum, int64_t* d_count,
                                    int64_t* d_min, int64_t* d_max, int64_t out_cap, int64_t* d_groups,
                                    int64_t* h_groups, void* d_scratch, size_t scratch_bytes,
                                    sirius_stream stream);

/* ------------------------------------------------------------------ top N groups
 * ORDER BY order DESC|ASC, key ASC LIMIT n_top over a group-by result (Sec. 4.2: top-N ends
 * several of the measured queries): d_out_idx[0 .. min(n_top, g)) receives the positions of the
 * chosen groups in the input arrays, best first; the caller gathers the columns it wants
 * (sirius_gather_i64).  d_keys: the g group keys (unique); d_order: the column ordered by (an
 * aggregate, or the keys themselves).  Ties of the order value go to the smaller key, so the
 * result is unique.  n_top in [1, 8192].  The count min(n_top, g) goes to *d_count (nullable) and
 * *h_count (nullable; synchronises).  Scratch: sirius_topn_scratch_bytes(n_top).  Errors:
 * INVALID, SCRATCH, OOM, CUDA. */
size_t sirius_topn_scratch_bytes(int64_t n_top);
sirius_status sirius_topn_groups(const int64_t* d_keys, const int64_t* d_order, int64_t g, int32_t descending,
                                 int64_t n_top, uint32_t* d_out_idx, int64_t* d_count, int64_t* h_count,
                                 void* d_scratch, size_t scratch_bytes, sirius_stream stream);

/* ------------------------------------------------------------------ A7: fused pipeline
 * SELECT g, SUM(val), COUNT(*), MIN(val), MAX(val) FROM fact JOIN dim ON fk = pk
 * WHERE pred <op> literal GROUP BY g, with g = dim.grp or (dim.grp, dim.flag).
 * Build phase over the dim (pipeline breaker): every dim row's group key is entered into a
 * group table (insert-or-find), and (pk -> group slot) into a join table.  Probe phase: one
 * pass over the fact table evaluates the predicate, probes the join table and aggregates into
 * the group slot directly -- no intermediate row ids are materialised.  Finalize compacts the
 * groups with at least one row.  All columns are caller device memory. */
/* A further dim joined as a filter (a semi-join, for star queries with several dims): a fact
 * row takes part only if its key (fk, fk_hi) equals the key (pk, pk_hi) of some row of this
 * dim that passes attr <op> literal (attr NULL: every row passes).  The dim contributes no
 * column to the result. */
typedef struct {
  const int32_t* fk;        /* fact column, n values: the key into this dim, or its low word */
  const int32_t* fk_hi;     /* NULL, or the high word of a two-column key */
  const int32_t* pk;        /* dim keys, m values, or their low words */
  const int32_t* pk_hi;     /* NULL, or the high words (must match fk_hi being NULL or not) */
  const int32_t* attr;      /* NULL, or the dim column the predicate tests */
  int64_t m;
  int32_t op;               /* sirius_cmp of attr against literal */
  int32_t literal;
} sirius_semijoin;

#define SIRIUS_MAX_SEMIJOINS 3

typedef struct {
  /* fact (probe side), n rows */
  const int32_t* fk;        /* join key, or its low word */
  const int32_t* fk_hi;     /* NULL, or the high word of a two-column key */
  const int32_t* pred;      /* filter column */
  const int64_t* val;       /* aggregated column (fixed-point decimal as int64) */
  int64_t n;
  /* dim (build side), m rows */
  const int32_t* pk;        /* join key, or its low word */
  const int32_t* pk_hi;     /* NULL, or the high word (must match fk_hi being NULL or not) */
  const int32_t* grp;       /* group key column */
  const int8_t* flag;       /* NULL, or a second group key column (key = grp * 256 + (uint8)flag) */
  int64_t m;
  /* query */
  int32_t op;               /* sirius_cmp */
  int32_t literal;
  uint32_t aggs;            /* SIRIUS_AGG_* mask (COUNT is always computed) */
  int32_t agg_mode;         /* 0 auto; 1 per-block shared-memory table (group table of at most
                               3510 slots); 2 global reductions; 3 partitioned: the probe pass
                               writes (group slot, value) per joined row, grouped by 4096-slot
                               partition within 4096-row tiles, and a second pass aggregates
                               each partition in shared memory (group table of at most
                               2^19 + 1 slots, group_cap_hint <= 2^18; larger tables use 2);
                               4 global reductions behind a per-block cache of 2048
                               hot groups in shared memory (skewed keys); 5 routed: the group
                               slots are dealt out to the blocks of one cooperative launch,
                               each aggregating its share in shared memory, and every joined
                               row's (slot, value) travels to its owner through an exchange
                               buffer in scratch, one grid-wide barrier per round of rows
                               (group tables up to 256 x 2000 slots; larger tables and star
                               queries use 4; duplicate build keys make the launch use global
                               reductions).  Auto: 1 when it fits, else 4 from 1Mi fact rows,
                               else 2 */
  int64_t group_cap_hint;   /* expected distinct group keys in the dim; 0 -> m */
  float load_factor;        /* join table load factor; 0 -> default 0.5 */
  int32_t block_threads;    /* probe kernel block size; 0 -> default */
  int32_t blocks_per_sm;    /* probe kernel residency target; 0 -> occupancy maximum */
  int32_t probe_variant;    /* 0 auto; 1 direct (each thread loads its rows and buckets);
                               2 staged (TMA column tiles + cp.async bucket gathers, global
                               aggregation, 16-byte aligned columns); 3 single launch
                               (sirius_run_pipeline: every phase -- clearing, key range, build,
                               probe, finalize -- in one cooperative launch of one block per SM,
                               phases separated by grid-wide barriers; not for star queries or
                               partitioned aggregation, which run as 1; other calls take 3 as 1).
                               Auto: 3 when n <= 2^22, m <= 2^20 and neither block_threads nor
                               blocks_per_sm is set, else 1 */
  int32_t join_mode;        /* 0 auto: one-column build keys that are unique and span a range
                               of at most 2m values are joined through a direct-address array
                               (decided on the device during the build); 1 hash table always */
  int32_t split_probe;      /* queries with one-column keys asking for MIN or MAX, aggregated with
                               agg_mode 2 or 4 (not star queries, whose probe keeps one pass):
                               0 auto, 1 one probe pass, 2 split pass -- the
                               first 1/16 of the fact rows aggregate in full, then the smallest
                               MAX and the largest MIN over the groups seen so far (with a bitmap
                               of those among the first 2^17 group slots) let the other rows
                               skip the MIN / MAX reductions they cannot change (direct-address
                               join only; exact).  Auto: 2 when n >= 2^26, n >= 256 x the group
                               slots (sirius_groupby_capacity(group_cap_hint) + 1), dpred is
                               NULL and join_mode is 0; else 1 */
  /* dim-side predicate (predicate transfer, Sec. 3.4): NULL, or a dim column of m values; only
     the dim rows with dpred[j] <dop> dliteral take part in the join (a filter on the build
     side, so the probe pass finds no partner for the other rows' keys) */
  const int32_t* dpred;
  int32_t dop;              /* sirius_cmp */
  int32_t dliteral;
  int32_t bloom;            /* Bloom pre-filter of the probe keys: 0 auto (on when dpred is set),
                               1 off, 2 on.  Built from the keys of the dim rows that take part
                               (16 bits per dim row, three bits in one 64-bit word per key) and
                               tested before each hash-table probe, so most probes of absent keys
                               skip their random bucket read; the direct-address join, itself an
                               exact filter, does not use it */
  int32_t nsemi;            /* further dims joined as filters, 0..SIRIUS_MAX_SEMIJOINS (star query;
                               sirius_run_pipeline only: the batched, resident-index and
                               host-column calls reject them) */
  sirius_semijoin semi[SIRIUS_MAX_SEMIJOINS];
} sirius_pipeline_desc;

typedef struct {
  int64_t* keys;            /* device outputs, out_cap entries each; NULL when not wanted */
  int64_t* sum;
  int64_t* count;
  int64_t* min;
  int64_t* max;
  int64_t out_cap;
  int64_t* d_groups;        /* device: receives G (nullable) */
  int32_t* d_status;        /* device: receives the sirius_status of the device work (nullable) */
  int32_t sync;             /* 1: synchronise and fill `groups` and `status` below */
  int32_t status;           /* host, when sync: device-side status */
  int64_t groups;           /* host, when sync: G */
} sirius_result;

size_t sirius_pipeline_scratch_bytes(const sirius_pipeline_desc* q);
/* Errors: INVALID, SCRATCH, OOM, CUDA; with sync also TABLE_FULL (more distinct group keys in
 * the dim than the group table takes: raise group_cap_hint) and CAPACITY (G > out_cap; the
 * needed G is in result->groups).  Without sync the same codes reach result->d_status. */
sirius_status sirius_run_pipeline(const sirius_pipeline_desc* q, sirius_result* result,
                                  void* d_scratch, size_t scratch_bytes, sirius_stream stream);

/* ------------------------------------------------------------------ resident build side
 * The build phase of sirius_run_pipeline as a call of its own, so that a dim table's join and
 * group tables stay resident in device memory and serve many probe passes (the pre-allocated
 * data caching region, Sec. 3.2.3).  The dim index depends only on the dim fields of `q`
 * (pk, pk_hi, grp, flag, m, dpred / dop / dliteral, bloom, group_cap_hint, load_factor, join_mode).  d_mem: caller device memory of
 * sirius_dim_index_bytes(q) bytes, 256-byte aligned, passed in `bytes`.  The build fills
 * join_capacity, group_capacity, direct_capacity, key_width and bloom_log2.  h_status (nullable) synchronises and receives
 * the device status (TABLE_FULL: more distinct group keys than the hint allows). */
typedef struct {
  void* d_mem;
  size_t bytes;
  int64_t join_capacity;
  int64_t group_capacity;
  int64_t direct_capacity;   /* entries of the direct-address array (0: hash table only) */
  int32_t key_width;
  int32_t bloom_log2;        /* log2 of the Bloom filter's 64-bit words (0: no filter) */
} sirius_dim_index;

size_t sirius_dim_index_bytes(const sirius_pipeline_desc* q);
sirius_status sirius_dim_index_build(const sirius_pipeline_desc* q, sirius_dim_index* idx,
                                     int32_t* h_status, sirius_stream stream);
/* The probe, aggregate and finalize phases against a built dim index: uses the fact and query
 * fields of `q`.  Scratch: sirius_probe_scratch_bytes(q, idx) (the aggregates, plus the tuple
 * buffers of partitioned aggregation).  The dim index is only read, so any number of probes
 * may use it at once, each with its own scratch. */
size_t sirius_probe_scratch_bytes(const sirius_pipeline_desc* q, const sirius_dim_index* idx);
sirius_status sirius_run_probe(const sirius_pipeline_desc* q, const sirius_dim_index* idx,
                               sirius_result* result, void* d_scratch, size_t scratch_bytes,
                               sirius_stream stream);

/* ------------------------------------------------------------------ host-resident columns
 * sirius_run_pipeline for columns in host memory (every column pointer of `q` is host memory,
 * pinned for full copy bandwidth; the result arrays are host memory too).  The dim columns are
 * copied and built first; the fact table then streams through the probe pass in chunks of
 * chunk_rows rows (0 = 16 Mi rows): each column of chunk i+1 is copied on a stream of its own
 * while chunk i is probed (batch execution over host data, Sec. 3.4).  chunk_rows < 0: no
 * staging at all -- the probe pass reads the fact columns in place through the host link
 * (they must be pinned; INVALID otherwise).  The G result rows are copied back; the call
 * synchronises and fills result->groups / result->status.  Scratch:
 * sirius_pipeline_host_scratch_bytes(q, chunk_rows, out_cap). */
size_t sirius_pipeline_host_scratch_bytes(const sirius_pipeline_desc* q, int64_t chunk_rows,
                                          int64_t out_cap);
sirius_status sirius_run_pipeline_host(const sirius_pipeline_desc* q, sirius_result* result,
                                       int64_t chunk_rows, void* d_scratch, size_t scratch_bytes,
                                       sirius_stream stream);

/* ------------------------------------------------------------------ A8: batched pipelines
 * Many independent pipelines in one set of persistent launches: each phase (initialise, build,
 * probe, finalize, publish) is one kernel whose blocks walk the concatenated work units of
 * all queries, so uneven query sizes balance across the GPU and small queries cost no launches
 * of their own (pipelines as tasks of one global queue, Sec. 3.2.2; batch execution, Sec. 3.4).
 * A plan owns the device task table, its pinned staging copy and, once captured, a CUDA graph
 * of the whole batch (copy in, five kernels, copy out) that serves any batch of up to
 * max_queries queries: a replay only rewrites the staging table.
 * indexes (nullable): indexes[i].d_mem != NULL makes query i probe that resident dim index
 * (sirius_dim_index_build) instead of building one; it is only read, so queries may share one.
 * results[i]: device output arrays as for sirius_run_pipeline; with sync != 0 in results[0]
 * the call synchronises and fills every results[i].groups / .status.  The return value is the
 * first failing query's status; per-query statuses are in results[i].status.
 * Tuning: rows_per_unit (0 = 65536) is the probe work unit; queries whose group table fits
 * (<= 3510 slots) aggregate each unit in shared memory.  Scratch:
 * sirius_pipeline_batch_scratch_bytes(qs, nq, indexes); queries' tables live at fixed offsets
 * in it, so two batches in flight need two scratch buffers (and two plans). */
typedef struct sirius_batch_plan_s* sirius_batch_plan;

size_t sirius_pipeline_batch_scratch_bytes(const sirius_pipeline_desc* qs, int32_t nq,
                                           const sirius_dim_index* indexes);
sirius_status sirius_batch_plan_create(int32_t max_queries, sirius_batch_plan* out);
sirius_status sirius_batch_plan_run(sirius_batch_plan plan, const sirius_pipeline_desc* qs,
                                    int32_t nq, const sirius_dim_index* indexes,
                                    sirius_result* results, int64_t rows_per_unit,
                                    int32_t use_graph, void* d_scratch, size_t scratch_bytes,
                                    sirius_stream stream);
void sirius_batch_plan_destroy(sirius_batch_plan plan);
/* One-off form: creates a plan, runs without a graph, destroys the plan. */
sirius_status sirius_run_pipeline_batch(const sirius_pipeline_desc* qs, int32_t nq,
                                        const sirius_dim_index* indexes, sirius_result* results,
                                        void* d_scratch, size_t scratch_bytes,
                                        sirius_stream stream);

/* ------------------------------------------------------------------ self-tests of bounded waits
 * Every wait of a kernel of this library on another block's progress is bounded: when the bound
 * runs out the wait records SIRIUS_ERR_TIMEOUT in device memory and the kernel returns, so a lost
 * arrival never hangs the device.  These two calls (no counterpart in the paper) make such a wait
 * run out on purpose -- the awaited flag is one that nothing sets -- and report the status the
 * device recorded; the context stays usable afterwards.  Both synchronise `stream`.
 *
 * sirius_selftest_lookback_timeout: one warp plays tile 1 of the filter's decoupled look-back
 * (sirius_filter) while tile 0 never publishes; the wait gives up after about half a second.
 * *h_status receives SIRIUS_ERR_TIMEOUT.  d_mem: at least 256 bytes, 256-byte aligned, device
 * memory owned by the caller (overwritten).
 *
 * sirius_selftest_grid_barrier: `blocks` blocks (1 .. SM count, a cooperative launch) pass one
 * grid-wide barrier of the single-launch pipeline (probe_variant 3) waiting for blocks + missing
 * arrivals (missing 0 or 1), each wait bounded by max_spins sleeps of 64 ns (1 .. 2^23).
 * missing = 0: every block passes (*h_status SIRIUS_OK, *h_passed = blocks); missing = 1: every
 * wait runs out (*h_status SIRIUS_ERR_TIMEOUT, *h_passed = 0).  d_mem: at least 256 bytes,
 * 256-byte aligned, device memory owned by the caller (overwritten).  Errors: INVALID for
 * arguments out of range, CUDA on a launch error. */
sirius_status sirius_selftest_lookback_timeout(void* d_mem, size_t bytes, int32_t* h_status,
                                               sirius_stream stream);
sirius_status sirius_selftest_grid_barrier(int32_t blocks, int32_t missing, uint32_t max_spins,
                                           void* d_mem, size_t bytes, int32_t* h_status,
                                           int32_t* h_passed, sirius_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SIRIUS_H */
