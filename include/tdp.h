/*
 * tdp.h -- C ABI of the Tensor Data Platform hot path on B300 (sm_103a).
 *
 * The paper (Sec. 2) stores every table column as a tensor and runs each
 * relational operator as a tensor program on the GPU; Sec. 4 adds
 * differentiable ("soft") versions of filter and grouped aggregation so that
 * a query can be trained end to end, and swaps the exact operators back in at
 * inference.  This header is the boundary of that path: relational filter,
 * group-by aggregation, equi-join, top-k and the radix sort under the
 * group-by; the soft filter / soft aggregation with their adjoints; the
 * probability-encoded (PE) soft group-by and its exact counterpart; and the
 * glyph-CNN layers of the trainable query.
 *
 * Conventions shared by every call
 * ---------------------------------
 *  - Column data, outputs, workspaces, counts and status words are DEVICE
 *    pointers owned by the caller.  Descriptor arrays (tdp_col, tdp_pred,
 *    tdp_agg, index lists, output-pointer lists) are HOST memory, read during
 *    the call only.
 *  - Every call is asynchronous on the given stream.  The library does not
 *    allocate memory and does not synchronise the stream.  Scratch memory is
 *    the caller's workspace `ws` of `ws_bytes` bytes, sized by the matching
 *    tdp_*_workspace() query; a smaller workspace returns
 *    TDP_ERR_WORKSPACE_TOO_SMALL before anything is launched.  Workspaces
 *    start on a 256-byte boundary (as every CUDA allocation does); a
 *    workspace that is not 16-byte aligned returns TDP_ERR_INVALID_ARG.
 *  - The return value reports argument and launch errors found on the host.
 *    Errors found on the device (capacity exceeded, duplicate build key, a
 *    bounded wait that ran out, arithmetic overflow) are OR-ed into the
 *    caller's `int32_t *d_status` word, readable once the stream has reached
 *    that point.  The caller zeroes d_status.
 *  - Output row counts are written to a device int64.  When a result has more
 *    rows than `capacity`, at most `capacity` rows are written, the true count
 *    is still written and TDP_ERR_CAPACITY is set in d_status.
 *  - n < 2^31 rows per column; row ids are int32.
 *  - No call falls back to the CPU.
 */
#ifndef TDP_H
#define TDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st *tdp_stream_t;

typedef enum {
    TDP_OK = 0,
    TDP_ERR_INVALID_ARG = 1,
    TDP_ERR_UNSUPPORTED_DTYPE = 2,
    TDP_ERR_WORKSPACE_TOO_SMALL = 3,
    /* device-side flags (OR-ed into d_status; also returned as codes) */
    TDP_ERR_CAPACITY = 4,
    TDP_ERR_DUP_BUILD_KEY = 8,
    TDP_ERR_TIMEOUT = 16,
    TDP_ERR_OVERFLOW = 32,
    TDP_ERR_CUDA = 64
} tdp_status;

typedef enum { TDP_I8 = 0, TDP_U8 = 1, TDP_I32 = 2, TDP_I64 = 3, TDP_F32 = 4, TDP_BF16 = 5 } tdp_dtype;

typedef enum { TDP_LT = 0, TDP_LE = 1, TDP_GT = 2, TDP_GE = 3, TDP_EQ = 4, TDP_NE = 5 } tdp_cmp;

typedef enum {
    TDP_AGG_COUNT = 0,          /* COUNT(*)                                    */
    TDP_AGG_SUM = 1,            /* SUM(a)                                      */
    TDP_AGG_SUM_MUL_KMINUS = 2, /* SUM(a * (k - b)), e.g. price*(100-discount) */
    TDP_AGG_AVG = 3,            /* AVG(a), rounded half away from zero         */
    TDP_AGG_MIN = 4,
    TDP_AGG_MAX = 5
} tdp_agg_op;

typedef enum {
    TDP_GROUPBY_AUTO = 0,
    TDP_GROUPBY_SORT = 1,
    TDP_GROUPBY_SMALL_DOMAIN = 2,
    TDP_GROUPBY_PARTITION = 3
} tdp_groupby_strategy;

/* Join flags */
#define TDP_JOIN_UNIQUE_BUILD 1u /* build keys must be unique (N:1 join)      */

/*
 * One column: a device array of n elements of `dtype`.  Integer columns may
 * carry metadata bounds lo <= value <= hi (has_bounds != 0), the "encoded
 * tensor" metadata of Sec. 2 that selects an operator strategy: group-by
 * keys with bounds whose domain product is small are aggregated directly
 * (no sort).
 */
typedef struct {
    const void *data;
    int32_t dtype;
    int32_t has_bounds;
    int64_t n;
    int64_t lo;
    int64_t hi;
} tdp_col;

/* Predicate `cols[col] <cmp> lit`; a predicate list is a conjunction. */
typedef struct {
    int32_t col;
    int32_t cmp;
    int64_t lit;
} tdp_pred;

/* Aggregate `op` over column a (and b, k for SUM(a*(k-b))); COUNT ignores a. */
typedef struct {
    int32_t op;
    int32_t a;
    int32_t b;
    int32_t reserved;
    int64_t k;
} tdp_agg;

/* ------------------------------------------------------------------ misc */

/* Human-readable text of a status code (static string, never NULL). */
const char *tdp_status_str(int32_t status);

/* ABI version of this header (major * 100 + minor). */
int32_t tdp_abi_version(void);

/*
 * Upper bound, in polls, of every device-side wait: the decoupled look-back
 * of the probe, sort, reduce-by-key and finalize kernels, the filter's grid
 * barrier, and the mbarrier waits on bulk / TMA copies and tensor-core
 * commits.  A wait that runs out sets TDP_ERR_TIMEOUT and the kernel carries
 * on without hanging; once one wait of a launch has timed out, the other
 * waits of that launch give up at once.  Default 1<<20 (about 0.2 s of
 * polling).  Affects later launches only.  Returns the previous value.
 *
 * This limit is the library's one piece of process-wide mutable state (an
 * atomic read at every launch); every other setting is a call argument.
 */
uint32_t tdp_set_spin_limit(uint32_t polls);

/*
 * Self-test of the bounded wait: one thread waits for `*d_flag` to become
 * non-zero for at most `polls` polls.  If the flag stays zero, TDP_ERR_TIMEOUT
 * is OR-ed into *d_status and the kernel returns.  No counterpart in the
 * paper: it exists so a test can exercise the time-out path without a hang.
 */
tdp_status tdp_debug_wait_flag(const int32_t *d_flag, uint32_t polls, int32_t *d_status,
                               tdp_stream_t stream);

/* ---------------------------------------------------------------- filter */

/* Workspace bytes for tdp_filter over n rows. */
size_t tdp_filter_workspace(int64_t n);

/*
 * Filter with stream compaction: SQL WHERE p_0 AND p_1 AND ... (the filter
 * queries of Sec. 5.1 and the WHERE clause of Sec. 5.2).
 *
 *   cols[ncols]       host array of column descriptors (I8/U8/I32/I64), each
 *                     with at least n elements
 *   preds[npreds]     conjunction of integer comparisons, npreds in 0..8
 *   d_n               optional device int64: only rows 0 .. min(n, *d_n)-1
 *                     are considered (n stays the host-side upper bound)
 *   out_rowid         device int32[capacity]: ids of qualifying rows in
 *                     ascending order (stable), or NULL
 *   d_count           device int64: number of qualifying rows
 *   gather_cols[ngather], gather_out[ngather]
 *                     optional fused gather (ngather in 0..8): gather_out[j]
 *                     receives cols[gather_cols[j]] at the qualifying rows,
 *                     same order and capacity as out_rowid
 *
 * Two phases in one cooperative launch of persistent blocks, each owning a
 * contiguous chunk of rows: (1) the chunk's predicate columns stream through
 * shared-memory tiles filled by bulk copies and each row's result is kept as
 * one bit in shared memory, and the block publishes its count; (2) after one
 * bounded grid-wide barrier each block's output offset is the sum of the
 * counts before it, and the block writes its row ids (and gathered columns)
 * in order.  Tables larger than one round of chunks take several rounds.
 */
tdp_status tdp_filter(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                      int64_t n, const int64_t *d_n, int32_t *out_rowid, int64_t capacity, int64_t *d_count,
                      const int32_t *gather_cols, int32_t ngather, void *const *gather_out,
                      void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/* -------------------------------------------------------------- group-by */

/*
 * Workspace bytes for tdp_groupby_agg.  `n` is the upper bound of input rows,
 * keys/nkeys the key column descriptors (their bounds decide the strategy
 * under AUTO), naggs the number of aggregates.
 */
size_t tdp_groupby_agg_workspace(int64_t n, const tdp_col *keys, int32_t nkeys, int32_t naggs,
                                 int32_t strategy);

/*
 * GROUP BY key columns with aggregates (Sec. 2 "GROUP BY ... COUNT(*)",
 * Sec. 4 trainable GROUP BY, Sec. 5.2 AVG), optionally fused with a filter.
 *
 *   cols[ncols]        all columns referenced below (each >= n elements)
 *   preds[npreds]      optional fused WHERE conjunction (0..8 predicates)
 *   n                  number of input rows when sel == NULL, else the
 *                      capacity of sel
 *   sel, d_nsel        optional device row-id list and its device count: the
 *                      input rows are sel[0 .. *d_nsel) instead of 0..n-1;
 *                      with sel == NULL a non-NULL d_nsel limits the input to
 *                      rows 0 .. min(n, *d_nsel)-1
 *   key_cols[nkeys]    indices into cols of the key columns (1..4, integer)
 *   aggs[naggs]        1..8 aggregates; a, b index cols
 *   strategy           AUTO picks SMALL_DOMAIN when every key column has
 *                      bounds and the dense table of the domain fits in one
 *                      block's shared memory, else PARTITION when every key
 *                      column has bounds and the domain allows it (below),
 *                      else SMALL_DOMAIN when the domain is <= 2^22, else SORT.
 *                      Asking for SMALL_DOMAIN or PARTITION where it does not
 *                      apply returns TDP_ERR_INVALID_ARG.
 *   out_keys[nkeys]    device arrays (dtype of each key column, capacity rows)
 *   out_aggs[naggs]    device int64 arrays (capacity rows)
 *   d_ngroups          device int64: number of groups
 *
 * Groups are written in ascending key order (lexicographic over key_cols).
 * Sums are exact int64; TDP_ERR_OVERFLOW is not detected on the device, so
 * the caller keeps sums within int64 (true for the documented workloads).
 * AVG = (2*sum + sign(sum)*count) / (2*count) with truncating division.
 * SORT: packs the keys into an unsigned radix key (offset by lo when bounds
 * are present), radix-sorts (key, row id) and reduces the sorted runs.
 * SMALL_DOMAIN: one pass that accumulates into private copies of the dense
 * key domain and merges them: per thread (in shared memory, plain adds, no
 * atomics) when the domain times the accumulator slots is at most 63 and
 * the input is not a row-id list, else per warp or per block.
 * PARTITION: bounded keys whose dense domain D fits 16384 buckets of B group
 * ids (B = 4096 with one aggregate slot besides COUNT, smaller with more, so
 * D <= 64M for one sum): rows are counted per bucket, scattered to bucket
 * segments with their aggregate inputs, and each bucket is reduced in a dense
 * shared-memory table and written in ascending key order.  Within a bucket
 * the rows are combined in no fixed order, which does not change exact
 * integer sums, minima or maxima.
 */
tdp_status tdp_groupby_agg(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                           int64_t n, const int32_t *sel, const int64_t *d_nsel,
                           const int32_t *key_cols, int32_t nkeys, const tdp_agg *aggs, int32_t naggs,
                           int32_t strategy, void *const *out_keys, int64_t *const *out_aggs,
                           int64_t capacity, int64_t *d_ngroups, void *ws, size_t ws_bytes,
                           int32_t *d_status, tdp_stream_t stream);

/* ------------------------------------------------------------ radix sort */

/* Workspace bytes for tdp_sort_pairs of n pairs with `key_bits` significant bits. */
size_t tdp_sort_pairs_workspace(int64_t n, int32_t key_bits);

/*
 * Stable LSD radix sort of (uint64 key, uint32 value) pairs by the low
 * `key_bits` bits of the key (1..64; higher bits must be zero), 8-bit digits:
 * one histogram pass over all digits, then one scatter pass per digit whose
 * per-digit offsets come from decoupled look-back ("onesweep").  The sorted
 * pairs are written to keys_out/vals_out (which must not alias the inputs).
 * n counts the pairs (n < 2^30).
 */
tdp_status tdp_sort_pairs(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t key_bits,
                          uint64_t *keys_out, uint32_t *vals_out, void *ws, size_t ws_bytes,
                          int32_t *d_status, tdp_stream_t stream);

/* ------------------------------------------------------------------ join */

/* Smallest power-of-two slot count (>= 8) with load factor <= 1/2 for n keys. */
int64_t tdp_join_default_slots(int64_t n_keys);

/*
 * Build an open-addressing hash table for an inner equi-join on int32 keys
 * (the hash join of Sec. 2's relational operators over key tensors).
 * The table is nslots x 8 bytes of device memory owned by the caller
 * (nslots a power of two >= 8, base 32-byte aligned): nslots slots of one
 * int32 key (low word) and its int32 payload (high word), in buckets of 4
 * slots (32 bytes, one sector, so one load of a bucket gives its keys and
 * their payloads); a multiplicative hash picks a bucket and a full bucket
 * without the key passes the search on to the next one (linear probing over
 * buckets).  An empty slot holds (INT32_MIN, 0), so that key cannot be
 * stored: a build row with key INT32_MIN sets TDP_ERR_OVERFLOW and is
 * dropped, and a probe row with that key finds nothing.  One 64-bit CAS per
 * insert (key and payload together).
 *
 *   cols/preds         build-side columns and an optional fused filter
 *   n, d_n             rows 0..n-1, or 0..min(n, *d_n)-1 when d_n != NULL
 *   key_col            index of the int32 key column
 *   payload_col        index of an int32 column stored as the payload, or -1
 *                      to store the build row id
 *   flags              TDP_JOIN_UNIQUE_BUILD: a repeated key sets
 *                      TDP_ERR_DUP_BUILD_KEY (the second row is dropped)
 *   table              device uint64[nslots]; this call fills it with the
 *                      empty pattern first
 *
 * A full table (no free slot within min(nslots / 4, 8192) buckets) sets
 * TDP_ERR_CAPACITY; a lookup that walks that far sets it too.  Argument
 * errors (nslots not a power of two >= 8, a misaligned table, a key column
 * that is not int32) are returned as TDP_ERR_INVALID_ARG /
 * TDP_ERR_UNSUPPORTED_DTYPE before anything runs.
 */
tdp_status tdp_join_build(const tdp_col *cols, int32_t ncols, const tdp_pred *preds, int32_t npreds,
                          int64_t n, const int64_t *d_n, int32_t key_col, int32_t payload_col, uint32_t flags,
                          uint64_t *table, int64_t nslots, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes for tdp_join_probe over n probe rows. */
size_t tdp_join_probe_workspace(int64_t n);

/*
 * Probe a table built by tdp_join_build (N:1 join, unique build keys).
 * Emits one row per probe row whose key is found, in probe-row order:
 *   out_probe_row[i]   the probe row id (or NULL)
 *   out_payload[i]     the build payload (int32) (or NULL)
 *   gather_out[j][i]   cols[gather_cols[j]] at the probe row (fused gather)
 * Optional fused probe-side filter `preds`; optional probe row list
 * sel / d_nsel as in tdp_groupby_agg (with sel == NULL, d_nsel bounds a dense
 * prefix of the probe rows).  d_count receives the match count.
 */
tdp_status tdp_join_probe(const uint64_t *table, int64_t nslots, const tdp_col *cols, int32_t ncols,
                          const tdp_pred *preds, int32_t npreds, int64_t n, const int32_t *sel,
                          const int64_t *d_nsel, int32_t key_col, int32_t *out_probe_row,
                          int32_t *out_payload, const int32_t *gather_cols, int32_t ngather,
                          void *const *gather_out, int64_t capacity, int64_t *d_count, void *ws,
                          size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes for tdp_join: the table plus the probe's scan state. */
size_t tdp_join_workspace(int64_t n_build, int64_t n_probe, int64_t nslots);

/*
 * Inner equi-join in one call: tdp_join_build over the build columns into a
 * table placed in `ws` (nslots <= 0 picks tdp_join_default_slots(n_build)),
 * then tdp_join_probe.  Build keys must be unique (N:1).
 */
tdp_status tdp_join(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                    int32_t nbuild_preds, int64_t n_build, int32_t build_key_col, int32_t build_payload_col,
                    const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                    int32_t nprobe_preds, int64_t n_probe, int32_t probe_key_col, int64_t nslots,
                    int32_t *out_probe_row, int32_t *out_payload, const int32_t *gather_cols,
                    int32_t ngather, void *const *gather_out, int64_t capacity, int64_t *d_count,
                    void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes for tdp_join_nm. */
size_t tdp_join_nm_workspace(int64_t n_build, int64_t n_probe);

/*
 * Inner equi-join with repeated build keys (N:M): every (probe row, build
 * row) pair with equal int32 keys, ordered by probe row and, for one probe
 * row, by build row -- the SQL inner join of Sec. 2's relational operators
 * without the unique-key restriction of tdp_join.
 *
 *   build_cols / build_preds   build side and its fused filter; rows
 *                              0..n_build-1, or 0..min(n_build, *d_nbuild)-1
 *   probe_cols / probe_preds   probe side and its fused filter; rows
 *                              0..n_probe-1, or 0..min(n_probe, *d_nprobe)-1
 *   out_probe_row, out_build_row
 *                              device int32[capacity]: the pairs in that order
 *   d_count                    device int64: the number of pairs (may exceed
 *                              both input sizes); more than capacity writes
 *                              capacity pairs and sets TDP_ERR_CAPACITY
 *
 * The qualifying build rows are sorted by key with the stable radix sort
 * (equal keys keep build-row order); the runs of equal keys go into the hash
 * table as one entry each (key -> run); every probe row looks its key up once,
 * the run lengths give every probe row its output offset, and the row then
 * writes its run.  As in tdp_join_build, the key INT32_MIN cannot be stored:
 * such build rows set TDP_ERR_OVERFLOW and are dropped, and such probe rows
 * match nothing.
 */
tdp_status tdp_join_nm(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                       int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild, int32_t build_key_col,
                       const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                       int32_t nprobe_preds, int64_t n_probe, const int64_t *d_nprobe, int32_t probe_key_col,
                       int32_t *out_probe_row, int32_t *out_build_row, int64_t capacity, int64_t *d_count,
                       void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/* Workspace bytes for tdp_join_probe_agg. */
size_t tdp_join_probe_agg_workspace(int64_t n, int64_t domain, int32_t naggs);

/*
 * Fused probe + group-by ("group-join"): probe the table with the probe key
 * and GROUP BY the build payload (int32 in [lo, hi], the group key), with
 * aggregates over probe-side columns.  Output as tdp_groupby_agg: groups in
 * ascending payload order, out_keys int32, out_aggs int64 per aggregate,
 * d_ngroups.  Probe rows with no match are dropped (inner join).  Probe rows
 * are 0..n-1, or 0..min(n, *d_n)-1 when d_n != NULL.
 */
tdp_status tdp_join_probe_agg(const uint64_t *table, int64_t nslots, const tdp_col *cols, int32_t ncols,
                              const tdp_pred *preds, int32_t npreds, int64_t n, const int64_t *d_n,
                              int32_t key_col,
                              int64_t payload_lo, int64_t payload_hi, const tdp_agg *aggs, int32_t naggs,
                              int32_t *out_keys, int64_t *const *out_aggs, int64_t capacity,
                              int64_t *d_ngroups, void *ws, size_t ws_bytes, int32_t *d_status,
                              tdp_stream_t stream);

/* Workspace bytes for tdp_groupjoin (0 when the arguments are invalid). */
size_t tdp_groupjoin_workspace(int64_t n_build, int64_t key_lo, int64_t key_hi, int32_t naggs, int32_t topk);

/*
 * Group-join whose group key is the join key (Sec. 2 relational operators;
 * the shipping-priority shape "JOIN ... ON key GROUP BY key"):
 *
 *   SELECT key, aggs(probe columns)
 *   FROM build JOIN probe ON build.key = probe.key
 *   WHERE build_preds AND probe_preds GROUP BY key ORDER BY key
 *
 * Build keys must be unique (N:1) and lie in the metadata bounds
 * [key_lo, key_hi] (int32 values, key_hi - key_lo < 2^31): a repeated build
 * key sets
 * TDP_ERR_DUP_BUILD_KEY and a build key outside the bounds sets
 * TDP_ERR_OVERFLOW (that row is dropped).  Probe keys outside the bounds
 * match nothing.  The build key set becomes an order-preserving dense code
 * (Sec. 2, Data Encoding): a bitmap of the key domain with a running rank
 * per 32-key word, 8 bytes per 32 keys of the domain in the workspace.  The
 * probe adds each matching row straight into the accumulators of its code,
 * and the groups are read out in code order, which is key order.
 *
 *   build_cols / build_preds   build side (fused filter); rows 0..n_build-1,
 *                              or 0..min(n_build, *d_nbuild)-1
 *   probe_cols / probe_preds   probe side (fused filter); rows 0..n_probe-1,
 *                              or 0..min(n_probe, *d_nprobe)-1
 *   build_key_col, probe_key_col  int32 key columns
 *   aggs[naggs]                1..8 aggregates over probe columns (COUNT,
 *                              SUM, SUM(a*(k-b)), AVG, MIN, MAX), exact int64
 *   out_keys (int32), out_aggs[naggs] (int64), capacity, d_ngroups
 *                              groups in ascending key order, as
 *                              tdp_groupby_agg writes them
 *   d_nmatch                   optional device int64: the number of joined
 *                              rows (the inner join's row count)
 *   topk, topk_agg             optional fused ORDER BY aggs[topk_agg] DESC,
 *                              key ASC LIMIT topk (1..16; 0: none) over the
 *                              groups: min(topk, groups) results go to
 *                              out_top_vals / out_top_keys and their count
 *                              to *d_topk (as tdp_topk writes them); the
 *                              groups must fit `capacity`
 *
 * Equal to tdp_join_build + tdp_join_probe + tdp_groupby_agg over the
 * joined rows (and tdp_topk over the groups), bit for bit.
 */
tdp_status tdp_groupjoin(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                         int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild, int32_t build_key_col,
                         const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                         int32_t nprobe_preds, int64_t n_probe, const int64_t *d_nprobe, int32_t probe_key_col,
                         int64_t key_lo, int64_t key_hi, const tdp_agg *aggs, int32_t naggs, int32_t *out_keys,
                         int64_t *const *out_aggs, int64_t capacity, int64_t *d_ngroups, int64_t *d_nmatch,
                         int32_t topk, int32_t topk_agg, int64_t *out_top_vals, int32_t *out_top_keys,
                         int64_t *d_topk, void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);

/*
 * The same group-join in three steps over one workspace, so that a build
 * side can be probed by several batches of probe rows (and each step timed
 * on its own).  Every step takes the same n_build, key_lo, key_hi, aggs,
 * naggs and topk, and the workspace of tdp_groupjoin_workspace(n_build,
 * key_lo, key_hi, naggs, topk); the steps run in stream order.
 *
 *   tdp_groupjoin_build   clears the workspace, inserts the qualifying build
 *                         keys (duplicates and keys outside [key_lo, key_hi]
 *                         flagged as in tdp_groupjoin) and ranks them; the
 *                         aggregates' ops fix the accumulator layout (their
 *                         column indices are not read)
 *   tdp_groupjoin_probe   adds the qualifying probe rows that find their key
 *                         to the groups and to the joined-row count; may be
 *                         called any number of times between build and finish
 *                         (each call with its own probe columns)
 *   tdp_groupjoin_finish  writes the groups in ascending key order, the
 *                         joined-row count (d_nmatch, optional) and the
 *                         optional top-k, as tdp_groupjoin does
 */
tdp_status tdp_groupjoin_build(const tdp_col *build_cols, int32_t nbuild_cols, const tdp_pred *build_preds,
                               int32_t nbuild_preds, int64_t n_build, const int64_t *d_nbuild, int32_t build_key_col,
                               int64_t key_lo, int64_t key_hi, const tdp_agg *aggs, int32_t naggs, int32_t topk,
                               void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);
tdp_status tdp_groupjoin_probe(const tdp_col *probe_cols, int32_t nprobe_cols, const tdp_pred *probe_preds,
                               int32_t nprobe_preds, int64_t n_probe, const int64_t *d_nprobe, int32_t probe_key_col,
                               int64_t n_build, int64_t key_lo, int64_t key_hi, const tdp_agg *aggs, int32_t naggs,
                               int32_t topk, void *ws, size_t ws_bytes, int32_t *d_status, tdp_stream_t stream);
tdp_status tdp_groupjoin_finish(int64_t n_build, int64_t key_lo, int64_t key_hi, const tdp_agg *aggs, int32_t naggs,
                                int32_t *out_keys, int64_t *const *out_aggs, int64_t capacity, int64_t *d_ngroups,
                                int64_t *d_nmatch, int32_t topk, int32_t topk_agg, int64_t *out_top_vals,
                                int32_t *out_top_keys, int64_t *d_topk, void *ws, size_t ws_bytes,
                                int32_t *d_status, tdp_stream_t stream);

/* ------------------------------------------------------- dictionary codes */

/* Workspace bytes for tdp_dict_encode (0 when the arguments are invalid). */
size_t tdp_dict_encode_workspace(int64_t n, int32_t max_len);

/*
 * Order-preserving dictionary encoding of a string column (Sec. 2, Data
 * Encoding): row i is the byte string bytes[offsets[i] .. offsets[i+1])
 * (offsets: device int32[n + 1]).  codes[i] (device int32[n]) is the number of
 * distinct strings of the column smaller than row i's string in bytewise
 * unsigned lexicographic order (a proper prefix first), so codes compare as
 * the strings do and can be grouped, joined and sorted in their place (as
 * bounded keys [0, ndict - 1]).  The dictionary -- the distinct strings in
 * order -- is written as dict_offsets (device int32[dict_cap + 1]) and
 * dict_bytes (device uint8[bytes_cap]); *d_ndict and *d_nbytes receive its
 * sizes (TDP_ERR_CAPACITY when it does not fit; the codes are complete).
 *
 * Strings may hold up to max_len bytes (1..32): longer rows set
 * TDP_ERR_OVERFLOW and are encoded as the empty string.  The rows are sorted
 * by (zero-padded 8-byte words, length) with a stable LSD radix sort (one
 * pass for the length, then one per word from the last), and one pass over
 * the sorted rows numbers the runs of equal strings.
 */
tdp_status tdp_dict_encode(const int32_t *offsets, const uint8_t *bytes, int64_t n, int32_t max_len, int32_t *codes,
                           int32_t *dict_offsets, uint8_t *dict_bytes, int64_t dict_cap, int64_t bytes_cap,
                           int64_t *d_ndict, int64_t *d_nbytes, void *ws, size_t ws_bytes, int32_t *d_status,
                           tdp_stream_t stream);

/* ----------------------------------------------------------------- top-k */

/* Workspace bytes for tdp_topk over n rows. */
size_t tdp_topk_workspace(int64_t n, int32_t k);

/*
 * ORDER BY value DESC, key ASC LIMIT k over n (value int64, key int32) rows
 * (the top-k queries of Sec. 5.1).  n rows, or *d_n rows when d_n != NULL
 * (n is then the capacity).  Writes min(k, rows) results and their count to
 * *d_k.  1 <= k <= 16.
 */
tdp_status tdp_topk(const int64_t *vals, const int32_t *keys, int64_t n, const int64_t *d_n, int32_t k,
                    int64_t *out_vals, int32_t *out_keys, int64_t *d_k, void *ws, size_t ws_bytes,
                    int32_t *d_status, tdp_stream_t stream);

/* ------------------------------------------------- soft (trainable) query */

/*
 * Workspace bytes for the soft aggregation / soft filter backward calls.
 * The grouped soft calls take 1 <= n_groups <= 4096 and a gid outside
 * [0, n_groups) leaves its row out of the sums.
 */
size_t tdp_soft_workspace(int64_t n, int32_t n_groups);

/*
 * Soft filter, Sec. 4 (logistic relaxation of the step function of a
 * predicate x > theta):  mask[i] = sigmoid((x[i] - theta[gid[i]]) / tau).
 * x, mask: fp32[n]; gid: int32[n] in [0, n_groups); theta: fp32[n_groups].
 */
tdp_status tdp_soft_filter_fwd(const float *x, const int32_t *gid, const float *theta, float tau,
                               int64_t n, float *mask, tdp_stream_t stream);

/*
 * Adjoint of tdp_soft_filter_fwd for upstream gradient grad_mask:
 *   grad_theta[g] = -(1/tau) * sum_{gid[i]=g} grad_mask[i] m_i (1 - m_i)
 *   grad_x[i]     =  (1/tau) * grad_mask[i] m_i (1 - m_i)      (optional)
 * The mask is recomputed, not read.  grad_theta is overwritten.
 */
tdp_status tdp_soft_filter_bwd(const float *x, const int32_t *gid, const float *theta, float tau,
                               int64_t n, int32_t n_groups, const float *grad_mask, float *grad_x,
                               float *grad_theta, void *ws, size_t ws_bytes, tdp_stream_t stream);

/*
 * Soft grouped aggregation, Sec. 4 (soft_count / soft_groupby): with
 * m_i = sigmoid((x[i] - theta[gid[i]]) / tau),
 *   sum[g] = sum_{gid[i]=g} v[i] m_i ,   cnt[g] = sum_{gid[i]=g} m_i .
 * The mask is never stored.  Each block keeps, per group, a compensated
 * fp32 pair (hi, lo) in shared memory: every term is added to hi by an
 * atomic whose returned old value gives the exact rounding error of the
 * addition (TwoSum), and that error is added to lo, so hi + lo carries the
 * block's group sum to about fp32^2 whatever the order of the atomics.  The
 * per-block sums are widened to float64 and combined in block order by a
 * fixed tree.  sum, cnt: fp32[n_groups], overwritten.
 */
tdp_status tdp_soft_agg_fwd(const float *x, const float *v, const int32_t *gid, const float *theta,
                            float tau, int64_t n, int32_t n_groups, float *sum, float *cnt, void *ws,
                            size_t ws_bytes, tdp_stream_t stream);

/*
 * tdp_soft_agg_fwd without a workspace, for callers that cannot allocate
 * device memory: code where a cudaMalloc is not allowed or would synchronise
 * the device at a bad moment, or an embedding host that only passes in
 * buffers it registered up front.  The paper has no counterpart; this is a
 * deployment variant of the call above, with the same arguments minus ws.
 * It runs the same kernels.  Up to about 4.2M rows (256 blocks of the
 * reduction) the grid, and so every summation order, equals that of
 * tdp_soft_agg_fwd and the results are bitwise equal; above that the grid is
 * capped at 256 blocks with longer chunks, the float64 combine adds
 * different block sums, and the results agree with tdp_soft_agg_fwd within
 * the soft operators' tolerance (1e-5 relative per group), not bitwise.
 *
 * Scratch: the per-block float64 partial sums live in one fixed 4 MiB array
 * in the library's device image (256 blocks x 2 sums x 1024 groups), which
 * every GPU that loads the library holds until the process exits.
 *   - n_groups must be <= 1024; larger values return
 *     TDP_ERR_WORKSPACE_TOO_SMALL (use tdp_soft_agg_fwd then).
 *   - The first call on a device looks up the array's device address with
 *     that device current (one cudaGetSymbolAddress, no allocation); make
 *     that first call before any stream capture.  The address is cached for
 *     the life of the process: after a cudaDeviceReset of that device it is
 *     stale, so do not call this entry point again in that process.
 *   - All calls share the one array: two calls whose kernels overlap on the
 *     GPU (different streams, or different threads) race and give wrong
 *     sums.  Serialise them.  Each call overwrites the parts it reads, so
 *     nothing has to be cleared between calls.
 * No device memory is allocated or freed by this call.
 */
tdp_status tdp_soft_agg_fwd_noalloc(const float *x, const float *v, const int32_t *gid, const float *theta,
                                    float tau, int64_t n, int32_t n_groups, float *sum, float *cnt,
                                    tdp_stream_t stream);

/*
 * Adjoint of tdp_soft_agg_fwd for upstream gradients gsum, gcnt (fp32[G]):
 *   grad_theta[g] = -(1/tau) sum_{gid[i]=g} (gsum[g] v_i + gcnt[g]) m_i (1-m_i)
 *   grad_v[i]     = gsum[gid[i]] m_i                                (optional)
 *   grad_x[i]     = (gsum[gid[i]] v_i + gcnt[gid[i]]) m_i (1-m_i) / tau (optional)
 * The mask is recomputed from x, theta.  grad_theta is overwritten.
 */
tdp_status tdp_soft_agg_bwd(const float *x, const float *v, const int32_t *gid, const float *theta,
                            float tau, int64_t n, int32_t n_groups, const float *gsum, const float *gcnt,
                            float *grad_theta, float *grad_v, float *grad_x, void *ws, size_t ws_bytes,
                            tdp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TDP_H */
