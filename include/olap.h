/*
 * olap.h -- C ABI of the GB300 key-only OLAP offload library.
 *
 * The library implements the two execution-layer primitives the paper
 * offloads to the GPU and the cost gate that decides when to offload
 * ("GPU-Augmented OLAP Execution Engine: GPU Offloading", arXiv 2601.19911):
 *
 *   - Top-K selection, ORDER BY key LIMIT K (Sec. III-A): key-only input,
 *     radix-based selection, the Top-K row pointers returned in order.
 *   - Key-based hash join build and probe (Sec. III-B): a key-only hash table,
 *     parallel probing, the set of matched (probe, build) row pointers returned
 *     for late materialization on the host (Sec. II-C).
 *   - The Risky Gate (Sec. II-B, Sec. V-D): fitted CPU / transfer / kernel /
 *     post-processing cost models, the offload decision and the break-even N*.
 *
 * Key-only contract (Sec. II-C): only (key, row-id) crosses the host-device
 * link; row-ids are uint32 and may be implicit (NULL => row-id = index), in
 * which case only the keys cross.  Late materialization is the caller's job.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an olap_status; nothing throws across the ABI.
 *     olap_last_error() describes the last failure on a context.
 *   - The caller owns every input and output buffer.  The library owns the
 *     context, its device scratch, its pinned staging buffers and join tables.
 *   - Pointers tagged OLAP_MEM_DEVICE must be device memory of the context's
 *     device; OLAP_MEM_HOST_PINNED must be page-locked host memory;
 *     OLAP_MEM_HOST may be any host memory (read by a copy kernel where the
 *     device accesses pageable memory through the host page tables, else
 *     staged through pinned buffers; see olap_host_access).
 *   - Keys must be naturally aligned (8 bytes for 8-byte key types, 4 for
 *     4-byte ones).
 *   - Blocking calls return after the result is in the output buffers.
 *     Calls suffixed _async only enqueue work on the given stream, take device
 *     pointers only, and report device-side status through a device word.
 *   - A context works on its own non-blocking stream, which waits for no
 *     other stream: device buffers a blocking call reads or writes must be
 *     complete (inputs written, outputs no longer in use) when it is made,
 *     and an _async call on another stream must be ordered by the caller.
 *   - There is no CPU fallback: when no GPU is usable a call fails with
 *     OLAP_E_CUDA.  The gate only advises; running the CPU path is the
 *     caller's engine's job.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef OLAP_H
#define OLAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OLAP_OK = 0,
    OLAP_E_INVALID = 1,        /* bad argument (null pointer, bad enum, size limit) */
    OLAP_E_NOMEM = 2,          /* device or pinned allocation failed / budget exceeded */
    OLAP_E_CUDA = 3,           /* a CUDA runtime call failed (no device, launch error) */
    OLAP_E_OVERFLOW = 4,       /* output capacity too small; required count reported */
    OLAP_E_TIMEOUT = 5,        /* a bounded device-side wait expired; context reset */
    OLAP_E_UNIMPLEMENTED = 6,
    OLAP_E_DEVICE = 7          /* device-side validation rejected a descriptor */
} olap_status;

/* Key types of Top-K.  Floats are ordered by IEEE 754-2019 totalOrder (the
 * paper's key column is a double, Sec. V-A); integers by value.  The join
 * takes int64 keys only. */
typedef enum {
    OLAP_KEY_I64 = 0,
    OLAP_KEY_F32 = 1,
    OLAP_KEY_F64 = 2,
    OLAP_KEY_U64 = 3,
    OLAP_KEY_I32 = 4,
    OLAP_KEY_U32 = 5
} olap_key_type;
typedef enum { OLAP_ASC = 0, OLAP_DESC = 1 } olap_order;
typedef enum { OLAP_MEM_HOST = 0, OLAP_MEM_HOST_PINNED = 1, OLAP_MEM_DEVICE = 2 } olap_mem;

typedef struct olap_ctx olap_ctx;
typedef struct olap_join_table olap_join_table;

/* Context options.  Zero means "library default" for every field. */
typedef struct {
    int device;                 /* CUDA device ordinal */
    void* stream;               /* cudaStream_t to run on; NULL => the context creates one */
    uint64_t mem_budget_bytes;  /* cap on device scratch + tables held by the context */
    double margin_ms;           /* gate margin (Sec. IV, gate margin 0/5/10 ms) */
    int block_threads;          /* threads per CTA of the Top-K streaming filter (256/512/1024;
                                   0 => 512) */
    double load_factor;         /* join table load factor in (0, 0.9]; 0 => 0.5 */
    uint64_t staging_bytes;     /* size of each pinned staging buffer; 0 => 64 MiB */
    int topk_filter;            /* olap_filter: how the Top-K streaming pass reads keys */
    int topk_tile_bytes;        /* bulk-copy size of the streaming pass (multiple of 8 KiB) */
    int topk_stages;            /* bulk copies in flight per CTA (1..16) */
    int topk_ctas_per_sm;       /* resident CTAs per SM of the Top-K grid (1..4) */
    int join_partitions;        /* join probe: 0 => automatic (partition the probe rows by
                                   home bucket when the table is well above L2), 1 => direct
                                   probe, a power of two 2..256 => that many partitions */
    int join_bucket_loads;      /* olap_loads: cache path of the probe's bucket reads */
    int l2_fetch_bytes;         /* 0 => leave the device's L2 fetch granularity; 32, 64 or 128
                                   => set it (cudaLimitMaxL2FetchGranularity) when the context
                                   is created; it applies to the whole process on that device */
    int topk_digit_bits;        /* radix digit width of the Top-K selects (8..12; 0 => 12), also
                                   for batches created on this context */
    int host_access;            /* olap_host_access: how pageable host memory is copied */
    int batch_overlap;          /* batches: 0 => the Top-K and probe kernels run one after the
                                   other, 1 => side by side (two branches of the graph); each
                                   already fills the GPU, and side by side measured no faster */
    int batch_topk_ctas_per_sm; /* batches: resident Top-K CTAs per SM (1 or 2; 0 => 2) */
    int join_prefilter;         /* olap_prefilter: Bloom pre-probe of the join (Sec. III-B) */
    int staging_threads;        /* host threads that copy pageable data into and out of the
                                   pinned staging buffers (1..64; 0 => 4) */
} olap_opts;

/* Bloom pre-probe of the join ("bloom-filter/partitioned hash", Sec. III-B).
 * A table far above L2 gets a blocked Bloom filter over its keys (about 16
 * bits per build row, one 32-byte block per key) when it is built.  Before a
 * probe, a sample of the probe keys is tested on the device; when few pass,
 * one streaming pass drops every probe row the filter rules out and only the
 * rest is probed (partitioned or direct).  No host synchronisation: the
 * decision and the surviving row count stay on the device. */
typedef enum {
    OLAP_PREFILTER_AUTO = 0,    /* filter built for tables above half of L2; used when at most
                                   60 % of a 4096-key sample of a probe of >= 2^20 rows passes */
    OLAP_PREFILTER_OFF = 1,     /* no filter built, none used */
    OLAP_PREFILTER_ON = 2       /* filter built for every table (with rows) and used for every
                                   probe */
} olap_prefilter;

/* How pageable host inputs and outputs (OLAP_MEM_HOST) cross the host link. */
typedef enum {
    OLAP_HOST_AUTO = 0,         /* a copy kernel reads / writes the pageable memory itself when the
                                   device accesses it coherently through the host page tables
                                   (cudaDevAttrPageableMemoryAccessUsesHostPageTables, e.g. Grace
                                   over NVLink-C2C); else as OLAP_HOST_STAGED */
    OLAP_HOST_STAGED = 1        /* CPU copies through two pinned staging buffers, overlapped with
                                   the DMA of the other */
} olap_host_access;

/* Cache path of the join probe's random bucket reads. */
typedef enum {
    OLAP_LOADS_AUTO = 0,        /* the default: L2_ONLY, L1 for a probe made direct by a skewed sample */
    OLAP_LOADS_L1 = 1,          /* read-only path through L1 (ld.global.nc) */
    OLAP_LOADS_L2_ONLY = 2      /* bypass L1 (ld.global.cg): no L1 line fills for 32-byte reads */
} olap_loads;

/* Streaming-pass flavour of Top-K: 16-byte register loads (the default), or
 * bulk asynchronous copies (TMA engine) through a ring of shared-memory
 * stages. */
typedef enum { OLAP_FILTER_AUTO = 0, OLAP_FILTER_BULK = 1, OLAP_FILTER_REGS = 2 } olap_filter;

/* Create a context on opts->device (opts may be NULL for all defaults).
 * Fails with OLAP_E_CUDA when no CUDA device is usable. */
olap_status olap_ctx_create(const olap_opts* opts, olap_ctx** out);
void olap_ctx_destroy(olap_ctx* ctx);
/* Message for the last failed call on ctx (never NULL; "" after success). */
const char* olap_last_error(const olap_ctx* ctx);
/* The cudaStream_t the context runs on. */
void* olap_ctx_stream(const olap_ctx* ctx);
/* Wait for all work the context enqueued. */
olap_status olap_ctx_sync(olap_ctx* ctx);
/* 1 when the context copies pageable host memory with a kernel that reads it
 * directly (OLAP_HOST_AUTO on a device with host-page-table access), else 0;
 * 0 for NULL. */
int olap_ctx_host_direct(const olap_ctx* ctx);
/* Self-test of the bounded device-side waits (every spin in the library
 * gives up after a limit and reports OLAP_E_TIMEOUT instead of hanging): one
 * thread runs the grid barriers' wait on a device word that nothing writes,
 * for at most limit_cycles (1 .. 2^31) SM clock cycles, then returns.
 * *out_status receives the device status the wait recorded -- OLAP_E_TIMEOUT
 * when the bound works.  Returns OLAP_E_INVALID for a bad limit, else OLAP_OK
 * (or E_CUDA).  The context stays usable. */
olap_status olap_selftest_wait(olap_ctx* ctx, uint64_t limit_cycles, int32_t* out_status);

/* ------------------------------------------------------------------------
 * Top-K selection, ORDER BY key {ASC|DESC} LIMIT k (Sec. III-A; Sec. V-B
 * names the query form ORDER BY value DESC LIMIT 100).
 *
 * keys        n keys of `type` (olap_key_type: int64, uint64, int32, uint32
 *             by value; float32 / float64 by IEEE 754-2019 totalOrder, so
 *             -0 < +0 and NaNs sort outside +-inf by sign), in memory
 *             `in_where`; 8-byte keys 8-byte aligned, 4-byte keys 4-byte
 *             aligned.
 * rowids      n uint32 row-ids in the same memory kind, or NULL for
 *             row-id = index.
 * order       OLAP_ASC or OLAP_DESC on the key; ties on equal keys are always
 *             broken by row-id ascending.
 * out_keys    min(k, n) keys (original bit patterns, same type), in order.
 * out_rowids  min(k, n) row-ids in the same order.
 * out_where   memory kind of both outputs.
 * out_count   (host) receives min(k, n).
 * Limits: n < 2^32.  k = 0 or n = 0 => OLAP_OK with count 0.
 * With row-ids in page-locked host memory and the sampled path (n > 2^21,
 * k <= n / 256), the row-ids are not copied: the kernels read the
 * candidates' row-ids in place over the host link (olap_topk_info_last
 * reports it); the keys are copied as usual.
 * The result is bit-exact: it equals a stable sort by (key, row-id) cut at k.
 * ------------------------------------------------------------------------ */
olap_status olap_topk(olap_ctx* ctx, const void* keys, olap_key_type type, const uint32_t* rowids,
                      olap_mem in_where, uint64_t n, uint64_t k, olap_order order,
                      void* out_keys, uint32_t* out_rowids, olap_mem out_where,
                      uint64_t* out_count);

/* Top-K over a two-column key: ORDER BY c0 [ASC|DESC], c1 [ASC|DESC] LIMIT k
 * (Sec. III-A's ORDER BY key LIMIT K, Sec. V-B, with a second key column, as
 * SQL's ORDER BY lists allow).  Rows are compared on c0 in order0, then on c1
 * in order1, then by row-id ascending.  Both columns hold n keys of a 4-byte
 * type (int32, uint32 or float32 by IEEE totalOrder; other widths return
 * OLAP_E_UNIMPLEMENTED), in memory `where` with the row-ids (NULL => index).
 * out_keys0 / out_keys1 receive each column's key bits of the min(k, n)
 * selected rows, out_rowids their row-ids, in order (memory `out_where`).
 * The composite key maps to one 64-bit rank word (c0's order-preserving
 * 32 bits above c1's), which the same select refines.  Errors as olap_topk.
 * Blocking. */
olap_status olap_topk_pair(olap_ctx* ctx, const void* keys0, olap_key_type type0, olap_order order0,
                           const void* keys1, olap_key_type type1, olap_order order1, const uint32_t* rowids,
                           olap_mem where, uint64_t n, uint64_t k, void* out_keys0, void* out_keys1,
                           uint32_t* out_rowids, olap_mem out_where, uint64_t* out_count);

/* Asynchronous Top-K on device pointers only, enqueued on `stream` (NULL =>
 * the context's stream).  Writes min(k, n) results; `dev_status` (device
 * int32, may be NULL) receives an olap_status from the device side.  The
 * context's scratch is reused by the next call on the same context, so calls
 * on one context must be serialised on one stream. */
olap_status olap_topk_async(olap_ctx* ctx, const void* d_keys, olap_key_type type,
                            const uint32_t* d_rowids, uint64_t n, uint64_t k, olap_order order,
                            void* d_out_keys, uint32_t* d_out_rowids, int32_t* dev_status,
                            void* stream);

/* What the last Top-K on this context did (diagnostics; blocks until the
 * context's stream is idle).  path: 0 = radix refine over the input (small n
 * or large k), 1 = sampled threshold + one streaming pass + refine over the
 * candidates, 2 = sample misjudged, refine over the input.  phase_ns:
 * sample, filter, refine, split, finish/sort, total, and within finish the
 * small-bucket sort and the survivor sort (device %globaltimer).
 * rowids_in_place: 1 when the call (a blocking olap_topk or olap_topk_pair
 * on the sampled path with row-ids in page-locked host memory) read the candidates'
 * row-ids in host memory instead of copying all n to the device. */
typedef struct {
    int path;
    int refine_passes;
    uint64_t candidates;
    uint64_t phase_ns[8];
    int rowids_in_place;
    int reserved;
} olap_topk_info;
olap_status olap_topk_info_last(olap_ctx* ctx, olap_topk_info* out);

/* Per-kernel device time, from CUDA events recorded on the launching stream
 * around each kernel of the Top-K and join probe calls made while timing is
 * on (off by default; each timed call records up to four events more). */
olap_status olap_ctx_time_kernels(olap_ctx* ctx, int on);
typedef struct {
    float topk_prepare_ms;           /* sample threshold kernel */
    float topk_filter_ms;            /* streaming filter (-1: the plan had none) */
    float topk_select_ms;            /* cooperative select kernel */
    float join_probe_ms;             /* the whole probe: its one kernel, or the count, scatter and
                                        probe kernels of the partitioned probe */
} olap_kernel_ms;
/* Times of the last timed Top-K and join probe on this context (waits for
 * them); -1 for a kernel that was not timed. */
olap_status olap_kernel_ms_last(olap_ctx* ctx, olap_kernel_ms* out);

/* Kernels this context has launched since it was created: every launch of
 * the library's own kernels made for it (Top-K, join build and probe, copy
 * kernels of pageable memory, full-row extraction and gather, tuning inputs),
 * and each replay of a batch graph counted as the kernels inside it.  Copies
 * and memsets are not kernels.  Host bookkeeping only. */
olap_status olap_ctx_launches(const olap_ctx* ctx, uint64_t* count);

/* ------------------------------------------------------------------------
 * Autotuner.  The paper fixes no kernel parameters; this picks them by
 * measurement on the caller's shape: the Top-K streaming-filter block size
 * (256/512/1024) and radix digit width (8/10/11/12 bits), and the join's load
 * factor (0.25/0.35/0.5/0.7), probe mode (automatic partitioning or direct)
 * and bucket-read cache path.  Candidates run on tuning inputs the library
 * generates on the device (uniform keys; probe rows hitting the build side
 * with the given rate); each is timed with CUDA events on the context
 * stream, the median of `reps` runs after one untimed run.  On success the
 * context keeps the fastest configuration (block_threads, topk_digit_bits,
 * load_factor, join_partitions, join_bucket_loads of its options); batches
 * created afterwards use its digit width.  Blocking.  Errors: E_INVALID for
 * bad sizes (each below 2^32) or probe rows without build rows; E_NOMEM when
 * no join candidate fits the budget; E_CUDA.  Device memory for the tuning
 * inputs is allocated and freed inside the call.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint64_t topk_n;                 /* keys of the Top-K shape (0 => leave Top-K as is) */
    int topk_key_type;               /* olap_key_type */
    int reps;                        /* timed runs per candidate (0 => 5) */
    uint64_t topk_k;
    uint64_t join_build_n;           /* build rows of the join shape (0 => leave the join as is) */
    uint64_t join_probe_n;           /* probe rows */
    double join_hit_rate;            /* fraction of probe rows that find a build key */
    uint64_t seed;                   /* of the tuning inputs */
} olap_tune_request;

typedef struct {
    int block_threads;               /* chosen Top-K filter block size */
    int topk_digit_bits;             /* chosen radix digit width */
    double topk_ms;                  /* median Top-K time with the choice */
    double topk_default_ms;          /* median Top-K time with 512 threads, 12-bit digits */
    double load_factor;              /* chosen join load factor */
    int join_partitions;             /* 0 automatic, 1 direct */
    int join_bucket_loads;           /* olap_loads */
    double join_probe_ms;            /* median probe time with the choice */
    double join_probe_default_ms;    /* load 0.5, automatic partitioning, L2-only reads */
    double join_build_ms;            /* build time at the chosen load factor */
    int candidates;                  /* configurations timed */
    int pad;
} olap_tune_result;

olap_status olap_autotune(olap_ctx* ctx, const olap_tune_request* req, olap_tune_result* out);

/* ------------------------------------------------------------------------
 * Full-row offload, the foil of key-only transfer with late materialization
 * (Sec. II-C: only (key, row-id) cross the link and the host re-reads the
 * other columns for the few returned row-ids; Sec. V-E measures both).  Here
 * the whole rows cross the link: the key field is extracted on the device,
 * the Top-K is selected as in olap_topk, and the K selected rows are gathered
 * on the device and returned whole.
 *
 * rows        n fixed-width rows of row_bytes bytes in memory `in_where`; the
 *             key of row i (type `type`) is at byte key_offset of it.
 * out_rows    min(k, n) rows of row_bytes, in order, in memory `out_where`.
 * out_rowids  min(k, n) row indices, or NULL.
 * Errors: E_INVALID for a key field outside the row (key_offset + key width >
 * row_bytes), bad kinds, n >= 2^32 or NULL buffers; E_NOMEM; E_CUDA;
 * E_TIMEOUT as olap_topk.  Blocking.
 * ------------------------------------------------------------------------ */
olap_status olap_topk_rows(olap_ctx* ctx, const void* rows, olap_mem in_where, uint64_t n, uint32_t row_bytes,
                           uint32_t key_offset, olap_key_type type, uint64_t k, olap_order order, void* out_rows,
                           uint32_t* out_rowids, olap_mem out_where, uint64_t* out_count);

/* ------------------------------------------------------------------------
 * Key-based hash join, build and probe (Sec. III-B: "parallel probing using a
 * key-only hash table", pointers returned for late materialization, Sec. II-C).
 *
 * The table is an open-addressing table of 16-byte slots {int64 key, uint32
 * row-id, uint32 count of further copies of the key along its chain}, two
 * slots per 32-byte bucket, with linear probing over buckets (a bucket with a
 * free slot ends every chain; a probe also stops at its key's last copy).
 * Capacity is the power of two of buckets that keeps n / (2 * buckets) at or
 * below the load factor.  Build rows whose key equals the table's empty
 * marker (all bits set, i.e. -1) are kept in a side list, so every int64 key
 * value joins correctly.  A table far above L2 also carries a blocked Bloom
 * filter for the pre-probe (see olap_prefilter).  The table stays resident on
 * the device until olap_join_free; it may be probed any number of times, from
 * any context on the same device.
 *
 * Result: every (probe row-id, build row-id) pair whose keys are equal, as a
 * multiset (duplicate keys on either side multiply), in no particular order.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint32_t probe_rowid;
    uint32_t build_rowid;
} olap_pair;

/* Build a table from n int64 keys (memory `where`) with row-ids (NULL =>
 * index; n < 2^32 then).  load_factor in (0, 0.9]; 0 takes the context's
 * option (default 0.5).  *out receives the table, owned by the caller until
 * olap_join_free.  Blocking. */
olap_status olap_join_build(olap_ctx* ctx, const int64_t* keys, const uint32_t* rowids, olap_mem where,
                            uint64_t n, double load_factor, olap_join_table** out);

/* Probe: for n keys (memory `where`, row-ids or NULL => index) write the
 * matching pairs to out (memory `out_where`, room for `capacity` pairs).
 * *out_count receives the number of pairs.  If it exceeds capacity the call
 * returns OLAP_E_OVERFLOW, *out_count holds the exact number needed and the
 * contents of out are unspecified; retry with capacity >= *out_count.
 * Blocking. */
olap_status olap_join_probe(olap_ctx* ctx, const olap_join_table* table, const int64_t* keys,
                            const uint32_t* rowids, olap_mem where, uint64_t n, olap_pair* out,
                            olap_mem out_where, uint64_t capacity, uint64_t* out_count);

/* Asynchronous probe on device pointers, enqueued on `stream` (NULL => the
 * context's stream).  d_count (device uint64) receives the pair count, which
 * may exceed capacity (then only `capacity` pairs were written).  Calls on
 * one context must be serialised on one stream. */
olap_status olap_join_probe_async(olap_ctx* ctx, const olap_join_table* table, const int64_t* d_keys,
                                  const uint32_t* d_rowids, uint64_t n, olap_pair* d_out, uint64_t capacity,
                                  uint64_t* d_count, void* stream);

/* How a probe of n rows against `table` runs on this context (Sec. III-B,
 * parallel probing): *parts = 1 for the direct probe (one kernel), else the
 * number of radix partitions of the partitioned probe (a count, a scatter and
 * a probe kernel).  Decided by the context's join_partitions option and, when
 * automatic, by the table's size against the device's L2.  An automatic
 * partitioned plan is confirmed on the device by a sample of the probe keys:
 * when they repeat (a skewed stream: at least a fifth of the sampled keys
 * that reach the probe equal an earlier one), the partition kernels return at
 * once and the probe reads its rows directly, its bucket reads through L1
 * unless join_bucket_loads says otherwise; olap_join_probe_info_last reports
 * what ran.  Host arithmetic only; OLAP_E_INVALID for a NULL or freed table
 * or a NULL *parts. */
olap_status olap_join_probe_partitions(olap_ctx* ctx, const olap_join_table* table, uint64_t n, int* parts);

/* How the last probe enqueued on this context ran: *parts as
 * olap_join_probe_partitions, or 1 when the device-side sample made an
 * automatic partitioned probe direct; *prefiltered = 1 when the Bloom pre-probe
 * dropped rows before the probe (0 when it was not used or the sample said
 * not to); *rows_probed = the probe rows left after it (n when not used).
 * Waits for the context's stream.  OLAP_E_INVALID for NULL outputs or when no
 * probe has run on the context. */
olap_status olap_join_probe_info_last(olap_ctx* ctx, int* parts, int* prefiltered, uint64_t* rows_probed);

/* Table facts: build rows, buckets (2 slots each), rows in the side list,
 * bytes of its Bloom filter (0: none).  Any output may be NULL. */
olap_status olap_join_table_info(const olap_join_table* table, uint64_t* n_build, uint64_t* n_buckets,
                                 uint64_t* n_side, uint64_t* bloom_bytes);

/* Free a table (NULL is ignored).  Waits for the table's device to finish
 * work that may still read it. */
void olap_join_free(olap_join_table* table);

/* ------------------------------------------------------------------------
 * Batched execution: many Top-K queries and probe batches in one persistent
 * launch fed by a device work queue and captured in a CUDA graph, against
 * one launch per query (the small-N overhead of Sec. IV, small-N interval).
 *
 * Every item is one Top-K (keys, n, k <= 4096, order; outputs as olap_topk,
 * count receives min(k, n)) or one probe (keys, n, against a resident table;
 * pairs as olap_join_probe, count receives the pair count, which may exceed
 * capacity).  All pointers are device pointers; count is a device uint64;
 * status (device int32, may be NULL) receives OLAP_OK or OLAP_E_DEVICE when
 * the device-side check of the descriptor rejects it.  The items' buffers
 * must outlive the batch; their contents may change between runs.
 * ------------------------------------------------------------------------ */
typedef struct olap_batch olap_batch;

typedef struct {
    int op;                          /* olap_op */
    int key_type;                    /* Top-K: olap_key_type */
    int order;                       /* Top-K: olap_order */
    const void* keys;
    const uint32_t* rowids;          /* NULL => index */
    uint64_t n;
    uint64_t k;                      /* Top-K */
    void* out_keys;                  /* Top-K */
    uint32_t* out_rowids;            /* Top-K */
    const olap_join_table* table;    /* probe */
    olap_pair* out_pairs;            /* probe */
    uint64_t capacity;               /* probe */
    uint64_t* count;                 /* device: rows (Top-K) or pairs (probe) written */
    int32_t* status;                 /* device, optional */
} olap_batch_item;

/* Check the items, upload the work queues (Top-K items largest first, one CTA
 * each; probe items largest first, cut into chunks of 32768 probe rows that
 * any CTA may take) and capture the persistent launches in a CUDA graph.
 * Blocking. */
olap_status olap_batch_create(olap_ctx* ctx, const olap_batch_item* items, uint64_t n_items, olap_batch** out);
/* Run every item once: one graph launch on `stream` (NULL => context stream). */
olap_status olap_batch_run(olap_batch* batch, void* stream);
/* The same work as one library call per item (olap_topk_async /
 * olap_join_probe_async) on `stream`: the per-query baseline. */
olap_status olap_batch_run_per_query(olap_batch* batch, void* stream);
/* Number of descriptors the device rejected in the last run (waits for it). */
olap_status olap_batch_errors(olap_batch* batch, int* errors);
void olap_batch_free(olap_batch* batch);

/* ------------------------------------------------------------------------
 * Risky Gate (Sec. II-B; fitted constants and break-even N*, Sec. V-D).
 *
 * The gate offloads only when the estimated CPU cost exceeds the estimated
 * GPU cost by more than a margin (ms):
 *   C_cpu  = a * x + b, x = N * log2(N) or N * K (Top-K; the form with the
 *            smaller residual on the calibration samples is kept, N log2 N on
 *            a tie) or N * M (probe; M = expected candidates per probe)
 *   C_gpu  = C_tx + C_ker + C_post, C_tx = c * bytes + d (key-only transfer),
 *            C_ker = e * N + f, C_post = g * rows returned + h
 *            (result return and late materialization)
 *   offload  <=>  C_cpu - C_gpu > margin  (strict)
 * Every fit is least squares in the centred closed form of the 2x2 normal
 * equations, ordinary or weighted by 1/y^2 (relative error; the measured
 * times span decades of N and unweighted the largest sizes decide the small-N
 * costs the gate exists for).  N* is the smallest integer N in [1, 2^34] where
 * C_cpu(N) - C_gpu(N) > margin for the query's K (or M), with transfer bytes
 * and returned rows scaled with N as the query says; 1 if that already holds
 * at N = 1 and 0 ("never") if it fails at 2^34.  Pure host arithmetic: these
 * calls touch no device.  The gate only advises; it runs no CPU path.
 * ------------------------------------------------------------------------ */
typedef enum { OLAP_OP_TOPK = 0, OLAP_OP_PROBE = 1 } olap_op;
/* CPU cost forms (Sec. II-B names alpha*N*log N and alpha*N*K).  OLAP_CPU_MAX
 * keeps both Top-K fits and estimates the larger of the two: a risk-averse
 * reading for a host engine whose cost follows neither form alone (a heap
 * selection costs about N for small K and grows with K log K for large K). */
typedef enum { OLAP_CPU_NLOGN = 0, OLAP_CPU_NK = 1, OLAP_CPU_NM = 2, OLAP_CPU_MAX = 3 } olap_cpu_form;
typedef enum { OLAP_FIT_ORDINARY = 0, OLAP_FIT_RELATIVE = 1 } olap_fit;

typedef struct {
    olap_op op;
    int weighting;                /* olap_fit */
    uint64_t count;               /* number of samples (>= 2) */
    const double* n;              /* input rows N */
    const double* k_or_m;         /* Top-K: K; probe: M */
    const double* tx_bytes;       /* bytes moved to the device */
    const double* out_rows;       /* rows returned (K, or pairs) */
    const double* t_cpu_ms;       /* measured CPU engine time */
    const double* t_tx_ms;        /* measured transfer time */
    const double* t_ker_ms;       /* measured kernel time */
    const double* t_post_ms;      /* measured result return + materialization time */
    int topk_cpu;                 /* Top-K: 0 => the form with the smaller residual;
                                     OLAP_CPU_MAX => both forms, the larger estimate */
    int pad;
    double cpu_split_n;           /* 0 => one CPU fit over every sample.  > 0 => the host engine
                                     changes regime at this size (it goes parallel, say): the CPU
                                     cost is fitted on its own over the samples with n < cpu_split_n
                                     and over those with n >= cpu_split_n (each side needs at least
                                     two samples of distinct x, else OLAP_E_INVALID) */
} olap_gate_samples;

typedef struct {
    olap_op op;
    olap_cpu_form cpu_form;
    double a, b;                  /* CPU: a * x + b */
    double c, d;                  /* transfer: c * bytes + d */
    double e, f;                  /* kernel: e * N + f */
    double g, h;                  /* post-processing: g * rows + h */
    double margin_ms;
    double rss_nlogn, rss_nk;     /* Top-K: residual sums of squares of both CPU forms (summed over
                                     both regimes when split) */
    double a2, b2;                /* OLAP_CPU_MAX: the N*K form (a, b hold the N*log2 N form) */
    double split_n;               /* 0 => one regime; else a, b (a2, b2) hold the CPU fit for
                                     n < split_n and a_hi, b_hi (a2_hi, b2_hi) the fit for
                                     n >= split_n, both in cpu_form */
    double a_hi, b_hi, a2_hi, b2_hi;
} olap_gate_model;

typedef struct {
    olap_op op;
    uint64_t n;                   /* input rows */
    double k_or_m;                /* K (Top-K) or M (probe) */
    double tx_bytes;              /* bytes this query moves to the device */
    double out_rows;              /* rows this query returns */
    double bytes_per_row;         /* for N*: transfer bytes per input row */
    double out_per_row;           /* for N* of a probe: returned rows per input row */
} olap_gate_query;

typedef struct {
    int offload;                  /* 1 => run on the GPU */
    double c_cpu, c_tx, c_ker, c_post, c_gpu;
    double gain_ms;               /* c_cpu - c_gpu */
    double margin_ms;
    uint64_t n_star;              /* break-even N for this query's shape */
} olap_gate_decision;

/* Fit the model from measured samples; margin_ms is stored in it. */
olap_status olap_gate_calibrate(const olap_gate_samples* samples, double margin_ms, olap_gate_model* out);
/* Decide one query and report its costs and break-even N*. */
olap_status olap_gate_estimate(const olap_gate_model* model, const olap_gate_query* query,
                               olap_gate_decision* out);

/* ------------------------------------------------------------------------
 * Serving loop (gated against always-on offload, Sec. II-B and Sec. IV).
 *
 * Requests arrive at given times (or all at once in closed loop).  Each is
 * decided on arrival -- by the gate, or always GPU, or always host -- and then
 * queued.  GPU requests are admitted first-come first-served into one of
 * gpu_slots slots, each with its own context (stream, device scratch and
 * pinned double buffers), as soon as a slot is free and the request's device
 * memory fits the budget next to the requests already running (a request is
 * always admitted when nothing else runs).  Requests in different slots
 * overlap on the device: this is continuous batching, not a queue in front of
 * one stream.  Host requests run on cpu_workers threads through the caller's
 * engine callback: the library has no CPU implementation of the primitives.
 * Latency = completion time - arrival time.  Keys and outputs are host
 * memory (key-only H2D through pinned staging, results D2H).
 * ------------------------------------------------------------------------ */
typedef struct {
    int op;                          /* olap_op */
    int key_type;                    /* Top-K: olap_key_type */
    int order;                       /* Top-K: olap_order */
    int table_id;                    /* probe: index of the table in the caller's engine */
    const void* keys;                /* host */
    const uint32_t* rowids;          /* host or NULL */
    uint64_t n;
    uint64_t k;                      /* Top-K */
    const olap_join_table* table;    /* probe (device table) */
    double expected_pairs;           /* probe: the caller's estimate, for the gate */
    double arrival_ms;               /* from the start of the run */
    void* out_keys;                  /* Top-K host outputs (>= min(k, n)) */
    uint32_t* out_rowids;
    olap_pair* out_pairs;            /* probe host output */
    uint64_t capacity;
    /* filled in by olap_serve */
    uint64_t out_count;
    int status;                      /* olap_status of the request */
    int on_gpu;
    double start_ms, done_ms;
} olap_serve_request;

/* The caller's host engine: run `req` on the CPU, write its outputs and
 * out_count; return an olap_status. */
typedef int (*olap_host_engine_fn)(void* user, olap_serve_request* req);

typedef enum { OLAP_SERVE_GATED = 0, OLAP_SERVE_ALWAYS_GPU = 1, OLAP_SERVE_ALWAYS_HOST = 2 } olap_serve_policy;

typedef struct {
    int policy;                      /* olap_serve_policy */
    int gpu_slots;                   /* concurrent GPU requests (default 4) */
    int cpu_workers;                 /* host engine threads (default 8) */
    uint64_t mem_budget_bytes;       /* device memory for in-flight requests (0 = unlimited) */
    const olap_gate_model* topk_model;
    const olap_gate_model* probe_model;
    olap_host_engine_fn host_engine;
    void* host_user;
    int closed_loop;                 /* 1: ignore arrival times, all arrive at 0 */
    const olap_opts* ctx_opts;       /* options of the slot contexts (device, staging) */
} olap_serve_opts;

typedef struct {
    double wall_ms;
    double throughput_rps;
    double p50_ms, p95_ms, p99_ms, mean_ms, max_ms;
    uint64_t n_gpu, n_host, n_failed;
    double offload_fraction;
    uint64_t peak_reserved_bytes;
} olap_serve_stats;

/* Serve n requests (sorted by arrival or not; served in arrival order) and
 * report latency percentiles and throughput.  Blocking. */
olap_status olap_serve(olap_serve_request* reqs, uint64_t n, const olap_serve_opts* opts, olap_serve_stats* out);

/* ------------------------------------------------------------------------
 * Top-K that allocates nothing (no counterpart in the paper: a deployment
 * entry point for callers that cannot let a library allocate GPU memory --
 * engines whose device memory is wholly reserved by their own pool, plug-in
 * or UDF hosts that forbid allocation inside an operator, and latency-critical
 * paths that cannot accept the device-wide synchronisation cudaMalloc and
 * cudaFree may cause).
 *
 * Same arguments and result as olap_topk_async, but without a context: the
 * working memory is a fixed 2 MiB array built into the library, which stays
 * on every GPU that has loaded it until the process exits.  Apart from the
 * first call on a device (below), a call makes no cudaMalloc/cudaFree and no
 * other allocation.
 *   - Limits: n <= OLAP_NOALLOC_MAX_N and k <= OLAP_NOALLOC_MAX_K.
 *   - OLAP_E_INVALID, returned before anything is launched, means one of:
 *     n or k above those limits; an unknown key type or order; d_keys NULL
 *     with n > 0; an output pointer NULL with min(k, n) > 0; d_keys not
 *     aligned to its key width.  OLAP_E_CUDA means a CUDA call failed (no
 *     current device, the set-up below, or the launch).
 *   - Runs on the current CUDA device, on `stream` (NULL = legacy default).
 *   - The first call on a device does a one-time set-up with that device
 *     current: it looks up the array's device address, which makes CUDA load
 *     the array's code module on that device if it is not loaded yet (lazy
 *     module loading is CUDA's default).  That load takes the array's 2 MiB of
 *     device memory and may synchronise the device, so make the first call on
 *     each device during start-up, before any stream capture; later calls
 *     allocate nothing.
 *   - All calls on a device share the one array and it keeps the previous
 *     call's contents (the library clears what must start at zero).  Calls
 *     whose work overlaps on the GPU race on it: order them on one stream.
 * ------------------------------------------------------------------------ */
#define OLAP_NOALLOC_MAX_N (1ull << 24)
#define OLAP_NOALLOC_MAX_K 4096ull
olap_status olap_topk_noalloc(const void* d_keys, olap_key_type type, const uint32_t* d_rowids,
                              uint64_t n, uint64_t k, olap_order order, void* d_out_keys,
                              uint32_t* d_out_rowids, int32_t* dev_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OLAP_H */
