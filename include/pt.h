/*
 * pt.h -- C ABI of the B300 predicate-transfer library (libpt.so).
 *
 * Predicate transfer (Yang, Zhao, Yu, Koutris, "Predicate Transfer:
 * Efficient Pre-Filtering on Multi-Join Queries", CIDR 2024) pre-filters
 * the tables of a multi-join query before the joins run.  Each table is a
 * vertex of the join graph, each equi-join an edge (Section 3.1).  Edges
 * are pointed from the smaller table to the bigger one (Section 3.2,
 * "Predicate Transfer Graph"); a forward pass visits the tables in
 * topological order and a backward pass repeats it over the reversed edges
 * (Section 3.2, "Transfer Schedule", Fig. 3).  Visiting a table scans its
 * join-key columns once: a row survives if its local predicate holds (a
 * selection bitmap here) and every incoming Bloom filter accepts its key;
 * the survivors' keys are inserted into one new Bloom filter per outgoing
 * edge (Section 3.2, "Filter Transformation", Fig. 2).
 *
 * Everything a run computes is done by CUDA kernels on one GPU; there is
 * no CPU fallback.  All functions return a pt_status; none throws.  On an
 * error, pt_last_error() holds a one-line message.  Device work is
 * enqueued on the context's stream and is asynchronous unless a function
 * says otherwise; errors of asynchronous work surface at the next call
 * that synchronizes (pt_get_*).
 *
 * Filter specification (the paper names Apache Arrow's filter but fixes
 * no layout; this library fixes one):
 *   key     int32 values are sign-extended to 64 bits; int64 taken as is.
 *   hash    H(x) = mix(x ^ seed + 0x9E3779B97F4A7C15) with mix() the
 *           SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014);
 *           a two-column key hashes as H(a, b) = mix(H(a) ^ b).
 *   layout  nblocks blocks of block_bits (256 or 512) bits, stored as
 *           uint32 words; block j is words [j*block_bits/32, ...), bit t of
 *           a block is bit (t & 31) of word (t >> 5) of the block.
 *   bits    block j = ((h >> 32) * nblocks) >> 32; with lo = (uint32)h,
 *           h1 = lo mod block_bits, h2 = (lo >> 16) | 1, a key sets bits
 *           (h1 + i*h2) mod block_bits for i = 0 .. k-1.
 *   size    nblocks = max(1, ceil(min(c, n_probe) * bits_per_key /
 *           block_bits)), c = survivors of the visit that builds the
 *           filter, n_probe = rows of the table at the edge's other end.
 * Bitmaps are uint32[ceil(n/32)]: row r is bit (r & 31) of word r >> 5;
 * bits at and beyond n are zero in every bitmap the library writes.
 */
#ifndef PT_H
#define PT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx; /* opaque, owned by the library */

typedef enum {
    PT_OK = 0,
    PT_ERR_INVALID = 1,     /* bad argument, malformed graph, out-of-range id */
    PT_ERR_OOM = 2,         /* device or host allocation failed */
    PT_ERR_CUDA = 3,        /* a CUDA call failed (message in pt_last_error) */
    PT_ERR_STATE = 4,       /* call out of order (e.g. run before pt_plan) */
    PT_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    PT_ERR_UNSUPPORTED = 6  /* valid request the library does not implement */
} pt_status;

typedef enum { PT_I32 = 0, PT_I64 = 1 } pt_dtype;

/* where a buffer passed to the library lives */
typedef enum { PT_MEM_DEVICE = 0, PT_MEM_HOST = 1 } pt_mem;

typedef struct {
    int32_t bits_per_key; /* 1..64; bits of filter per expected key */
    int32_t k;            /* 1..16; bits set per key */
    int32_t block_bits;   /* 256 or 512 */
    int32_t reserved;     /* must be 0 */
    uint64_t seed;        /* hash seed, XORed into every key */
} pt_filter_cfg;

typedef struct {
    const void* data; /* n_rows values; device pointer (PT_MEM_DEVICE, borrowed,
                         must stay valid and unchanged while runs use it) or
                         host pointer (PT_MEM_HOST, copied in; pinned memory
                         makes the copy asynchronous) */
    int32_t dtype;    /* pt_dtype */
    int32_t mem;      /* pt_mem */
} pt_column;

/* An equi-join t0.c0[i] = t1.c1[i] for i < ncols (ncols = 1, or 2 for a
 * composite key).  Column indexes refer to pt_register_table's list.
 * flags: 0, or PT_EDGE_ONE_WAY for the edge of a left outer join t0 LEFT
 * JOIN t1 (Section 3.4, "Supporting More Operators"): filters flow only from
 * t0 to t1, so t1 never removes a row of t0.  The edge then transfers in
 * the one pass that orients it from t0 to t1 (the forward pass when t0 is
 * the smaller table, else the backward pass) and builds no filter in the
 * other (pt_get_filter reports 0 blocks there).  A right outer join is the
 * same edge with t0 and t1 swapped; a full outer join has no edge.  Other
 * bits are rejected with PT_ERR_UNSUPPORTED. */
enum { PT_EDGE_ONE_WAY = 1 };
typedef struct {
    int32_t t0;
    int32_t ncols;
    int32_t c0[2];
    int32_t t1;
    int32_t c1[2];
    uint32_t flags;
} pt_edge;

/* Per-visit accounting, read back after a pass (see pt_get_visit_stats). */
typedef struct {
    int64_t n_rows;
    int64_t survivors;     /* popcount of the visit's survivor bitmap */
    int64_t probe_sectors; /* 32-byte key sectors read by the probes: per probed
                              column, sectors holding a row still alive when
                              that column's edge is probed */
    int64_t build_sectors; /* per distinct build column, sectors holding a survivor */
    int64_t filter_bytes;  /* bytes of the outgoing filters built by the visit */
    int32_t n_in;          /* incoming edges in this pass */
    int32_t n_out;         /* outgoing edges in this pass */
    int32_t has_input_bitmap;
    int32_t first_probe;   /* 1: the visit's first probe ran as its own pass
                              (pt_set_first_probe) */
    int64_t first_probe_sectors; /* the part of probe_sectors that pass read */
} pt_visit_stats;

/* Version of this ABI: (major << 16) | minor. */
uint32_t pt_abi_version(void);

/* Create a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t that all device work of the context is enqueued on; NULL
 * makes the context create (and own) a non-blocking stream.  cfg is
 * copied.  Errors: PT_ERR_INVALID (cfg out of range), PT_ERR_CUDA. */
pt_status pt_create(pt_ctx** out, const pt_filter_cfg* cfg, void* cuda_stream);

/* Free every buffer the context owns (filters, bitmaps, row ids, copies of
 * host columns) after waiting for its stream.  NULL is a no-op. */
pt_status pt_destroy(pt_ctx* ctx);

/* Register a table (a vertex of the join graph, Section 3.1): n_rows rows
 * (0 <= n_rows < 2^31) and n_cols (1..16) key columns.  sel is the local
 * predicate's result as a bitmap (layout above) in memory sel_mem, or NULL
 * for "every row".  Device buffers are borrowed; host buffers are copied to
 * library-owned device memory on the context's stream.  *table_id receives
 * ids 0, 1, 2 ... in registration order.  Only before pt_plan. */
pt_status pt_register_table(pt_ctx* ctx, int64_t n_rows, int32_t n_cols, const pt_column* cols,
                            const uint32_t* sel, int32_t sel_mem, int32_t* table_id);

/* Replace the column data and selection of a registered table (same n_rows,
 * same column count and dtypes).  Host buffers are copied again on the
 * context's stream; device buffers are re-borrowed.  Allowed after pt_plan:
 * the next run uses the new data. */
pt_status pt_update_table(pt_ctx* ctx, int32_t table_id, const pt_column* cols, const uint32_t* sel,
                          int32_t sel_mem);

/* Set the join graph: n_edges (0..64) equi-join edges.  Both sides of an
 * edge need the same number of columns; int32 and int64 columns may be
 * joined (values compare after sign extension).  Only before pt_plan. */
pt_status pt_set_join_graph(pt_ctx* ctx, int32_t n_edges, const pt_edge* edges);

/* Build the transfer schedule (Section 3.2): each edge points from the
 * table with fewer rows to the one with more (ties: lower table id first),
 * which makes a DAG; tables are visited in ascending (rows, id) order in the
 * forward pass and in the reverse order in the backward pass.  Allocates
 * all device memory a run needs.  order_out (nullable, n_tables entries)
 * receives the forward visiting order; mem_bytes_out (nullable) the bytes
 * of device memory allocated.  Errors: PT_ERR_OOM (also forced, without any
 * device allocation, when the environment variable PT_INJECT_OOM is "1"),
 * PT_ERR_INVALID. */
pt_status pt_plan(pt_ctx* ctx, int32_t* order_out, int64_t* mem_bytes_out);

/* The schedule pt_plan builds (only before pt_plan).
 *
 * PT_SCHEDULE_TRANSFER (default): predicate transfer, a forward and a
 * backward pass over the transfer DAG (Section 3.2): a table's outgoing
 * filters hold the keys of the rows that survived its incoming ones.
 *
 * PT_SCHEDULE_ONE_HOP: the Bloom join of Section 2.1, a one-hop transfer in
 * one direction.  Each edge's filter is built from its builder's selected
 * rows only (its local predicate) and probed by the other end; nothing is
 * transferred further.  The builder is the edge's smaller table (the DAG's
 * orientation), or t0 for a PT_EDGE_ONE_WAY edge.  Pass 0 ("forward") builds
 * every filter: its visits are the tables with an outgoing edge, and their
 * pass-0 survivors are their selections.  Pass 1 ("backward") probes: every
 * table starts from its selection and keeps the rows all its incoming
 * filters accept.  pt_get_survivors returns pass 1's result; pt_get_filter
 * and pt_get_pass_survivors take pass 0 for what the builders built and
 * pass 1 for the probes.  Only pt_run_transfer / pt_run_forward /
 * pt_run_backward follow it (a pt_server always transfers).  Returns
 * PT_ERR_STATE after pt_plan. */
enum { PT_SCHEDULE_TRANSFER = 0, PT_SCHEDULE_ONE_HOP = 1 };
pt_status pt_set_schedule(pt_ctx* ctx, int32_t schedule);

/* Forward pass: visit every table in topological order of the transfer
 * graph; a visit's input is its selection bitmap.  Asynchronous. */
pt_status pt_run_forward(pt_ctx* ctx);

/* Backward pass over the reversed edges; a visit's input is the table's
 * forward survivors (Section 3.2, Fig. 3).  Requires a completed
 * pt_run_forward since the last pt_update_table.  Asynchronous. */
pt_status pt_run_backward(pt_ctx* ctx);

/* pt_run_forward then pt_run_backward as one call.  When the context's
 * graph mode is on (pt_set_graph_mode), the first call captures both
 * passes into a CUDA graph and later calls replay it.  Results equal the
 * two separate calls; one launch fewer per table whose backward visit
 * probes nothing (its forward survivors pass through): its forward scan
 * zeroes that visit's filters of the previous run and its backward insert
 * counts the build sectors, so no scan-kind kernel launches for it. */
pt_status pt_run_transfer(pt_ctx* ctx);

/* 1 = capture the transfer into a CUDA graph on first pt_run_transfer and
 * replay it afterwards; 0 = launch kernels directly (default). */
pt_status pt_set_graph_mode(pt_ctx* ctx, int32_t on);

/* Copy the survivors of table_id after the last completed pass (backward
 * if it ran, else forward) into bitmap_out (ceil(n/32) words, host or
 * device memory) and their number into *count_out (either pointer may be
 * NULL).  Synchronizes the context's stream. */
pt_status pt_get_survivors(pt_ctx* ctx, int32_t table_id, uint32_t* bitmap_out, int64_t* count_out);

/* Same for a given pass (0 = forward, 1 = backward).  PT_ERR_INVALID for a
 * table the pass does not visit (pass 0 of PT_SCHEDULE_ONE_HOP visits the
 * builders only). */
pt_status pt_get_pass_survivors(pt_ctx* ctx, int32_t pass, int32_t table_id, uint32_t* bitmap_out,
                                int64_t* count_out);

/* Copy the filter built on edge edge_id in pass (0/1) into words_out
 * (nblocks*block_bits/32 words, host or device; NULL = size only) and its
 * size in blocks into *nblocks_out.  Synchronizes the context's stream. */
pt_status pt_get_filter(pt_ctx* ctx, int32_t pass, int32_t edge_id, uint32_t* words_out,
                        int64_t* nblocks_out);

/* Join phase (Section 3.3, "unified query plan": the join runs on the
 * reduced tables): the number of tuples in the join of every registered
 * table's survivors after the latest pass (uint64, mod 2^64), counted on
 * the device without building a tuple.  The join graph must be acyclic (a
 * forest) and of inner joins: each tree is rooted at its largest table,
 * and bottom-up each child's rows are summed per key into a device hash
 * table, by which each parent row's weight is multiplied; a tree's count
 * is its root's weight sum and the join's is their product.  The transfer
 * keeps every row that takes part in the join, so this equals the count
 * over the unreduced selected rows.  Errors: PT_ERR_STATE before a pass
 * has run; PT_ERR_UNSUPPORTED for a cycle or a one-way edge; PT_ERR_OOM
 * when the temporary device memory (8 bytes per row plus the hash table)
 * cannot be allocated; PT_ERR_TIMEOUT if a wait on a hash-table slot runs
 * out (the kernel then stops; the context stays usable).  Synchronizes. */
pt_status pt_join_count(pt_ctx* ctx, uint64_t* count_out);

/* Accounting of one visit of the last run of that pass.  PT_ERR_INVALID for
 * a table the pass does not visit.  Synchronizes. */
pt_status pt_get_visit_stats(pt_ctx* ctx, int32_t pass, int32_t table_id, pt_visit_stats* out);

/* Launch shape of the scan kernel: threads per CTA (64..256, multiple of
 * 32), shared-memory filter budget per CTA in bytes (0 = probe every filter
 * from L2), and CTAs per SM to aim for (0 = as many as fit).  Takes effect
 * at the next run; invalidates a captured graph. */
pt_status pt_set_launch(pt_ctx* ctx, int32_t threads, int32_t smem_filter_bytes, int32_t ctas_per_sm);

/* Thread-block clusters of the scan: an incoming filter too large for one
 * CTA's shared-memory budget is spread over the CTAs of a cluster (block j
 * held by CTA j mod C) and probed through distributed shared memory.
 * max_cluster is 1 (off, the default: on B300 the remote probes measured
 * slower than probes through L1/L2), 2 or 4.  Takes effect at the next run. */
pt_status pt_set_cluster(pt_ctx* ctx, int32_t max_cluster);

/* First-probe passes (on by default).  A forward-pass visit of a table
 * without a selection bitmap, with incoming edges and at least 2^20 rows,
 * starts with every row alive; its first probe in probe order is then a
 * plain stream over that edge's key column(s), run as a separate kernel
 * with twice the resident warps of the scan kernel.  It writes the rows
 * that pass as a bitmap, and the scan kernel runs the visit's other probes
 * on it.  Results and sector accounting are the same either way; enable = 0
 * keeps every probe in the scan kernel.  Takes effect at the next run. */
pt_status pt_set_first_probe(pt_ctx* ctx, int32_t enable);

/* Programmatic dependent launches (on by default): a visit's scan (or list
 * probe) and insert are launched so that each may start while the kernel
 * before it on its stream ends; every such kernel first waits on the device
 * for that kernel's results (griddepcontrol.wait).  Results are the same
 * either way.  Not used in runs timed by pt_set_kernel_timing.  Takes effect
 * at the next run. */
pt_status pt_set_dependent_launch(pt_ctx* ctx, int32_t enable);

/* Early scans (off by default; only with first-probe passes and
 * PT_ORDER_LEVEL_LIP).  When a visit with a first-probe pass has incoming
 * filters from builders below its highest builder level besides the one its
 * first-probe pass takes, the probes of those filters run as a scan of their
 * own right after the first-probe pass, while the higher-level builders
 * still run; the visit's scan then probes the highest level's filters only.
 * The probe order, survivors, filters and sector accounting are unchanged.
 * Off by default: on the snowflake benchmark the early scan competes with
 * the higher-level builders' gathers and the step is slower.  Takes effect
 * at the next run. */
pt_status pt_set_early_scan(pt_ctx* ctx, int32_t enable);

/* Order in which a visit probes its incoming filters (Section 3.2,
 * "Transfer Schedule": LIP-style ordering of the incoming filters is an
 * optional optimization).  PT_ORDER_LEVEL_LIP (default): ascending level of
 * the building visit in the pass's DAG, then ascending c_b / n_b (the
 * building visit's survivors over its table's rows), then edge id -- the
 * first filter then exists early, so a first-probe pass can start before
 * the visit's higher-level builders finish.  PT_ORDER_LIP: c_b / n_b, then
 * edge id.  PT_ORDER_EDGE: edge id (unordered).  Survivors and filters never
 * depend on it; the key sectors a visit reads (pt_visit_stats) do.  Takes
 * effect at the next run. */
enum { PT_ORDER_LEVEL_LIP = 0, PT_ORDER_LIP = 1, PT_ORDER_EDGE = 2 };
pt_status pt_set_probe_order(pt_ctx* ctx, int32_t order);

/* CTAs per SM of a first-probe pass (1..3; 0 = as many as fit, the
 * default).  A first-probe pass over a large table keeps its CTAs resident
 * until it ends; with fewer per SM, the kernels of the visits that run
 * beside it (every kernel of a visit fits in the room one first-probe CTA
 * leaves) start on the same SMs instead of waiting for it.  Results do not
 * depend on it.  Takes effect at the next run; invalidates a captured graph. */
pt_status pt_set_first_probe_ctas(pt_ctx* ctx, int32_t ctas_per_sm);

/* Streams the visits of one DAG level are spread over: 1..3 (default 3,
 * visits of a level and a first-probe pass beside its visit's builders run
 * concurrently).  1 runs every launch one after another on one stream, so
 * that kernel timing (pt_set_kernel_timing) measures each kernel alone.
 * Results do not depend on it.  Takes effect at the next run. */
pt_status pt_set_streams(pt_ctx* ctx, int32_t streams);

/* Kernel timing.  pt_set_kernel_timing(ctx, 1) records CUDA events around
 * every first-probe launch, every scan (probe + compact) launch and every
 * visit's size/clear + insert pair, on the stream each runs on.  Direct
 * launches accumulate from the moment timing is switched on.  In graph mode
 * the events are part of the captured graph (external event-record nodes;
 * switching timing recaptures), so their values are those of the most
 * recent replay.  pt_get_kernel_time returns the summed milliseconds and
 * counts of the probe phase (first-probe and scan launches) and of the
 * build phase (size/clear + insert pairs); pt_get_kernel_times returns the
 * three kinds apart.  Both synchronize the context's stream. */
typedef struct {
    double first_ms;        /* first-probe launches */
    double scan_ms;         /* scan launches */
    double build_ms;        /* size/clear + insert pairs */
    int32_t first_launches;
    int32_t scan_launches;
    int32_t build_pairs;
    int32_t reserved;
} pt_kernel_times;
pt_status pt_set_kernel_timing(pt_ctx* ctx, int32_t on);
pt_status pt_get_kernel_time(pt_ctx* ctx, double* scan_ms, int32_t* scan_launches, double* other_ms,
                             int32_t* other_launches);
pt_status pt_get_kernel_times(pt_ctx* ctx, pt_kernel_times* out);

/* The same events one launch at a time, in the order they were enqueued:
 * kind (0 scan, 1 size/clear + insert pair, 2 first probe), the pass and
 * the table of the visit, the start relative to the first timed launch
 * and the duration, both in milliseconds.  With graph mode on, the last
 * replay's; else every direct launch since timing was switched on.  Writes
 * at most max entries and sets *n to the number there are.  Synchronizes
 * the context's stream. */
typedef struct {
    int32_t kind;
    int32_t pass;
    int32_t table;
    int32_t reserved;
    double start_ms;
    double ms;
} pt_launch_time;
pt_status pt_get_launch_times(pt_ctx* ctx, int32_t max, pt_launch_time* out, int32_t* n);

/* Number of kernels the library launched since the context was created
 * (a graph replay counts each of its kernel nodes). */
pt_status pt_get_launch_count(pt_ctx* ctx, int64_t* launches);

/* Host-only planner, usable without a GPU: orient the edges of a join
 * graph of n_tables tables with the given row counts (src_out/dst_out,
 * n_edges entries), the forward visiting order (order_out, n_tables) and
 * each table's forward level (level_out, n_tables; longest path from a
 * source, so tables of one level are independent). */
pt_status pt_plan_graph(int32_t n_tables, const int64_t* n_rows, int32_t n_edges, const pt_edge* edges,
                        int32_t* src_out, int32_t* dst_out, int32_t* order_out, int32_t* level_out);

/* ---- serving: resident tables, continuous batching ------------------------
 * A server keeps tables resident in device memory and runs many transfer
 * queries over them.  A query names up to 6 table instances (one use of a
 * resident table with its own selection bitmap; the same table may appear
 * more than once, as an alias) and up to 8 equi-join edges between
 * instances (pt_edge with t0/t1 = instance indexes, c0/c1 = column indexes
 * of those instances' tables).  Its transfer is the forward and backward
 * pass of Section 3.2 over its instances, with the filter specification
 * above; the survivor bitmaps equal those of a planned context on the same
 * tables, selections and edges.
 *
 * A scheduler thread admits waiting queries in arrival order while their
 * device memory (bitmaps, filters, row ids, selection copies) fits the
 * arena, groups up to max_batch of them and runs the group as one batch:
 * per pass and per DAG level, one scan, one size/clear and one insert
 * launch over the visits of every query in the batch, replayed from a CUDA
 * graph.  Up to max_inflight (1..4) batches run at once; queries that
 * arrive meanwhile join the next batch as soon as a slot and memory free
 * up.  max_batch = max_inflight = 1 runs one query at a time.
 *
 * Resident key columns are each stored next to a column of their hashes,
 * computed once by pt_server_start.  Results stay in device memory until
 * pt_server_release.  Functions are thread-safe except that a ticket must
 * not be released while another thread reads its survivors. */
typedef struct pt_server pt_server;

/* Create a server on the current device with an arena of arena_bytes of
 * device memory for queries. */
pt_status pt_server_create(pt_server** out, const pt_filter_cfg* cfg, int64_t arena_bytes, int32_t max_batch,
                           int32_t max_inflight);

/* Register a resident table (before pt_server_start).  Device columns are
 * borrowed and must stay valid; host columns are copied. */
pt_status pt_server_register_table(pt_server* srv, int64_t n_rows, int32_t n_cols, const pt_column* cols,
                                   int32_t* table_id);

/* Compute the hash columns, allocate the batch descriptors and start the
 * scheduler.  Synchronous. */
pt_status pt_server_start(pt_server* srv);

/* Submit a query.  table_ids[i] is instance i's resident table;
 * sel_bitmaps (nullable, or NULL entries = every row) are selection bitmaps
 * in memory sel_mem: host bitmaps are copied before returning, device
 * bitmaps (16-byte aligned) are borrowed until the query is done. */
pt_status pt_server_submit(pt_server* srv, int32_t n_inst, const int32_t* table_ids, const uint32_t* const* sel_bitmaps,
                           int32_t sel_mem, int32_t n_edges, const pt_edge* edges, uint64_t* ticket);

/* *done = 1 once the query finished; *result is its status. */
pt_status pt_server_poll(pt_server* srv, uint64_t ticket, int32_t* done, pt_status* result);

/* Block until the query finished. */
pt_status pt_server_wait(pt_server* srv, uint64_t ticket, pt_status* result);

/* Final (backward-pass) survivors of instance inst: bitmap into bitmap_out
 * (host or device, nullable) and count into *count_out (nullable). */
pt_status pt_server_survivors(pt_server* srv, uint64_t ticket, int32_t inst, uint32_t* bitmap_out, int64_t* count_out);

/* Free a finished query's device memory and forget its ticket. */
pt_status pt_server_release(pt_server* srv, uint64_t ticket);

/* Latency percentiles (submit to completion) and throughput of the queries
 * completed since creation or the last pt_server_reset_stats. */
pt_status pt_server_stats(pt_server* srv, double* p50_ms, double* p99_ms, double* qps, int64_t* completed);
pt_status pt_server_reset_stats(pt_server* srv);

/* Stop the scheduler (after in-flight batches finish) and free everything. */
pt_status pt_server_destroy(pt_server* srv);

/* ---- one visit without any allocation ------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: engines that give all device memory
 * to their own pool up front, paths where an allocation (which can
 * synchronize the device) is not acceptable, and services that must not
 * meet an out-of-memory error in the middle of a query.  pt_visit_static
 * runs one visit of a table -- probe, survivor bitmap, compaction,
 * size/clear and insert -- with every input and output supplied by the
 * caller.  Its scratch (compacted
 * row ids, per-warp segment lengths, counters) is a fixed array of about
 * 4.1 MB that is part of the library's device image: every GPU that loads
 * the library holds it until the process exits, and nothing is allocated
 * per call.
 *
 * Limits and rules:
 *   - n_rows <= PT_STATIC_MAX_ROWS; larger visits return PT_ERR_INVALID.
 *   - All calls share the one scratch array: calls whose work overlaps on
 *     the GPU (different streams without ordering, or different host
 *     threads) race and give wrong results.  Calls on one stream are safe.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture.
 *   - The survivor count and sector counters are zeroed at the start of
 *     every call; nothing else carries over between calls.
 * Incoming filters are probed in the order given.  Key columns, filters and
 * bitmaps are device memory; filters 16-byte aligned.  Asynchronous on
 * cuda_stream; errors are reported through pt_last_error(NULL). */
#define PT_STATIC_MAX_ROWS (1 << 20)

typedef struct {
    pt_column col[2];       /* this table's key column(s) on the edge (device) */
    int32_t ncols;          /* 1 or 2 */
    int32_t reserved;
    const uint32_t* filter; /* the incoming filter's words (device) */
    const int64_t* nblocks; /* its size in blocks (device) */
} pt_static_probe;

typedef struct {
    pt_column col[2];       /* this table's key column(s) on the edge (device) */
    int32_t ncols;          /* 1 or 2 */
    int32_t reserved;
    uint32_t* filter;       /* output filter words (device, capacity_blocks*block_bits/32) */
    int64_t capacity_blocks;/* must cover the size rule for n_rows survivors */
    int64_t probe_rows;     /* rows of the table at the edge's other end */
    int64_t* nblocks_out;   /* device: blocks the filter uses */
} pt_static_build;

/* in_bits: input bitmap (device, NULL = every row); out_bits: survivor
 * bitmap (device, ceil(n_rows/32) words); count_out: device int64 that
 * receives the survivor count (nullable). */
pt_status pt_visit_static(const pt_filter_cfg* cfg, void* cuda_stream, int64_t n_rows, const uint32_t* in_bits,
                          int32_t n_in, const pt_static_probe* in, int32_t n_out, const pt_static_build* out,
                          uint32_t* out_bits, int64_t* count_out);

/* Message of the last failed call on ctx (or, when ctx is NULL, of the last
 * failed call that has no context: pt_create, pt_plan_graph, pt_server_*,
 * pt_visit_static).  Valid until the next call on ctx. */
const char* pt_last_error(pt_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
