// Host runtime and C ABI of libpt (declared in include/pt.h).
//
// The runtime keeps the registered tables and the join graph, builds the
// transfer schedule (Section 3.2 of the paper: size-ordered edges, one
// forward and one backward pass), lays out every buffer a run needs in one
// device allocation, and enqueues the kernels of each visit (a first-probe
// pass where it applies, the scan, the insert) on the context's streams.  No step of a run executes on the host: filter sizes
// depend on survivor counts that only the device knows, so they are
// computed by a kernel and no host synchronization happens between visits.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pt.h"
#include "pt_internal.h"

namespace {

thread_local std::string g_err;

constexpr size_t kAlign = 256;
constexpr int kMaxTables = 64;
constexpr int kMaxEdges = 64;
constexpr int kMaxCols = 16;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Col {
    const void* dev = nullptr;
    int32_t dtype = 0;
    void* owned = nullptr;  // device copy of a host column
};

struct Table {
    int64_t n = 0;
    std::vector<Col> cols;
    const uint32_t* sel = nullptr;
    void* sel_owned = nullptr;
};

// Launch shape of one visit's scan.
struct ScanShape {
    int grid = 1, block = 256;
    int cluster = 1;         // CTAs per cluster (filters too large for one CTA spread over the cluster)
    size_t smem = 0;         // dynamic shared memory: filters + per-warp queues
    size_t filter_smem = 0;  // the filters' part
    int words_per_warp = 4, total_warps = 8;
};

struct Visit {
    int table = 0;
    std::vector<int> in_edges, out_edges;
    std::vector<int> bcols;  // distinct build columns
    int64_t max_in_filter_bytes = 0;     // sum over incoming edges of the filters' largest sizes
    int64_t max_single_filter_bytes = 0; // the largest of them
    ScanShape shape;
    // a first-probe pass (every row alive, large table): its launch shape
    bool first = false;
    int first_grid = 0;
    size_t first_smem = 0;
    // a pair of first-probe launches, with and without the shared-memory budget
    // (an incoming filter may outgrow the budget); the second one's grid
    bool first_pair = false;
    int first_grid0 = 0;
    // an early scan (after the first-probe pass, of the other incoming edges whose
    // builders are below early_level, the highest builder level of the visit)
    bool early = false;
    int32_t early_level = 0;
    // a backward visit over the forward survivor list: its launch shape
    bool list = false;
    // a backward visit that probes nothing (a source of the reversed DAG): its
    // survivors, row ids and segment counts are its forward ones (aliased), no
    // scan runs, and its builds read the forward count
    bool pass_through = false;
    int list_grid = 0;
    size_t list_smem = 0;
};

}  // namespace

struct pt_ctx {
    pt::FilterCfg fcfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;

    std::vector<Table> tables;
    std::vector<pt_edge> edges;
    bool graph_set = false;
    bool planned = false;

    std::vector<int32_t> src, dst, order, level;
    std::vector<Visit> visits[2];
    int schedule = PT_SCHEDULE_TRANSFER;
    // [pass][edge]: the table that builds the edge's filter in that pass and
    // the one that probes it (-1: not built in that pass)
    std::vector<int32_t> bld[2], prb[2];
    int fpass[2] = {0, 1};  // the pass whose filters (and builders' counts) pass p probes

    void* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<uint32_t*> surv[2];
    std::vector<uint32_t*> ids[2], seg[2];  // [pass][table]: survivors' row ids in segments, and counts
    std::vector<uint64_t*> hfwd;            // [edge]: the forward builder's key hash of each of its survivors
    std::vector<bool> has_edge;             // [table]
    std::vector<int> vidx[2];               // [pass][table]: index into visits[pass]
    std::vector<uint32_t*> filt[2];
    std::vector<int64_t> filt_max_words;
    unsigned long long* counts[2] = {nullptr, nullptr};  // [table]
    unsigned long long* stats[2] = {nullptr, nullptr};   // [table][3]
    int32_t* first_idx = nullptr;                        // [table]: edge the first-probe pass tested
    std::vector<uint32_t*> mid;                          // [table]: its survivors, or nullptr
    std::vector<uint32_t*> mid2;                         // [table]: the early scan's survivors, or nullptr
    unsigned long long* early_count[2] = {nullptr, nullptr};  // [table]: the early scan's survivor count
    bool first_probe = true;                             // run first-probe passes where they apply
    bool early_scan = false;                             // run early scans where they apply
    bool pdl = true;                                     // programmatic dependent launches (scan, list, insert)
    int first_ctas = 0;                                  // first-probe CTAs per SM (0: as many as fit)
    bool first_pair = true;                              // pairs of first-probe launches (with / without smem)
    int64_t* nblocks[2] = {nullptr, nullptr};            // [edge]
    void* meta[2] = {nullptr, nullptr};
    size_t meta_bytes = 0;
    bool in_transfer = false;  // set while a transfer run enqueues both passes (see InTransfer)
    bool chain_ok = false;     // every backward visit's table has a forward visit (pt_plan)
    int insert_fit = 4;         // resident 256-thread insert CTAs per SM (prepare_shapes)
    int64_t seg_cap = 0;

    int scan_threads = 256;
    int smem_budget = 40 * 1024;  // more shared memory means less L1 for the filters probed through it
    int max_cluster = 1;  // 1: no clusters (remote probes measured slower than L2 ones)
    int streams = 3;      // visits of a level spread over this many streams (1: one after another)
    int ctas_per_sm = 0;
    int smem_attr_set[2] = {0, 0};
    int list_attr_set[2] = {0, 0};
    bool shapes_ready = false;

    int passes_done = 0;  // bit 0: forward, bit 1: backward

    bool graph_mode = false;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_kernels = 0;

    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    // events captured into the graph as external event nodes (graph mode with timing)
    bool capturing = false;
    bool graph_timed = false;
    std::vector<cudaEvent_t> gev;
    std::vector<int> gev_kind;
    size_t gev_used = 0;
    int64_t graph_replays = 0;

    int64_t launches = 0;
    std::string err;

    // Visits of one DAG level run concurrently: each visit is enqueued on one
    // of these streams and waits on the events of the visits that build its
    // incoming filters; every pass forks from and joins back into `stream`.
    static constexpr int kAux = 3;
    cudaStream_t aux[kAux] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> vev[2];  // per pass, per table: the visit's work is done
    cudaEvent_t pass_ev[2] = {nullptr, nullptr};
    std::vector<int> slot[2];         // per pass, per table: its stream (index into aux)
    std::vector<int32_t> lvl[2];      // per pass, per table: level (longest path from a source)
    // A first-probe pass runs on a stream of its own, as soon as the filters
    // of its visit's lowest-level builders exist (it probes one of those),
    // concurrently with the builders of the visit's other filters.
    std::vector<cudaStream_t> fstream;  // per table with a first-probe pass, else nullptr
    std::vector<cudaEvent_t> fev;       // its pass is done
    std::vector<cudaEvent_t> eev;       // and the early scan after it, where there is one
};

namespace {

pt_status fail(pt_ctx* ctx, pt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_err = buf;
    return st;
}

#define PT_CUDA(ctx, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail((ctx), PT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool rank_less(const std::vector<int64_t>& n, int a, int b) {
    if (n[a] != n[b]) return n[a] < n[b];
    return a < b;
}

pt_status check_edges(pt_ctx* ctx, int32_t n_tables, const std::vector<int>& n_cols,
                      const std::vector<std::vector<int32_t>>* dtypes, int32_t n_edges, const pt_edge* e) {
    if (n_edges < 0 || n_edges > kMaxEdges) return fail(ctx, PT_ERR_INVALID, "n_edges %d out of range", n_edges);
    if (n_edges > 0 && !e) return fail(ctx, PT_ERR_INVALID, "edges is NULL");
    for (int i = 0; i < n_edges; ++i) {
        const pt_edge& x = e[i];
        if (x.flags & ~(uint32_t)PT_EDGE_ONE_WAY) return fail(ctx, PT_ERR_UNSUPPORTED, "edge %d: unknown flags 0x%x", i, x.flags);
        if (x.ncols < 1 || x.ncols > 2) return fail(ctx, PT_ERR_INVALID, "edge %d: ncols %d", i, x.ncols);
        if (x.t0 < 0 || x.t0 >= n_tables || x.t1 < 0 || x.t1 >= n_tables)
            return fail(ctx, PT_ERR_INVALID, "edge %d: table id out of range", i);
        if (x.t0 == x.t1) return fail(ctx, PT_ERR_INVALID, "edge %d joins table %d with itself", i, x.t0);
        for (int j = 0; j < x.ncols; ++j) {
            if (x.c0[j] < 0 || x.c0[j] >= n_cols[x.t0] || x.c1[j] < 0 || x.c1[j] >= n_cols[x.t1])
                return fail(ctx, PT_ERR_INVALID, "edge %d: column index out of range", i);
        }
        (void)dtypes;
    }
    return PT_OK;
}

// Orientation, visiting order and levels (Section 3.2).
void plan_graph(const std::vector<int64_t>& n, const std::vector<pt_edge>& e, std::vector<int32_t>& src,
                std::vector<int32_t>& dst, std::vector<int32_t>& order, std::vector<int32_t>& level) {
    const int T = (int)n.size(), E = (int)e.size();
    src.assign(E, 0);
    dst.assign(E, 0);
    for (int i = 0; i < E; ++i) {
        if (rank_less(n, e[i].t0, e[i].t1)) {
            src[i] = e[i].t0;
            dst[i] = e[i].t1;
        } else {
            src[i] = e[i].t1;
            dst[i] = e[i].t0;
        }
    }
    order.resize(T);
    for (int i = 0; i < T; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank_less(n, a, b); });
    level.assign(T, 0);
    for (int v : order)  // ascending rank is a topological order: every edge goes up in rank
        for (int i = 0; i < E; ++i)
            if (src[i] == v) level[dst[i]] = std::max(level[dst[i]], level[v] + 1);
}

int64_t max_filter_words(int64_t n0, int64_t n1, const pt::FilterCfg& f) {
    const int64_t m = std::min(n0, n1);
    int64_t nb = (m * f.bits_per_key + f.block_bits - 1) / f.block_bits;
    if (nb < 1) nb = 1;
    return nb * (f.block_bits / 32);
}

void free_arena(pt_ctx* ctx) {
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    if (ctx->arena) {
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
    }
    ctx->arena_bytes = 0;
}

pt_status upload_table(pt_ctx* ctx, Table& t, int32_t n_cols, const pt_column* cols, const uint32_t* sel,
                       int32_t sel_mem, bool fresh) {
    for (int j = 0; j < n_cols; ++j) {
        const pt_column& c = cols[j];
        Col& d = t.cols[j];
        const size_t bytes = (size_t)t.n * (c.dtype == PT_I32 ? 4 : 8);
        if (c.mem == PT_MEM_HOST) {
            if (!d.owned && bytes > 0) {
                if (cudaMalloc(&d.owned, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    d.owned = nullptr;
                    return fail(ctx, PT_ERR_OOM, "device copy of a host column (%zu bytes)", bytes);
                }
            }
            if (bytes) PT_CUDA(ctx, cudaMemcpyAsync(d.owned, c.data, bytes, cudaMemcpyHostToDevice, ctx->stream));
            d.dev = d.owned;
        } else {
            d.dev = c.data;
        }
        d.dtype = c.dtype;
    }
    (void)fresh;
    const size_t sbytes = (size_t)((t.n + 31) / 32) * 4;
    if (sel && sel_mem == PT_MEM_HOST) {
        if (!t.sel_owned && sbytes) {
            if (cudaMalloc(&t.sel_owned, sbytes) != cudaSuccess) {
                cudaGetLastError();
                t.sel_owned = nullptr;
                return fail(ctx, PT_ERR_OOM, "device copy of a host selection bitmap");
            }
        }
        if (sbytes) PT_CUDA(ctx, cudaMemcpyAsync(t.sel_owned, sel, sbytes, cudaMemcpyHostToDevice, ctx->stream));
        t.sel = (const uint32_t*)t.sel_owned;
    } else {
        t.sel = sel;
    }
    return PT_OK;
}

pt_status check_columns(pt_ctx* ctx, int64_t n_rows, int32_t n_cols, const pt_column* cols, int32_t sel_mem) {
    if (n_cols < 1 || n_cols > kMaxCols) return fail(ctx, PT_ERR_INVALID, "n_cols %d out of range", n_cols);
    if (!cols) return fail(ctx, PT_ERR_INVALID, "cols is NULL");
    for (int j = 0; j < n_cols; ++j) {
        if (cols[j].dtype != PT_I32 && cols[j].dtype != PT_I64) return fail(ctx, PT_ERR_INVALID, "column %d: dtype %d", j, cols[j].dtype);
        if (cols[j].mem != PT_MEM_DEVICE && cols[j].mem != PT_MEM_HOST) return fail(ctx, PT_ERR_INVALID, "column %d: mem %d", j, cols[j].mem);
        if (n_rows > 0 && !cols[j].data) return fail(ctx, PT_ERR_INVALID, "column %d: data is NULL", j);
        if (cols[j].mem == PT_MEM_DEVICE && ((uintptr_t)cols[j].data % 16) != 0)
            return fail(ctx, PT_ERR_INVALID, "column %d: device data must be 16-byte aligned", j);
    }
    if (sel_mem != PT_MEM_DEVICE && sel_mem != PT_MEM_HOST) return fail(ctx, PT_ERR_INVALID, "sel_mem %d", sel_mem);
    return PT_OK;
}

// Shared memory one scan CTA may use when two share an SM (228 KB per SM,
// minus the kernel's static part).
constexpr int64_t kScanCtaSmem = 112 * 1024;
// Dynamic shared memory of a first-probe CTA: below the default 48 KB limit
// (which also covers the kernel's static shared memory), so no kernel
// attribute is needed.
constexpr int64_t kFirstCtaSmem = 46 * 1024;

// sparse: the visit's scan reads an input bitmap (the scan kernel without the
// dense path, which fits more CTAs per SM)
ScanShape scan_shape(pt_ctx* ctx, const Visit& vis, bool sparse) {
    ScanShape s{};
    const int64_t n = ctx->tables[vis.table].n;
    const int64_t n_words = (n + 31) / 32;
    s.block = ctx->scan_threads;
    const int warps_per_cta = s.block / 32;
    // after a first-probe pass the scan probes one edge fewer
    const int n_in = (int)vis.in_edges.size() - (vis.first && ctx->first_probe && sparse ? 1 : 0);
    const size_t queues = (size_t)warps_per_cta * pt::scan_warp_smem_bytes(n_in);
    int64_t budget = std::min<int64_t>(ctx->smem_budget, kScanCtaSmem - (int64_t)queues);
    budget = std::max<int64_t>(0, budget) / 16 * 16;
    // after a first-probe pass, no filter budget: the pass took the visit's first
    // filter; the others probe through L1, which the budget would shrink, and the
    // smaller CTAs start beside a first-probe pass that still holds the SMs
    // (measured on the benchmark: 0.502 -> 0.488 ms, the fact table's remaining
    // probes 75 -> 56 us, M's compaction 176 -> 151 us)
    const bool after_first = vis.first && ctx->first_probe && sparse;
    const int64_t want_filt = (vis.in_edges.empty() || after_first) ? 0 : std::min<int64_t>(budget, vis.max_in_filter_bytes);
    const size_t filt = (size_t)((want_filt + 15) / 16 * 16);
    s.smem = filt + queues;
    s.filter_smem = filt;
    // a cluster when some incoming filter may not fit one CTA's budget
    if (ctx->max_cluster > 1 && filt > 0 && vis.max_single_filter_bytes > (int64_t)filt) s.cluster = ctx->max_cluster;
    int fit = pt::scan_max_ctas_per_sm(ctx->fcfg.block_bits, s.block, s.smem, sparse);
    if (fit < 1) fit = 1;
    if (ctx->ctas_per_sm > 0) fit = std::min(fit, ctx->ctas_per_sm);
    int64_t max_grid = (int64_t)ctx->num_sms * fit;
    max_grid = std::max<int64_t>(s.cluster, max_grid / s.cluster * s.cluster);
    // at least a chunk each; a visit with an input bitmap takes no dense 32-word
    // sub-rounds, so its warps may take fewer words (more warps for a small table)
    const int64_t chunk = sparse ? pt::kSparseChunkWords : pt::kChunkWords;
    const int64_t want_warps = (n_words + chunk - 1) / chunk;
    int64_t grid = (want_warps + warps_per_cta - 1) / warps_per_cta;
    grid = (grid + s.cluster - 1) / s.cluster * s.cluster;
    grid = std::max<int64_t>(s.cluster, std::min(grid, max_grid));
    s.grid = (int)grid;
    s.total_warps = (int)(grid * warps_per_cta);
    int64_t wpw = (n_words + s.total_warps - 1) / s.total_warps;
    wpw = (wpw + chunk - 1) / chunk * chunk;
    if (wpw < chunk) wpw = chunk;
    s.words_per_warp = (int)wpw;
    return s;
}

// Survivor count of table v after pass p on the device (a pass-through
// backward visit's is its forward one).
unsigned long long* count_of(pt_ctx* ctx, int p, int v) {
    const bool through = p == 1 && ctx->vidx[1][v] >= 0 && ctx->visits[1][ctx->vidx[1][v]].pass_through;
    return ctx->counts[through ? 0 : p] + v;
}

pt::ColRef colref(const pt_ctx* ctx, int t, int c) {
    pt::ColRef r{};
    r.p = ctx->tables[t].cols[c].dev;
    r.dtype = ctx->tables[t].cols[c].dtype;
    return r;
}

// The arguments of visit `vis` in pass p.  A backward visit in list mode
// reads the forward survivors' row-id segments (and the hashes the forward
// inserts stored) instead of a bitmap, in the forward scan's segment
// geometry, which its own survivor segments keep.
void fill_visit_args(pt_ctx* ctx, int p, const Visit& vis, const ScanShape& sh, pt::VisitArgs& a) {
    std::memset(&a, 0, sizeof a);
    const int v = vis.table;
    a.n = ctx->tables[v].n;
    // the backward pass of a transfer starts from the forward survivors; every
    // other visit from the table's selection
    const bool one_hop = ctx->schedule == PT_SCHEDULE_ONE_HOP;
    a.in_bits = p == 0 || one_hop ? ctx->tables[v].sel : ctx->surv[0][v];
    a.out_bits = ctx->surv[p][v];
    a.count = count_of(ctx, p, v);
    a.stats = ctx->stats[p] + 3 * v;
    a.n_in = (int)vis.in_edges.size();
    a.n_out = (int)vis.out_edges.size();
    a.words_per_warp = sh.words_per_warp;
    a.total_warps = sh.total_warps;
    a.smem_words = (int32_t)(sh.filter_smem / 4);
    a.cluster = sh.cluster;
    a.insert_sizes = 1;
    if (p == 1 && vis.list) {
        const ScanShape& fs = ctx->visits[0][ctx->vidx[0][v]].shape;
        a.words_per_warp = fs.words_per_warp;
        a.total_warps = fs.total_warps;
        a.smem_words = (int32_t)(vis.list_smem / 4);
        a.cluster = 1;
        a.list_ids = ctx->ids[0][v];
        a.list_seg = ctx->seg[0][v];
    }
    for (int i = 0; i < a.n_in; ++i) {
        const int e = vis.in_edges[i];
        const pt_edge& ed = ctx->edges[e];
        const int32_t* cs = ed.t0 == v ? ed.c0 : ed.c1;
        const int fp = ctx->fpass[p];
        const int b = ctx->bld[fp][e];  // the table that built the filter
        pt::ProbeEdge& pe = a.in[i];
        pe.ncols = ed.ncols;
        pe.edge_id = e;
        pe.col[0] = colref(ctx, v, cs[0]);
        pe.col[1] = ed.ncols == 2 ? colref(ctx, v, cs[1]) : pe.col[0];
        pe.filter = ctx->filt[fp][e];
        pe.nblocks = ctx->nblocks[fp] + e;
        pe.build_count = count_of(ctx, fp, b);
        pe.build_rows = ctx->tables[b].n;
        pe.build_level = ctx->lvl[fp][b];
        // stored by the forward insert, unless this one-way edge built nothing forward
        if (p == 1 && vis.list && !((ed.flags & PT_EDGE_ONE_WAY) && ctx->src[e] != ed.t0)) pe.hin = ctx->hfwd[e];
    }
    for (int i = 0; i < a.n_out; ++i) {
        const int e = vis.out_edges[i];
        const pt_edge& ed = ctx->edges[e];
        const int32_t* cs = ed.t0 == v ? ed.c0 : ed.c1;
        const int other = ed.t0 == v ? ed.t1 : ed.t0;
        pt::BuildEdge& be = a.out[i];
        be.ncols = ed.ncols;
        be.edge_id = e;
        be.col[0] = colref(ctx, v, cs[0]);
        be.col[1] = ed.ncols == 2 ? colref(ctx, v, cs[1]) : be.col[0];
        be.filter = ctx->filt[p][e];
        be.nblocks = ctx->nblocks[p] + e;
        be.probe_rows = ctx->tables[other].n;
        if (p == 0 && !one_hop) be.hout = ctx->hfwd[e];
    }
    a.n_bcols = (int)vis.bcols.size();
    for (int i = 0; i < a.n_bcols; ++i) a.bcol[i] = colref(ctx, v, vis.bcols[i]);
    // every table with an edge keeps its forward survivors' ids (the backward
    // pass starts from them); backward ids are kept for its builds
    if (ctx->has_edge[v] && (p == 0 || a.n_out > 0 || vis.list)) {
        a.ids = ctx->ids[p][v];
        a.seg_count = ctx->seg[p][v];
    }
    // inside one transfer run, a table whose backward visit passes its forward
    // survivors through has no backward scan: its forward scan zeroes the
    // backward filters' previous words, and its backward insert counts the
    // build sectors
    if (ctx->in_transfer && ctx->schedule == PT_SCHEDULE_TRANSFER) {
        const int bv = ctx->vidx[1][v];
        const Visit* b = bv >= 0 ? &ctx->visits[1][bv] : nullptr;
        if (p == 0 && b && b->pass_through && a.n_out + (int)b->out_edges.size() <= pt::kMaxOut) {
            for (int e : b->out_edges) {
                pt::BuildEdge& be = a.out[a.n_out + a.n_clear_extra++];
                be.filter = ctx->filt[1][e];
                be.nblocks = ctx->nblocks[1] + e;
            }
        }
        if (p == 1 && vis.pass_through) a.insert_bsec = 1;
    }
}

// Compute every visit's scan shape and raise the kernels' dynamic shared
// memory limit; done before any capture (occupancy queries and function
// attributes are not stream work).
pt_status prepare_shapes(pt_ctx* ctx) {
    if (ctx->shapes_ready) return PT_OK;
    // the kernels' shared-memory limit first (occupancy queries depend on it)
    const int bi = ctx->fcfg.block_bits == 512 ? 1 : 0;
    if ((int)kScanCtaSmem > ctx->smem_attr_set[bi]) {
        PT_CUDA(ctx, pt::scan_set_smem_limit(ctx->fcfg.block_bits, kScanCtaSmem));
        ctx->smem_attr_set[bi] = (int)kScanCtaSmem;
    }
    ctx->insert_fit = std::max(1, pt::insert_max_ctas_per_sm(ctx->fcfg.block_bits, 256));
    for (int p = 0; p < 2; ++p)
        for (Visit& vis : ctx->visits[p]) {
            // an input bitmap: a transfer's backward visits, a selection, a first-probe pass
            const bool sparse = (p == 1 && ctx->schedule == PT_SCHEDULE_TRANSFER) ||
                                ctx->tables[vis.table].sel != nullptr || (vis.first && ctx->first_probe);
            vis.shape = scan_shape(ctx, vis, sparse);
        }
    if ((int)kScanCtaSmem > ctx->list_attr_set[bi]) {
        PT_CUDA(ctx, pt::probe_list_set_smem_limit(ctx->fcfg.block_bits, kScanCtaSmem));
        ctx->list_attr_set[bi] = (int)kScanCtaSmem;
    }
    for (Visit& vis : ctx->visits[1]) {
        if (!vis.list) continue;
        const ScanShape& fs = ctx->visits[0][ctx->vidx[0][vis.table]].shape;
        const int64_t want = vis.in_edges.empty() ? 0 : std::min<int64_t>(std::min<int64_t>(ctx->smem_budget, kScanCtaSmem),
                                                                         vis.max_in_filter_bytes);
        vis.list_smem = (size_t)(want / 16 * 16);
        const int wpc = pt::kListThreads / 32;
        vis.list_grid = std::max(1, (fs.total_warps + wpc - 1) / wpc);
    }
    for (int p = 0; p < 2; ++p)
        for (Visit& vis : ctx->visits[p]) {
            if (!vis.first) continue;
            // the filter budget of one CTA: the largest incoming filter, at most
            // the context's budget (a first filter that does not fit is probed from L2)
            const int64_t want = std::min<int64_t>(std::min<int64_t>(ctx->smem_budget, kFirstCtaSmem),
                                                   vis.max_single_filter_bytes);
            vis.first_smem = (size_t)(want / 16 * 16);
            int fit = pt::probe_first_max_ctas_per_sm(ctx->fcfg.block_bits, pt::kFirstThreads, vis.first_smem);
            if (fit < 1) fit = 1;
            if (ctx->first_ctas > 0) fit = std::min(fit, ctx->first_ctas);
            const int64_t tiles = (ctx->tables[vis.table].n + pt::kFirstTileRows - 1) / pt::kFirstTileRows;
            const int64_t want_ctas = (tiles + pt::kFirstThreads / 32 - 1) / (pt::kFirstThreads / 32);
            vis.first_grid = (int)std::max<int64_t>(1, std::min<int64_t>(want_ctas, (int64_t)ctx->num_sms * fit));
            vis.first_pair = ctx->first_pair && vis.first_smem > 0 && vis.max_single_filter_bytes > (int64_t)vis.first_smem;
            if (vis.first_pair) {
                int fit0 = pt::probe_first_max_ctas_per_sm(ctx->fcfg.block_bits, pt::kFirstThreads, 0);
                if (fit0 < 1) fit0 = 1;
                if (ctx->first_ctas > 0) fit0 = std::min(fit0, ctx->first_ctas);
                vis.first_grid0 = (int)std::max<int64_t>(1, std::min<int64_t>(want_ctas, (int64_t)ctx->num_sms * fit0));
            }
        }
    ctx->shapes_ready = true;
    return PT_OK;
}

// kind: 0 scan, 1 size/clear + insert, 2 first probe; the pass and table of
// the launch are kept beside it (kind | pass << 4 | table << 8).
pt_status record_event(pt_ctx* ctx, int kind, cudaStream_t st, int pass, int table) {
    if (!ctx->timing) return PT_OK;
    std::vector<cudaEvent_t>& ev = ctx->capturing ? ctx->gev : ctx->ev;
    std::vector<int>& kinds = ctx->capturing ? ctx->gev_kind : ctx->ev_kind;
    size_t& used = ctx->capturing ? ctx->gev_used : ctx->ev_used;
    if (used == ev.size()) {
        cudaEvent_t e;
        PT_CUDA(ctx, cudaEventCreate(&e));
        ev.push_back(e);
        kinds.push_back(0);
    }
    kinds[used] = kind | (pass << 4) | (table << 8);
    if (ctx->capturing)  // becomes an event-record node of the graph, recorded at every replay
        PT_CUDA(ctx, cudaEventRecordWithFlags(ev[used], st, cudaEventRecordExternal));
    else
        PT_CUDA(ctx, cudaEventRecord(ev[used], st));
    used++;
    return PT_OK;
}

pt_status enqueue_pass(pt_ctx* ctx, int p) {
    if (!ctx->shapes_ready) return fail(ctx, PT_ERR_STATE, "launch shapes not prepared");
    // Inside one transfer run the backward pass does not wait for the whole
    // forward pass: a backward visit reads only its own table's forward results
    // (survivors, row ids, the hashes its forward inserts kept, the filters its
    // forward scan zeroed) and the filters its backward builders make, so it
    // waits for its forward visit and those builders, and the pass-1 counters
    // are zeroed with the pass-0 ones before either pass starts
    const bool chained = ctx->in_transfer && ctx->schedule == PT_SCHEDULE_TRANSFER && ctx->chain_ok;
    if (!(chained && p == 1)) {
        // (the two passes' counters are adjacent in the arena: one memset for both)
        PT_CUDA(ctx, cudaMemsetAsync(ctx->meta[p], 0, ctx->meta_bytes * (chained ? 2 : 1), ctx->stream));
        PT_CUDA(ctx, cudaEventRecord(ctx->pass_ev[p], ctx->stream));
    }
    // enqueue by level (then visiting order): a stream never holds a visit
    // behind one of a higher level, which would delay it for nothing
    std::vector<const Visit*> seq;
    for (const Visit& vis : ctx->visits[p]) seq.push_back(&vis);
    std::stable_sort(seq.begin(), seq.end(), [&](const Visit* x, const Visit* y) {
        return ctx->lvl[p][x->table] < ctx->lvl[p][y->table];
    });
    // Waits on events only across streams: on one stream, order already holds
    // (every kernel a visit launches as a programmatic dependent waits for the
    // kernel before it at its start, so each waits, in turn, for all earlier
    // ones), and a wait on an event of the same stream would turn the
    // programmatic edge from the kernel before into a full one (measured
    // between consecutive visits of one stream: about 4.5 µs from the end of
    // one kernel's last CTA to the next one's first, against 1.5 µs)
    bool joined[pt_ctx::kAux] = {};
    for (const Visit* vp : seq) {
        const Visit& vis = *vp;
        const int v = vis.table;
        const int sv = ctx->slot[p][v] % ctx->streams;
        cudaStream_t st = ctx->aux[sv];
        if (chained && p == 1) {
            if (ctx->slot[0][v] % ctx->streams != sv) PT_CUDA(ctx, cudaStreamWaitEvent(st, ctx->vev[0][v], 0));
        } else {
            if (!joined[sv]) PT_CUDA(ctx, cudaStreamWaitEvent(st, ctx->pass_ev[p], 0));
            joined[sv] = true;
        }
        // the visits that build its filters in this pass (filters of an earlier
        // pass are complete when this one forks from the context stream)
        const bool same_pass = ctx->fpass[p] == p;
        if (same_pass)
            for (int e : vis.in_edges)
                if (ctx->slot[p][ctx->bld[p][e]] % ctx->streams != sv)
                    PT_CUDA(ctx, cudaStreamWaitEvent(st, ctx->vev[p][ctx->bld[p][e]], 0));
        const ScanShape& sh = vis.shape;
        pt::VisitArgs a;
        fill_visit_args(ctx, p, vis, sh, a);
        pt_status s1;
        if (vis.first && ctx->first_probe) {
            // in the default probe order the first probe tests a filter of one of
            // the lowest-level builders: it waits for those only, on its own
            // stream; in the other orders it may be any builder's.  When every
            // builder is at that level (a visit with one incoming edge), the visit's
            // own stream, which waits for them anyway, takes it: no event between
            // the builders and the pass, nor between the pass and the scan
            int32_t lmin = INT32_MAX;
            bool all_lowest = true;
            if (same_pass) {
                for (int e : vis.in_edges) lmin = std::min(lmin, ctx->lvl[p][ctx->bld[p][e]]);
                for (int e : vis.in_edges) all_lowest = all_lowest && ctx->lvl[p][ctx->bld[p][e]] == lmin;
            }
            cudaStream_t fs = ctx->streams > 1 && !all_lowest ? ctx->fstream[v] : st;
            if (fs != st) {
                PT_CUDA(ctx, cudaStreamWaitEvent(fs, ctx->pass_ev[p], 0));
                if (same_pass)
                    for (int e : vis.in_edges)
                        if (ctx->fcfg.probe_order != 0 || ctx->lvl[p][ctx->bld[p][e]] == lmin)
                            PT_CUDA(ctx, cudaStreamWaitEvent(fs, ctx->vev[p][ctx->bld[p][e]], 0));
            }
            // and for the first-probe passes of lower-level visits: those lead to
            // this visit's higher-level builders, and a first-probe pass over a
            // large table holds every SM until it ends (measured on the benchmark:
            // 0.541 -> 0.510 ms when the fact table's pass runs after M's)
            for (const Visit& o : ctx->visits[p])
                if (o.first && ctx->lvl[p][o.table] < ctx->lvl[p][v]) PT_CUDA(ctx, cudaStreamWaitEvent(fs, ctx->fev[o.table], 0));
            if ((s1 = record_event(ctx, 2, fs, p, v)) != PT_OK) return s1;
            if (vis.first_pair) {
                // the filter's size is known on the device only: one launch with the
                // shared-memory budget, one without (all of L1 for a filter that cannot
                // fit); each returns at once unless the size calls for it
                const int32_t bw = (int32_t)(vis.first_smem / 4);
                PT_CUDA(ctx, pt::launch_probe_first(a, ctx->fcfg, ctx->mid[v], ctx->first_idx + v, bw, bw, 1,
                                                    vis.first_grid, pt::kFirstThreads, vis.first_smem, fs));
                PT_CUDA(ctx, pt::launch_probe_first(a, ctx->fcfg, ctx->mid[v], ctx->first_idx + v, 0, bw, 2,
                                                    vis.first_grid0, pt::kFirstThreads, 0, fs));
                ctx->launches++;
            } else {
                PT_CUDA(ctx, pt::launch_probe_first(a, ctx->fcfg, ctx->mid[v], ctx->first_idx + v,
                                                    (int32_t)(vis.first_smem / 4), 0, 0, vis.first_grid,
                                                    pt::kFirstThreads, vis.first_smem, fs));
            }
            if ((s1 = record_event(ctx, 2, fs, p, v)) != PT_OK) return s1;
            PT_CUDA(ctx, cudaEventRecord(ctx->fev[v], fs));
            ctx->launches++;
            a.in_bits = ctx->mid[v];
            a.first_in = ctx->first_idx + v;
            cudaEvent_t done = ctx->fev[v];
            if (vis.early && ctx->early_scan && ctx->fcfg.probe_order == 0) {
                // the other filters of builders below the visit's highest level, in
                // probe order, as soon as those builders are done: their probes then
                // overlap the higher-level builders instead of following them
                if (same_pass)
                    for (int e : vis.in_edges) {
                        const int b = ctx->bld[p][e];
                        if (ctx->lvl[p][b] < vis.early_level) PT_CUDA(ctx, cudaStreamWaitEvent(fs, ctx->vev[p][b], 0));
                    }
                pt::VisitArgs ea = a;
                ea.level_hi = vis.early_level;
                ea.out_bits = ctx->mid2[v];
                ea.ids = nullptr;
                ea.seg_count = nullptr;
                ea.n_out = 0;
                ea.n_clear_extra = 0;
                ea.n_bcols = 0;
                ea.count = ctx->early_count[p] + v;
                if ((s1 = record_event(ctx, 0, fs, p, v)) != PT_OK) return s1;
                PT_CUDA(ctx, pt::launch_scan(ea, ctx->fcfg, sh.grid, sh.block, sh.smem, fs));
                if ((s1 = record_event(ctx, 0, fs, p, v)) != PT_OK) return s1;
                PT_CUDA(ctx, cudaEventRecord(ctx->eev[v], fs));
                ctx->launches++;
                done = ctx->eev[v];
                a.in_bits = ctx->mid2[v];
                a.level_lo = vis.early_level;
            }
            if (fs != st) PT_CUDA(ctx, cudaStreamWaitEvent(st, done, 0));
        }
        // a visit's kernels may start while the kernel before them on their stream
        // ends (they wait for its results on the device); not between the event
        // records of a timed run
        const bool pdl = ctx->pdl && !ctx->timing;
        // (a pass-through visit folded into its forward scan and its insert launches nothing here)
        if (!(vis.pass_through && a.insert_bsec)) {
            if ((s1 = record_event(ctx, 0, st, p, v)) != PT_OK) return s1;
            if (vis.pass_through)
                PT_CUDA(ctx, pt::launch_pass_through(a, ctx->fcfg, ctx->num_sms * 2, st, pdl));
            else if (p == 1 && vis.list)
                PT_CUDA(ctx, pt::launch_probe_list(a, ctx->fcfg, vis.list_grid, vis.list_smem, st, pdl));
            else
                PT_CUDA(ctx, pt::launch_scan(a, ctx->fcfg, sh.grid, sh.block, sh.smem, st, pdl));
            if ((s1 = record_event(ctx, 0, st, p, v)) != PT_OK) return s1;
            ctx->launches++;
        }
        if (a.n_out > 0) {
            // the scan above zeroed the previous run's filter words; the insert sizes
            // the filters from the survivor count and sets their bits.  256-thread
            // CTAs, at most one resident wave of them (a second wave would start only
            // as the first ends: measured 0.4384 -> 0.4372 ms against 1.5 waves);
            // segments are split between warps when there are more warps than segments
            if ((s1 = record_event(ctx, 1, st, p, v)) != PT_OK) return s1;
            const int grid_i = std::max(1, std::min(3 * a.total_warps / 8 + 1, ctx->num_sms * ctx->insert_fit));
            PT_CUDA(ctx, pt::launch_insert(a, ctx->fcfg, grid_i, 256, st, pdl));
            if ((s1 = record_event(ctx, 1, st, p, v)) != PT_OK) return s1;
            ctx->launches++;
        }
        PT_CUDA(ctx, cudaEventRecord(ctx->vev[p][v], st));
    }
    // join: the pass is complete on the context stream (in a chained transfer,
    // both passes, after the backward one)
    if (chained && p == 0) return PT_OK;
    for (int q = chained ? 0 : p; q <= p; ++q)
        for (const Visit& vis : ctx->visits[q]) PT_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->vev[q][vis.table], 0));
    return PT_OK;
}

pt_status require_plan(pt_ctx* ctx) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (!ctx->planned) return fail(ctx, PT_ERR_STATE, "pt_plan has not run");
    return PT_OK;
}

}  // namespace

namespace pt {
void set_global_error(const char* msg) { g_err = msg; }
}  // namespace pt

extern "C" {

uint32_t pt_abi_version(void) { return (1u << 16) | 0u; }

pt_status pt_create(pt_ctx** out, const pt_filter_cfg* cfg, void* cuda_stream) {
    if (!out || !cfg) return fail(nullptr, PT_ERR_INVALID, "out or cfg is NULL");
    *out = nullptr;
    if (cfg->block_bits != 256 && cfg->block_bits != 512)
        return fail(nullptr, PT_ERR_INVALID, "block_bits must be 256 or 512 (got %d)", cfg->block_bits);
    if (cfg->k < 1 || cfg->k > 16) return fail(nullptr, PT_ERR_INVALID, "k must be in 1..16 (got %d)", cfg->k);
    if (cfg->bits_per_key < 1 || cfg->bits_per_key > 64)
        return fail(nullptr, PT_ERR_INVALID, "bits_per_key must be in 1..64 (got %d)", cfg->bits_per_key);
    if (cfg->reserved != 0) return fail(nullptr, PT_ERR_INVALID, "reserved must be 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, PT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, PT_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    pt_ctx* ctx = new (std::nothrow) pt_ctx();
    if (!ctx) return fail(nullptr, PT_ERR_OOM, "host allocation");
    ctx->fcfg.bits_per_key = cfg->bits_per_key;
    ctx->fcfg.k = cfg->k;
    ctx->fcfg.block_bits = cfg->block_bits;
    ctx->fcfg.seed = cfg->seed;
    ctx->device = dev;
    ctx->num_sms = sms;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return fail(nullptr, PT_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return PT_OK;
}

pt_status pt_destroy(pt_ctx* ctx) {
    if (!ctx) return PT_OK;
    cudaStreamSynchronize(ctx->stream);
    free_arena(ctx);
    for (Table& t : ctx->tables) {
        for (Col& c : t.cols)
            if (c.owned) cudaFree(c.owned);
        if (t.sel_owned) cudaFree(t.sel_owned);
    }
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->gev) cudaEventDestroy(e);
    for (int p = 0; p < 2; ++p) {
        for (cudaEvent_t e : ctx->vev[p])
            if (e) cudaEventDestroy(e);
        if (ctx->pass_ev[p]) cudaEventDestroy(ctx->pass_ev[p]);
    }
    for (int i = 0; i < pt_ctx::kAux; ++i)
        if (ctx->aux[i]) cudaStreamDestroy(ctx->aux[i]);
    for (cudaStream_t f : ctx->fstream)
        if (f) cudaStreamDestroy(f);
    for (cudaEvent_t e : ctx->fev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->eev)
        if (e) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PT_OK;
}

pt_status pt_register_table(pt_ctx* ctx, int64_t n_rows, int32_t n_cols, const pt_column* cols,
                            const uint32_t* sel, int32_t sel_mem, int32_t* table_id) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (ctx->planned || ctx->graph_set) return fail(ctx, PT_ERR_STATE, "tables are registered before the join graph and the plan");
    if (n_rows < 0 || n_rows > 0x7FFFFFFFll) return fail(ctx, PT_ERR_INVALID, "n_rows %lld out of range", (long long)n_rows);
    if ((int)ctx->tables.size() >= kMaxTables) return fail(ctx, PT_ERR_INVALID, "more than %d tables", kMaxTables);
    pt_status st = check_columns(ctx, n_rows, n_cols, cols, sel_mem);
    if (st != PT_OK) return st;
    if (sel && sel_mem == PT_MEM_DEVICE && ((uintptr_t)sel % 16) != 0)
        return fail(ctx, PT_ERR_INVALID, "device selection bitmap must be 16-byte aligned");
    Table t;
    t.n = n_rows;
    t.cols.resize(n_cols);
    st = upload_table(ctx, t, n_cols, cols, sel, sel_mem, true);
    if (st != PT_OK) {
        for (Col& c : t.cols)
            if (c.owned) cudaFree(c.owned);
        if (t.sel_owned) cudaFree(t.sel_owned);
        return st;
    }
    ctx->tables.push_back(t);
    if (table_id) *table_id = (int32_t)ctx->tables.size() - 1;
    return PT_OK;
}

pt_status pt_update_table(pt_ctx* ctx, int32_t table_id, const pt_column* cols, const uint32_t* sel,
                          int32_t sel_mem) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (table_id < 0 || table_id >= (int)ctx->tables.size()) return fail(ctx, PT_ERR_INVALID, "table id %d", table_id);
    Table& t = ctx->tables[table_id];
    pt_status st = check_columns(ctx, t.n, (int32_t)t.cols.size(), cols, sel_mem);
    if (st != PT_OK) return st;
    for (size_t j = 0; j < t.cols.size(); ++j)
        if (cols[j].dtype != t.cols[j].dtype) return fail(ctx, PT_ERR_INVALID, "column %zu changes dtype", j);
    if (sel && sel_mem == PT_MEM_DEVICE && ((uintptr_t)sel % 16) != 0)
        return fail(ctx, PT_ERR_INVALID, "device selection bitmap must be 16-byte aligned");
    if (ctx->planned && ((sel == nullptr) != (t.sel == nullptr)))
        return fail(ctx, PT_ERR_INVALID, "a planned table keeps having (or not having) a selection bitmap");
    st = upload_table(ctx, t, (int32_t)t.cols.size(), cols, sel, sel_mem, false);
    if (st != PT_OK) return st;
    if (ctx->gexec) {  // captured kernel parameters hold the old pointers
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->passes_done = 0;
    return PT_OK;
}

pt_status pt_set_join_graph(pt_ctx* ctx, int32_t n_edges, const pt_edge* edges) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (ctx->planned) return fail(ctx, PT_ERR_STATE, "the join graph is fixed once planned");
    std::vector<int> ncols;
    for (const Table& t : ctx->tables) ncols.push_back((int)t.cols.size());
    pt_status st = check_edges(ctx, (int32_t)ctx->tables.size(), ncols, nullptr, n_edges, edges);
    if (st != PT_OK) return st;
    ctx->edges.assign(edges, edges + n_edges);
    ctx->graph_set = true;
    return PT_OK;
}

pt_status pt_plan(pt_ctx* ctx, int32_t* order_out, int64_t* mem_bytes_out) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (ctx->planned) return fail(ctx, PT_ERR_STATE, "already planned");
    const int T = (int)ctx->tables.size(), E = (int)ctx->edges.size();
    if (T == 0) return fail(ctx, PT_ERR_STATE, "no tables registered");
    std::vector<int64_t> n(T);
    for (int v = 0; v < T; ++v) n[v] = ctx->tables[v].n;
    plan_graph(n, ctx->edges, ctx->src, ctx->dst, ctx->order, ctx->level);

    const pt::FilterCfg& f = ctx->fcfg;
    ctx->filt_max_words.assign(E, 0);
    for (int e = 0; e < E; ++e)
        ctx->filt_max_words[e] = max_filter_words(n[ctx->edges[e].t0], n[ctx->edges[e].t1], f);

    // who builds and who probes each edge's filter in each pass
    const bool one_hop = ctx->schedule == PT_SCHEDULE_ONE_HOP;
    for (int p = 0; p < 2; ++p) {
        ctx->bld[p].assign(E, -1);
        ctx->prb[p].assign(E, -1);
    }
    for (int e = 0; e < E; ++e) {
        const pt_edge& ed = ctx->edges[e];
        const bool one_way = (ed.flags & PT_EDGE_ONE_WAY) != 0;
        if (one_hop) {
            // a Bloom join (Section 2.1): built in pass 0 from the smaller table's
            // selection (a one-way edge's t0), probed in pass 1 by the other end
            const int b = one_way ? ed.t0 : ctx->src[e];
            ctx->bld[0][e] = b;
            ctx->prb[1][e] = b == ed.t0 ? ed.t1 : ed.t0;
        } else {
            // forward along the DAG, backward against it; a one-way edge transfers
            // only from its t0 (Section 3.4): in one of the two passes
            for (int p = 0; p < 2; ++p) {
                const int from = p == 0 ? ctx->src[e] : ctx->dst[e];
                if (one_way && from != ed.t0) continue;
                ctx->bld[p][e] = from;
                ctx->prb[p][e] = p == 0 ? ctx->dst[e] : ctx->src[e];
            }
        }
    }
    ctx->fpass[0] = 0;
    ctx->fpass[1] = one_hop ? 0 : 1;

    for (int p = 0; p < 2; ++p) {
        ctx->visits[p].clear();
        for (int oi = 0; oi < T; ++oi) {
            Visit vis;
            vis.table = p == 0 ? ctx->order[oi] : ctx->order[T - 1 - oi];
            for (int e = 0; e < E; ++e) {
                const int into = ctx->prb[p][e];
                const int from = ctx->bld[p][e];
                if (into == vis.table) {
                    vis.in_edges.push_back(e);
                    vis.max_in_filter_bytes += ctx->filt_max_words[e] * 4;
                    vis.max_single_filter_bytes = std::max(vis.max_single_filter_bytes, ctx->filt_max_words[e] * 4);
                }
                if (from == vis.table) {
                    vis.out_edges.push_back(e);
                    const pt_edge& ed = ctx->edges[e];
                    const int32_t* cs = ed.t0 == vis.table ? ed.c0 : ed.c1;
                    for (int j = 0; j < ed.ncols; ++j)
                        if (std::find(vis.bcols.begin(), vis.bcols.end(), cs[j]) == vis.bcols.end()) vis.bcols.push_back(cs[j]);
                }
            }
            if ((int)vis.in_edges.size() > pt::kMaxIn || (int)vis.out_edges.size() > pt::kMaxOut ||
                (int)vis.bcols.size() > pt::kMaxBuildCols)
                return fail(ctx, PT_ERR_UNSUPPORTED, "table %d has more than %d incoming or %d outgoing edges in a pass",
                            vis.table, pt::kMaxIn, pt::kMaxOut);
            // the probing pass of a one-hop schedule visits every table (a table
            // without incoming filters keeps its selection); its building pass only
            // the builders
            if (one_hop && p == 0 && vis.out_edges.empty()) continue;
            // a first-probe pass: the visit's rows all start alive (the forward
            // pass of a transfer, the probing pass of a one-hop schedule)
            vis.first = p == (one_hop ? 1 : 0) && !vis.in_edges.empty() && ctx->tables[vis.table].sel == nullptr &&
                        ctx->tables[vis.table].n >= pt::kFirstMinRows;
            ctx->visits[p].push_back(vis);
        }
    }
    ctx->has_edge.assign(T, false);
    for (int e = 0; e < E; ++e) ctx->has_edge[ctx->edges[e].t0] = ctx->has_edge[ctx->edges[e].t1] = true;
    for (int p = 0; p < 2; ++p) {
        ctx->vidx[p].assign(T, -1);
        for (int i = 0; i < (int)ctx->visits[p].size(); ++i) ctx->vidx[p][ctx->visits[p][i].table] = i;
    }
    // a backward visit of a table with an edge starts from its forward survivor list
    if (!one_hop)
        for (Visit& vis : ctx->visits[1]) {
            vis.list = ctx->has_edge[vis.table];
            vis.pass_through = vis.list && vis.in_edges.empty() && !vis.out_edges.empty();
        }
    // a transfer run may chain each backward visit onto its table's forward visit
    ctx->chain_ok = !one_hop;
    for (const Visit& vis : ctx->visits[1]) ctx->chain_ok = ctx->chain_ok && ctx->vidx[0][vis.table] >= 0;

    // streams and events for concurrent visits (level = longest path from a
    // source of the pass's DAG)
    for (int i = 0; i < pt_ctx::kAux; ++i)
        if (!ctx->aux[i]) PT_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
    for (int p = 0; p < 2; ++p) {
        if (!ctx->pass_ev[p]) PT_CUDA(ctx, cudaEventCreateWithFlags(&ctx->pass_ev[p], cudaEventDisableTiming));
        ctx->vev[p].assign(T, nullptr);
        for (int v = 0; v < T; ++v) PT_CUDA(ctx, cudaEventCreateWithFlags(&ctx->vev[p][v], cudaEventDisableTiming));
        std::vector<int32_t>& lvl = ctx->lvl[p];
        lvl.assign(T, 0);
        for (const Visit& vis : ctx->visits[p])
            for (int e : vis.out_edges) {
                const int to = ctx->prb[p][e];
                if (to >= 0) lvl[to] = std::max(lvl[to], lvl[vis.table] + 1);
            }
        // streams (slot = index into aux): within a level, bigger tables choose
        // first, and a visit takes the stream of its biggest builder in this pass
        // unless another visit of the level has it; else the first stream the level
        // leaves free.  The chain of big visits, which is the critical path, then
        // stays on one stream: its kernels follow one another with no cross-stream
        // wait and launch as programmatic dependents
        ctx->slot[p].assign(T, 0);
        int max_l = 0;
        for (const Visit& vis : ctx->visits[p]) max_l = std::max(max_l, lvl[vis.table]);
        for (int l = 0; l <= max_l; ++l) {
            std::vector<int> vs;
            for (const Visit& vis : ctx->visits[p])
                if (lvl[vis.table] == l) vs.push_back(vis.table);
            std::stable_sort(vs.begin(), vs.end(), [&](int x, int y) { return n[x] > n[y]; });
            bool taken[pt_ctx::kAux] = {};
            int wrap = 0;
            for (int v : vs) {
                int pref = -1;
                int64_t biggest = -1;
                for (int e : ctx->visits[p][ctx->vidx[p][v]].in_edges) {
                    const int b = ctx->bld[p][e];
                    if (b >= 0 && ctx->vidx[p][b] >= 0 && n[b] > biggest) {
                        biggest = n[b];
                        pref = ctx->slot[p][b];
                    }
                }
                // a backward visit with no builder in its pass continues its forward
                // visit's stream (it reads that visit's results)
                if (pref < 0 && p == 1 && !one_hop && ctx->vidx[0][v] >= 0) pref = ctx->slot[0][v];
                int sl = pref >= 0 && !taken[pref] ? pref : -1;
                for (int i = 0; sl < 0 && i < pt_ctx::kAux; ++i)
                    if (!taken[i]) sl = i;
                if (sl < 0) sl = wrap++ % pt_ctx::kAux;  // more visits in the level than streams
                taken[sl] = true;
                ctx->slot[p][v] = sl;
            }
        }
    }
    // early scans: a visit with a first-probe pass and, besides the edge that pass
    // takes (one of the lowest level), more edges from builders below its highest
    // level
    for (int p = 0; p < 2; ++p)
        for (Visit& vis : ctx->visits[p]) {
            if (!vis.first) continue;
            int32_t lmax = 0, below = 0;
            for (int e : vis.in_edges) lmax = std::max(lmax, ctx->lvl[p][ctx->bld[p][e]]);
            for (int e : vis.in_edges) below += ctx->lvl[p][ctx->bld[p][e]] < lmax;
            vis.early = below >= 2;
            vis.early_level = lmax;
        }
    ctx->fstream.assign(T, nullptr);
    ctx->fev.assign(T, nullptr);
    ctx->eev.assign(T, nullptr);
    for (int p = 0; p < 2; ++p)
        for (const Visit& vis : ctx->visits[p]) {
            if (!vis.first) continue;
            PT_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->fstream[vis.table], cudaStreamNonBlocking));
            PT_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fev[vis.table], cudaEventDisableTiming));
            if (vis.early) PT_CUDA(ctx, cudaEventCreateWithFlags(&ctx->eev[vis.table], cudaEventDisableTiming));
        }

    // one device allocation holds every buffer of a run
    ctx->seg_cap = (int64_t)ctx->num_sms * 64;  // at most 64 resident warps per SM
    const std::vector<bool>& has_edge = ctx->has_edge;
    size_t off = 0;
    std::vector<size_t> o_surv[2], o_ids[2], o_seg[2], o_filt[2], o_mid(T, 0), o_hash(E, 0);
    std::vector<bool> has_mid(T, false), has_mid2(T, false);
    std::vector<size_t> o_mid2(T, 0);
    for (int p = 0; p < 2; ++p)
        for (const Visit& vis : ctx->visits[p]) {
            if (vis.first) has_mid[vis.table] = true;
            if (vis.early) has_mid2[vis.table] = true;
        }
    for (int p = 0; p < 2; ++p) {
        o_surv[p].resize(T);
        o_filt[p].resize(E);
        o_ids[p].resize(T);
        o_seg[p].resize(T);
    }
    for (int v = 0; v < T; ++v) {
        const size_t wb = (size_t)((n[v] + 31) / 32) * 4;
        for (int p = 0; p < 2; ++p) {
            o_surv[p][v] = off;
            off += align_up(std::max<size_t>(wb, 16));
        }
        for (int p = 0; p < 2; ++p) {
            o_ids[p][v] = off;
            if (has_edge[v]) off += align_up(std::max<size_t>((size_t)n[v] * 4, 16));
            o_seg[p][v] = off;
            if (has_edge[v]) off += align_up((size_t)ctx->seg_cap * 4);
        }
        o_mid[v] = off;  // whole 256-row tiles: the first-probe kernel writes 8 words at a time
        if (has_mid[v]) off += align_up((size_t)((n[v] + 255) / 256) * 32);
        o_mid2[v] = off;
        if (has_mid2[v]) off += align_up(std::max<size_t>((size_t)((n[v] + 31) / 32) * 4, 16));
    }
    for (int e = 0; e < E; ++e)
        for (int p = 0; p < 2; ++p) {
            o_filt[p][e] = off;
            off += align_up((size_t)ctx->filt_max_words[e] * 4);
        }
    // per edge: its forward builder's survivors' key hashes, slot-aligned with the ids
    for (int e = 0; e < E; ++e) {
        o_hash[e] = off;
        off += align_up(std::max<size_t>((size_t)n[ctx->src[e]] * 8, 16));
    }
    // zeroed at every pass: counts [T] u64, stats [T][3] u64, early-scan counts [T]
    // u64, first-probe edge [T] i32
    ctx->meta_bytes = align_up((size_t)T * 8 + (size_t)T * 24 + (size_t)T * 8 + (size_t)T * 4);
    size_t o_meta[2], o_nblocks[2];
    for (int p = 0; p < 2; ++p) {  // adjacent: a chained transfer zeroes both with one memset
        o_meta[p] = off;
        off += ctx->meta_bytes;
    }
    // filter sizes [E] i64, kept from run to run: a building visit's scan zeroes the
    // words its filters had in the previous run
    for (int p = 0; p < 2; ++p) {
        o_nblocks[p] = off;
        off += align_up((size_t)std::max(E, 1) * 8);
    }
    void* arena = nullptr;
    // PT_INJECT_OOM=1 makes this allocation fail on the host (tests of the error path)
    const char* inject = getenv("PT_INJECT_OOM");
    if ((inject && inject[0] == '1') || cudaMalloc(&arena, off) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PT_ERR_OOM, "device arena of %zu bytes", off);
    }
    ctx->arena = arena;
    ctx->arena_bytes = off;
    char* base = (char*)arena;
    for (int p = 0; p < 2; ++p) {
        ctx->surv[p].resize(T);
        ctx->filt[p].resize(E);
        for (int v = 0; v < T; ++v) ctx->surv[p][v] = (uint32_t*)(base + o_surv[p][v]);
        for (int e = 0; e < E; ++e) ctx->filt[p][e] = (uint32_t*)(base + o_filt[p][e]);
        ctx->meta[p] = base + o_meta[p];
        ctx->counts[p] = (unsigned long long*)(base + o_meta[p]);
        ctx->stats[p] = (unsigned long long*)(base + o_meta[p] + (size_t)T * 8);
        ctx->early_count[p] = (unsigned long long*)(base + o_meta[p] + (size_t)T * 32);
        ctx->nblocks[p] = (int64_t*)(base + o_nblocks[p]);
    }
    ctx->first_idx = (int32_t*)(base + o_meta[0] + (size_t)T * 40);
    ctx->mid.assign(T, nullptr);
    ctx->mid2.assign(T, nullptr);
    for (int v = 0; v < T; ++v) {
        if (has_mid[v]) ctx->mid[v] = (uint32_t*)(base + o_mid[v]);
        if (has_mid2[v]) ctx->mid2[v] = (uint32_t*)(base + o_mid2[v]);
    }
    for (int p = 0; p < 2; ++p) {
        ctx->ids[p].resize(T);
        ctx->seg[p].resize(T);
        for (int v = 0; v < T; ++v) {
            ctx->ids[p][v] = has_edge[v] ? (uint32_t*)(base + o_ids[p][v]) : nullptr;
            ctx->seg[p][v] = has_edge[v] ? (uint32_t*)(base + o_seg[p][v]) : nullptr;
        }
    }
    ctx->hfwd.resize(E);
    for (int e = 0; e < E; ++e) ctx->hfwd[e] = (uint64_t*)(base + o_hash[e]);
    for (const Visit& vis : ctx->visits[1])
        if (vis.pass_through) {
            ctx->surv[1][vis.table] = ctx->surv[0][vis.table];
            ctx->ids[1][vis.table] = ctx->ids[0][vis.table];
            ctx->seg[1][vis.table] = ctx->seg[0][vis.table];
        }
    // bitmaps of tables nobody visits with data still read as zero tails
    PT_CUDA(ctx, cudaMemsetAsync(arena, 0, off, ctx->stream));
    ctx->planned = true;
    ctx->passes_done = 0;
    if (order_out)
        for (int i = 0; i < T; ++i) order_out[i] = ctx->order[i];
    if (mem_bytes_out) *mem_bytes_out = (int64_t)off;
    return PT_OK;
}

pt_status pt_run_forward(pt_ctx* ctx) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if ((st = prepare_shapes(ctx)) != PT_OK) return st;
    st = enqueue_pass(ctx, 0);
    if (st != PT_OK) return st;
    ctx->passes_done = 1;
    return PT_OK;
}

pt_status pt_run_backward(pt_ctx* ctx) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if (!(ctx->passes_done & 1)) return fail(ctx, PT_ERR_STATE, "the backward pass needs a forward pass first");
    if ((st = prepare_shapes(ctx)) != PT_OK) return st;
    st = enqueue_pass(ctx, 1);
    if (st != PT_OK) return st;
    ctx->passes_done |= 2;
    return PT_OK;
}

// Both passes of a transfer, with pass-through visits folded (see
// fill_visit_args); the flag is set only while they are enqueued.
struct InTransfer {
    pt_ctx* ctx;
    explicit InTransfer(pt_ctx* c) : ctx(c) { ctx->in_transfer = true; }
    ~InTransfer() { ctx->in_transfer = false; }
};

pt_status pt_run_transfer(pt_ctx* ctx) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    InTransfer fold(ctx);
    if (!ctx->graph_mode) {
        st = pt_run_forward(ctx);
        if (st != PT_OK) return st;
        return pt_run_backward(ctx);
    }
    if ((st = prepare_shapes(ctx)) != PT_OK) return st;
    if (ctx->gexec && ctx->graph_timed != ctx->timing) {  // recapture with / without timing nodes
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    if (!ctx->gexec) {
        const int64_t before = ctx->launches;
        PT_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        ctx->gev_used = 0;
        pt_status s0 = enqueue_pass(ctx, 0);
        pt_status s1 = s0 == PT_OK ? enqueue_pass(ctx, 1) : s0;
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        ctx->capturing = false;
        ctx->graph_timed = ctx->timing;
        ctx->graph_replays = 0;
        ctx->graph_kernels = ctx->launches - before;
        ctx->launches = before;
        if (s1 != PT_OK) {
            if (g) cudaGraphDestroy(g);
            return s1;
        }
        if (ce != cudaSuccess) return fail(ctx, PT_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            ctx->gexec = nullptr;
            return fail(ctx, PT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ce));
        }
    }
    PT_CUDA(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream));
    ctx->graph_replays++;
    ctx->launches += ctx->graph_kernels;
    ctx->passes_done = 3;
    return PT_OK;
}

pt_status pt_set_graph_mode(pt_ctx* ctx, int32_t on) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    ctx->graph_mode = on != 0;
    if (!ctx->graph_mode && ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return PT_OK;
}

pt_status pt_get_pass_survivors(pt_ctx* ctx, int32_t pass, int32_t table_id, uint32_t* bitmap_out,
                                int64_t* count_out) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if (pass < 0 || pass > 1) return fail(ctx, PT_ERR_INVALID, "pass %d", pass);
    if (table_id < 0 || table_id >= (int)ctx->tables.size()) return fail(ctx, PT_ERR_INVALID, "table id %d", table_id);
    if (!(ctx->passes_done & (1 << pass))) return fail(ctx, PT_ERR_STATE, "pass %d has not run", pass);
    if (ctx->vidx[pass][table_id] < 0) return fail(ctx, PT_ERR_INVALID, "table %d has no visit in pass %d", table_id, pass);
    const size_t bytes = (size_t)((ctx->tables[table_id].n + 31) / 32) * 4;
    if (bitmap_out && bytes)
        PT_CUDA(ctx, cudaMemcpyAsync(bitmap_out, ctx->surv[pass][table_id], bytes, cudaMemcpyDefault, ctx->stream));
    unsigned long long c = 0;
    if (count_out)
        PT_CUDA(ctx, cudaMemcpyAsync(&c, count_of(ctx, pass, table_id), sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (count_out) *count_out = (int64_t)c;
    return PT_OK;
}

pt_status pt_get_survivors(pt_ctx* ctx, int32_t table_id, uint32_t* bitmap_out, int64_t* count_out) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    return pt_get_pass_survivors(ctx, (ctx->passes_done & 2) ? 1 : 0, table_id, bitmap_out, count_out);
}

pt_status pt_get_filter(pt_ctx* ctx, int32_t pass, int32_t edge_id, uint32_t* words_out, int64_t* nblocks_out) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if (pass < 0 || pass > 1) return fail(ctx, PT_ERR_INVALID, "pass %d", pass);
    if (edge_id < 0 || edge_id >= (int)ctx->edges.size()) return fail(ctx, PT_ERR_INVALID, "edge id %d", edge_id);
    if (!(ctx->passes_done & (1 << pass))) return fail(ctx, PT_ERR_STATE, "pass %d has not run", pass);
    int64_t nb = 0;
    PT_CUDA(ctx, cudaMemcpyAsync(&nb, ctx->nblocks[pass] + edge_id, sizeof nb, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (words_out && nb > 0)
        PT_CUDA(ctx, cudaMemcpyAsync(words_out, ctx->filt[pass][edge_id], (size_t)nb * ctx->fcfg.block_bits / 8,
                                     cudaMemcpyDefault, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (nblocks_out) *nblocks_out = nb;
    return PT_OK;
}

pt_status pt_get_visit_stats(pt_ctx* ctx, int32_t pass, int32_t table_id, pt_visit_stats* out) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if (pass < 0 || pass > 1 || !out) return fail(ctx, PT_ERR_INVALID, "pass %d / out NULL", pass);
    if (table_id < 0 || table_id >= (int)ctx->tables.size()) return fail(ctx, PT_ERR_INVALID, "table id %d", table_id);
    if (!(ctx->passes_done & (1 << pass))) return fail(ctx, PT_ERR_STATE, "pass %d has not run", pass);
    if (ctx->vidx[pass][table_id] < 0) return fail(ctx, PT_ERR_INVALID, "table %d has no visit in pass %d", table_id, pass);
    const int T = (int)ctx->tables.size(), E = (int)ctx->edges.size();
    std::vector<unsigned long long> c(T), s(3 * T);
    std::vector<int64_t> nb(std::max(E, 1));
    PT_CUDA(ctx, cudaMemcpyAsync(c.data(), ctx->counts[pass], T * 8, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaMemcpyAsync(s.data(), ctx->stats[pass], 3 * T * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (E) PT_CUDA(ctx, cudaMemcpyAsync(nb.data(), ctx->nblocks[pass], E * 8, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const Visit* vis = &ctx->visits[pass][ctx->vidx[pass][table_id]];
    std::memset(out, 0, sizeof *out);
    out->n_rows = ctx->tables[table_id].n;
    out->survivors = (int64_t)c[table_id];
    if (vis->pass_through) {  // its count is its forward one
        unsigned long long cf = 0;
        PT_CUDA(ctx, cudaMemcpy(&cf, count_of(ctx, pass, table_id), sizeof cf, cudaMemcpyDeviceToHost));
        out->survivors = (int64_t)cf;
    }
    out->probe_sectors = (int64_t)s[3 * table_id];
    out->build_sectors = (int64_t)s[3 * table_id + 1];
    out->first_probe_sectors = (int64_t)s[3 * table_id + 2];
    out->first_probe = out->first_probe_sectors > 0 ? 1 : 0;
    out->n_in = (int32_t)vis->in_edges.size();
    out->n_out = (int32_t)vis->out_edges.size();
    for (int e : vis->out_edges) out->filter_bytes += nb[e] * ctx->fcfg.block_bits / 8;
    out->has_input_bitmap = (pass == 1 && ctx->schedule == PT_SCHEDULE_TRANSFER) || ctx->tables[table_id].sel != nullptr;
    return PT_OK;
}

pt_status pt_set_streams(pt_ctx* ctx, int32_t streams) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (streams < 1 || streams > pt_ctx::kAux) return fail(ctx, PT_ERR_INVALID, "streams must be 1..%d (got %d)", pt_ctx::kAux, streams);
    if (streams != ctx->streams && ctx->gexec) {  // the captured launch sequence changes
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->streams = streams;
    return PT_OK;
}

pt_status pt_set_first_probe(pt_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (enable != 0 && enable != 1) return fail(ctx, PT_ERR_INVALID, "enable must be 0 or 1 (got %d)", enable);
    if (ctx->first_probe != (enable == 1)) {  // the launch sequence and scan shapes change
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        ctx->shapes_ready = false;
    }
    ctx->first_probe = enable == 1;
    return PT_OK;
}

pt_status pt_set_early_scan(pt_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (enable != 0 && enable != 1) return fail(ctx, PT_ERR_INVALID, "enable must be 0 or 1 (got %d)", enable);
    if (ctx->early_scan != (enable == 1) && ctx->gexec) {  // the launch sequence changes
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->early_scan = enable == 1;
    return PT_OK;
}

pt_status pt_set_dependent_launch(pt_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (enable != 0 && enable != 1) return fail(ctx, PT_ERR_INVALID, "enable must be 0 or 1 (got %d)", enable);
    if (ctx->pdl != (enable == 1) && ctx->gexec) {  // the captured launches change
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->pdl = enable == 1;
    return PT_OK;
}

pt_status pt_set_schedule(pt_ctx* ctx, int32_t schedule) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (schedule != PT_SCHEDULE_TRANSFER && schedule != PT_SCHEDULE_ONE_HOP)
        return fail(ctx, PT_ERR_INVALID, "schedule must be %d or %d (got %d)", PT_SCHEDULE_TRANSFER,
                    PT_SCHEDULE_ONE_HOP, schedule);
    if (ctx->planned) return fail(ctx, PT_ERR_STATE, "the schedule is fixed once planned");
    ctx->schedule = schedule;
    return PT_OK;
}

pt_status pt_set_probe_order(pt_ctx* ctx, int32_t order) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (order < 0 || order > 2) return fail(ctx, PT_ERR_INVALID, "order must be 0, 1 or 2 (got %d)", order);
    if (ctx->fcfg.probe_order != order && ctx->gexec) {  // captured kernel parameters hold the old order
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    ctx->fcfg.probe_order = order;
    return PT_OK;
}

pt_status pt_set_first_probe_ctas(pt_ctx* ctx, int32_t ctas_per_sm) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (ctas_per_sm < 0 || ctas_per_sm > 3) return fail(ctx, PT_ERR_INVALID, "ctas_per_sm must be 0..3 (got %d)", ctas_per_sm);
    if (ctx->first_ctas != ctas_per_sm) {
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        ctx->shapes_ready = false;
    }
    ctx->first_ctas = ctas_per_sm;
    return PT_OK;
}

pt_status pt_set_launch(pt_ctx* ctx, int32_t threads, int32_t smem_filter_bytes, int32_t ctas_per_sm) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (threads < 64 || threads > pt::kScanMaxThreads || threads % 32)
        return fail(ctx, PT_ERR_INVALID, "threads %d (64..%d, multiple of 32)", threads, pt::kScanMaxThreads);
    if (smem_filter_bytes < 0 || smem_filter_bytes > 220 * 1024) return fail(ctx, PT_ERR_INVALID, "smem %d", smem_filter_bytes);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(ctx, PT_ERR_INVALID, "ctas_per_sm %d", ctas_per_sm);
    ctx->scan_threads = threads;
    ctx->smem_budget = smem_filter_bytes / 16 * 16;
    ctx->ctas_per_sm = ctas_per_sm;
    ctx->shapes_ready = false;
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return PT_OK;
}

pt_status pt_set_cluster(pt_ctx* ctx, int32_t max_cluster) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    if (max_cluster != 1 && max_cluster != 2 && max_cluster != 4)
        return fail(ctx, PT_ERR_INVALID, "max_cluster %d (1, 2 or 4)", max_cluster);
    ctx->max_cluster = max_cluster;
    ctx->shapes_ready = false;
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return PT_OK;
}

pt_status pt_set_kernel_timing(pt_ctx* ctx, int32_t on) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    ctx->timing = on != 0;
    ctx->ev_used = 0;
    ctx->graph_replays = 0;
    return PT_OK;
}

namespace {
// Summed event times of kind 0 (scan), 1 (size/clear + insert), 2 (first probe).
pt_status kernel_times(pt_ctx* ctx, double* t, int* n) {
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    auto sum = [&](const std::vector<cudaEvent_t>& ev, const std::vector<int>& kinds, size_t used) -> pt_status {
        for (size_t i = 0; i + 1 < used; i += 2) {
            float ms = 0.f;
            PT_CUDA(ctx, cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            t[kinds[i] & 15] += ms;
            n[kinds[i] & 15] += 1;
        }
        return PT_OK;
    };
    pt_status st = sum(ctx->ev, ctx->ev_kind, ctx->ev_used);
    if (st != PT_OK) return st;
    if (ctx->gexec && ctx->graph_timed && ctx->graph_replays > 0) {
        st = sum(ctx->gev, ctx->gev_kind, ctx->gev_used);  // the most recent replay
        if (st != PT_OK) return st;
    }
    return PT_OK;
}
}  // namespace

pt_status pt_get_kernel_time(pt_ctx* ctx, double* scan_ms, int32_t* scan_launches, double* other_ms,
                             int32_t* other_launches) {
    if (!ctx) return fail(nullptr, PT_ERR_INVALID, "ctx is NULL");
    double t[3] = {0, 0, 0};
    int n[3] = {0, 0, 0};
    pt_status st = kernel_times(ctx, t, n);
    if (st != PT_OK) return st;
    if (scan_ms) *scan_ms = t[0] + t[2];
    if (scan_launches) *scan_launches = n[0] + n[2];
    if (other_ms) *other_ms = t[1];
    if (other_launches) *other_launches = n[1];
    return PT_OK;
}

pt_status pt_get_launch_times(pt_ctx* ctx, int32_t max, pt_launch_time* out, int32_t* n_out) {
    if (!ctx || !n_out || (max > 0 && !out)) return fail(ctx, PT_ERR_INVALID, "ctx, out or n_out is NULL");
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const bool graph = ctx->gexec && ctx->graph_timed && ctx->graph_replays > 0;
    const std::vector<cudaEvent_t>& ev = graph ? ctx->gev : ctx->ev;
    const std::vector<int>& kinds = graph ? ctx->gev_kind : ctx->ev_kind;
    const size_t used = graph ? ctx->gev_used : ctx->ev_used;
    int32_t n = 0;
    for (size_t i = 0; i + 1 < used; i += 2, ++n) {
        if (n >= max) continue;
        float ms = 0.f, start = 0.f;
        PT_CUDA(ctx, cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        PT_CUDA(ctx, cudaEventElapsedTime(&start, ev[0], ev[i]));
        pt_launch_time& o = out[n];
        std::memset(&o, 0, sizeof o);
        o.kind = kinds[i] & 15;
        o.pass = (kinds[i] >> 4) & 15;
        o.table = kinds[i] >> 8;
        o.start_ms = start;
        o.ms = ms;
    }
    *n_out = n;
    return PT_OK;
}

pt_status pt_get_kernel_times(pt_ctx* ctx, pt_kernel_times* out) {
    if (!ctx || !out) return fail(ctx, PT_ERR_INVALID, "ctx or out is NULL");
    double t[3] = {0, 0, 0};
    int n[3] = {0, 0, 0};
    pt_status st = kernel_times(ctx, t, n);
    if (st != PT_OK) return st;
    std::memset(out, 0, sizeof *out);
    out->first_ms = t[2];
    out->scan_ms = t[0];
    out->build_ms = t[1];
    out->first_launches = n[2];
    out->scan_launches = n[0];
    out->build_pairs = n[1];
    return PT_OK;
}

pt_status pt_get_launch_count(pt_ctx* ctx, int64_t* launches) {
    if (!ctx || !launches) return fail(ctx, PT_ERR_INVALID, "ctx or launches is NULL");
    *launches = ctx->launches;
    return PT_OK;
}

pt_status pt_plan_graph(int32_t n_tables, const int64_t* n_rows, int32_t n_edges, const pt_edge* edges,
                        int32_t* src_out, int32_t* dst_out, int32_t* order_out, int32_t* level_out) {
    if (n_tables < 1 || n_tables > kMaxTables || !n_rows) return fail(nullptr, PT_ERR_INVALID, "n_tables %d", n_tables);
    std::vector<int> ncols(n_tables, kMaxCols);  // column indexes are not known here
    pt_status st = check_edges(nullptr, n_tables, ncols, nullptr, n_edges, edges);
    if (st != PT_OK) return st;
    std::vector<int64_t> n(n_rows, n_rows + n_tables);
    std::vector<pt_edge> e(edges, edges + n_edges);
    std::vector<int32_t> src, dst, order, level;
    plan_graph(n, e, src, dst, order, level);
    for (int i = 0; i < n_edges; ++i) {
        if (src_out) src_out[i] = src[i];
        if (dst_out) dst_out[i] = dst[i];
    }
    for (int i = 0; i < n_tables; ++i) {
        if (order_out) order_out[i] = order[i];
        if (level_out) level_out[i] = level[i];
    }
    return PT_OK;
}

pt_status pt_join_count(pt_ctx* ctx, uint64_t* count_out) {
    pt_status st = require_plan(ctx);
    if (st != PT_OK) return st;
    if (!count_out) return fail(ctx, PT_ERR_INVALID, "count_out is NULL");
    if (!ctx->passes_done) return fail(ctx, PT_ERR_STATE, "no pass has run");
    const int p = (ctx->passes_done & 2) ? 1 : 0;  // the latest pass's survivors
    const int T = (int)ctx->tables.size(), E = (int)ctx->edges.size();
    // an acyclic graph of inner joins: no one-way edge, no cycle (union-find)
    std::vector<int> uf(T);
    for (int v = 0; v < T; ++v) uf[v] = v;
    auto find = [&](int x) {
        while (uf[x] != x) x = uf[x] = uf[uf[x]];
        return x;
    };
    for (int e = 0; e < E; ++e) {
        if (ctx->edges[e].flags) return fail(ctx, PT_ERR_UNSUPPORTED, "join count: edge %d is one-way (outer join)", e);
        const int a = find(ctx->edges[e].t0), b = find(ctx->edges[e].t1);
        if (a == b) return fail(ctx, PT_ERR_UNSUPPORTED, "join count: the join graph has a cycle (edge %d)", e);
        uf[a] = b;
    }
    // trees rooted at their largest table (ties: higher id); children before parents
    std::vector<int> parent(T, -1), pedge(T, -1), order, roots;
    std::vector<char> seen(T, 0);
    for (;;) {
        int root = -1;
        for (int v = 0; v < T; ++v)
            if (!seen[v] && (root < 0 || ctx->tables[v].n >= ctx->tables[root].n)) root = v;
        if (root < 0) break;
        roots.push_back(root);
        std::vector<int> stack{root};
        seen[root] = 1;
        while (!stack.empty()) {
            const int x = stack.back();
            stack.pop_back();
            order.push_back(x);
            for (int e = 0; e < E; ++e) {
                const pt_edge& ed = ctx->edges[e];
                const int y = ed.t0 == x ? ed.t1 : (ed.t1 == x ? ed.t0 : -1);
                if (y < 0 || seen[y]) continue;
                seen[y] = 1;
                parent[y] = x;
                pedge[y] = e;
                stack.push_back(y);
            }
        }
    }
    // survivor counts size each child's hash table (at most half full)
    std::vector<unsigned long long> cnt(T);
    for (int v = 0; v < T; ++v)
        PT_CUDA(ctx, cudaMemcpyAsync(&cnt[v], count_of(ctx, p, v), 8, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    uint64_t cap = 1024;
    for (int v = 0; v < T; ++v)
        if (parent[v] >= 0)
            while (cap < 2 * cnt[v]) cap <<= 1;
    std::vector<size_t> wo(T);
    size_t bytes = 0;
    for (int v = 0; v < T; ++v) {
        wo[v] = bytes;
        bytes += align_up(std::max<size_t>((size_t)ctx->tables[v].n * 8, 16));
    }
    const size_t o_table = bytes;
    bytes += align_up(cap * sizeof(pt::JoinSlot));
    const size_t o_scalars = bytes;  // err flag, then one sum per root
    bytes += align_up(16 + 8 * roots.size());
    void* mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PT_ERR_OOM, "join count: %zu bytes of device memory", bytes);
    }
    char* base = (char*)mem;
    auto w = [&](int v) { return (unsigned long long*)(base + wo[v]); };
    pt::JoinSlot* table = (pt::JoinSlot*)(base + o_table);
    int32_t* err = (int32_t*)(base + o_scalars);
    unsigned long long* sums = (unsigned long long*)(base + o_scalars + 16);
    auto run = [&]() -> pt_status {
        PT_CUDA(ctx, cudaMemsetAsync(base + o_scalars, 0, 16 + 8 * roots.size(), ctx->stream));
        for (int v = 0; v < T; ++v)
            PT_CUDA(ctx, pt::launch_join_init(ctx->surv[p][v], ctx->tables[v].n, w(v), ctx->num_sms, ctx->stream));
        for (size_t i = order.size(); i-- > 0;) {
            const int c = order[i], par = parent[c];
            if (par < 0) continue;
            const pt_edge& ed = ctx->edges[pedge[c]];
            const int32_t* cc = ed.t0 == c ? ed.c0 : ed.c1;
            const int32_t* cp = ed.t0 == par ? ed.c0 : ed.c1;
            uint64_t m = 1024;
            while (m < 2 * cnt[c]) m <<= 1;
            PT_CUDA(ctx, cudaMemsetAsync(table, 0, m * sizeof(pt::JoinSlot), ctx->stream));
            PT_CUDA(ctx, pt::launch_join_build(colref(ctx, c, cc[0]), colref(ctx, c, ed.ncols == 2 ? cc[1] : cc[0]),
                                               ed.ncols, w(c), ctx->tables[c].n, table, m - 1, err, ctx->num_sms,
                                               ctx->stream));
            PT_CUDA(ctx, pt::launch_join_probe(colref(ctx, par, cp[0]), colref(ctx, par, ed.ncols == 2 ? cp[1] : cp[0]),
                                               ed.ncols, w(par), ctx->tables[par].n, table, m - 1, ctx->num_sms,
                                               ctx->stream));
        }
        for (size_t i = 0; i < roots.size(); ++i)
            PT_CUDA(ctx, pt::launch_join_sum(w(roots[i]), ctx->tables[roots[i]].n, sums + i, ctx->num_sms, ctx->stream));
        return PT_OK;
    };
    st = run();
    int32_t herr = 0;
    std::vector<unsigned long long> hs(roots.size());
    if (st == PT_OK) {
        cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(hs.data(), sums, 8 * roots.size(), cudaMemcpyDeviceToHost, ctx->stream);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PT_ERR_CUDA, "join count: %s", cudaGetErrorString(e));
    }
    cudaFree(mem);
    if (st != PT_OK) return st;
    if (herr == 1) return fail(ctx, PT_ERR_TIMEOUT, "join count: a wait on a hash-table slot ran out");
    if (herr) return fail(ctx, PT_ERR_CUDA, "join count: hash table full");
    uint64_t total = 1;
    for (unsigned long long x : hs) total *= x;
    *count_out = total;
    return PT_OK;
}

const char* pt_last_error(pt_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

}  // extern "C"
