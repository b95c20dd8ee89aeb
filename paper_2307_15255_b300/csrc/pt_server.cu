// Serving loop for predicate-transfer queries over resident tables.
//
// Tables are registered once and stay in device memory, each key column next
// to a column of its precomputed hashes H(x), so that no query hashes a
// resident key again.  A query names table instances (an instance is one
// use of a resident table with its own selection bitmap; a table may appear
// twice) and equi-join edges between instances; its transfer is the same
// forward and backward pass over the size-ordered DAG as a planned context
// (Section 3.2 of the paper), and its survivor bitmaps are identical to a
// plain context's on the same inputs.
//
// Continuous batching: a scheduler thread admits waiting queries in arrival
// order as long as their device memory (bitmaps, filters, row ids, copies of
// their selections) fits the server's arena, groups up to max_batch of them
// into a batch and runs the batch as a handful of batched launches -- per
// pass and per DAG level one scan, one size/clear and one insert launch over
// a task list that covers every query's visits at that level.  Task lists
// and visit arguments are uploaded into device buffers, so the launch
// sequence is captured once per (forward levels, backward levels) shape as a
// CUDA graph and replayed for every batch.  Up to max_inflight batches run at
// once on their own streams; queries that arrive while batches are on the
// GPU are admitted as soon as a slot and memory free up.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pt.h"
#include "pt_internal.h"

namespace {

constexpr int kMaxInst = 6;
constexpr int kMaxQEdges = 8;
constexpr int kMaxLevels = kMaxInst;
constexpr int kMaxSlots = 4;
constexpr int kScanWarps = 8;            // batched scan CTA: 256 threads
constexpr int64_t kTileWords = 4096;     // scan task = 4096 bitmap words = 128k rows
constexpr int kClearParts = 16;
constexpr int kInsertParts = 64;
constexpr int kFilterSmem = 16 * 1024;   // shared-memory filter budget of a batched scan CTA: with the queues
                                         // two CTAs per SM fit, and L1 keeps room for the filters probed
                                         // through it (measured 0 / 16 / 40 / 56 KB: 1568 / 1591 / 1172 /
                                         // 1318 batched queries per second)
constexpr int kCluster = 1;              // batched scan CTAs per cluster (1: no cluster-spread filters)
constexpr size_t kAl = 256;
constexpr int kLaunchesPerLevel = 4;     // first probe, scan, size/clear, insert
constexpr int kMetaWordsPerPass = kMaxInst * 4 + kMaxQEdges;  // count, 3 sector counters per instance; nblocks per edge
constexpr int kFirstSmem = 40 * 1024;    // filter budget of a batched first-probe CTA (three per SM)

size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Col {
    const void* key = nullptr;  // device
    int32_t dtype = 0;
    void* owned = nullptr;      // device copy of a host column
    uint64_t* hashed = nullptr; // device, H(key) per row
};

struct ResTable {
    int64_t n = 0;
    std::vector<Col> cols;
};

// First-fit allocator over the server's device arena (offsets).
class Arena {
   public:
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

   private:
    std::map<size_t, size_t> free_;
};

struct QVisit {
    int inst = 0;
    int level = 0;
    bool first = false;  // a first-probe pass (forward, every row alive, a large table)
    std::vector<int> in_edges, out_edges;
    std::vector<int> bcols;
    int64_t grid = 1;  // scan tasks (CTAs)
    int wpw = 32;      // words per scan warp
};

enum QState { kPending = 0, kRunning = 1, kDone = 2 };

struct Query {
    uint64_t ticket = 0;
    int n_inst = 0;
    int table[kMaxInst] = {};
    std::vector<uint32_t> sel[kMaxInst];  // host copies of the selections (empty = none or borrowed)
    const uint32_t* sel_dev[kMaxInst] = {};  // borrowed device selections
    int n_edges = 0;
    pt_edge edges[kMaxQEdges] = {};
    int32_t src[kMaxQEdges] = {}, dst[kMaxQEdges] = {};
    std::vector<QVisit> visits[2];
    int levels[2] = {0, 0};
    int lvl[2][kMaxInst] = {};  // per pass, per instance: level of its visit
    // device layout (offsets inside the query's arena allocation)
    size_t bytes = 0, base = 0;
    size_t o_surv[2][kMaxInst] = {}, o_ids[kMaxInst] = {}, o_seg[kMaxInst] = {}, o_sel[kMaxInst] = {};
    size_t o_mid[kMaxInst] = {}, o_first[kMaxInst] = {};  // a first-probe pass's bitmap and edge slot
    size_t o_filt[2][kMaxQEdges] = {};
    int64_t filt_words[kMaxQEdges] = {};
    // state
    int state = kPending;
    pt_status result = PT_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t count[2][kMaxInst] = {};
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char* d_desc = nullptr;
    unsigned char* h_desc = nullptr;  // pinned
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    std::vector<Query*> batch;
    bool busy = false;
};

// Layout of a slot's descriptor buffer.
struct DescLayout {
    size_t o_visits = 0, o_ranges = 0, o_tasks = 0, o_meta = 0, bytes = 0;
    int max_visits = 0, max_tasks = 0;
};

}  // namespace

struct pt_server {
    pt::FilterCfg fcfg{};
    int device = 0, num_sms = 0;
    int max_batch = 1, max_inflight = 1;
    std::vector<ResTable> tables;
    bool started = false;

    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    Arena alloc;

    DescLayout dl;
    Slot slots[kMaxSlots];
    int scan_grid = 1, clear_grid = 1, insert_grid = 1, first_grid = 1, first_grid0 = 1;
    size_t scan_smem = 0;
    cudaStream_t copy_stream = nullptr;

    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Query*> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Query>> queries;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    pt_status fatal = PT_OK;
    std::string fatal_msg;

    // statistics over completed queries
    std::vector<double> latencies;
    double first_submit = 0, last_done = 0;
    int64_t completed = 0, batches = 0, batched_queries = 0;
};

namespace {

pt_status fail(pt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pt::set_global_error(buf);
    return st;
}

#define SRV_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(PT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int64_t max_filter_words(int64_t n0, int64_t n1, const pt::FilterCfg& f) {
    const int64_t m = std::min(n0, n1);
    int64_t nb = (m * f.bits_per_key + f.block_bits - 1) / f.block_bits;
    if (nb < 1) nb = 1;
    return nb * (f.block_bits / 32);
}

// Size-ordered orientation and both passes' visits with their levels
// (Section 3.2), plus the query's device layout.
pt_status plan_query(pt_server* S, Query* q) {
    const int T = q->n_inst, E = q->n_edges;
    int64_t n[kMaxInst];
    for (int v = 0; v < T; ++v) n[v] = S->tables[q->table[v]].n;
    auto less = [&](int a, int b) { return n[a] != n[b] ? n[a] < n[b] : a < b; };
    for (int e = 0; e < E; ++e) {
        const pt_edge& x = q->edges[e];
        if (less(x.t0, x.t1)) {
            q->src[e] = x.t0;
            q->dst[e] = x.t1;
        } else {
            q->src[e] = x.t1;
            q->dst[e] = x.t0;
        }
    }
    std::vector<int> order(T);
    for (int i = 0; i < T; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), less);
    const pt::FilterCfg& f = S->fcfg;
    for (int p = 0; p < 2; ++p) {
        q->visits[p].clear();
        std::vector<int> lvl(T, 0);
        for (int oi = 0; oi < T; ++oi) {
            QVisit vis;
            vis.inst = p == 0 ? order[oi] : order[T - 1 - oi];
            for (int e = 0; e < E; ++e) {
                const int into = p == 0 ? q->dst[e] : q->src[e];
                const int from = p == 0 ? q->src[e] : q->dst[e];
                if (into == vis.inst) vis.in_edges.push_back(e);
                if (from == vis.inst) {
                    vis.out_edges.push_back(e);
                    const pt_edge& ed = q->edges[e];
                    const int32_t* cs = ed.t0 == vis.inst ? ed.c0 : ed.c1;
                    for (int j = 0; j < ed.ncols; ++j)
                        if (std::find(vis.bcols.begin(), vis.bcols.end(), cs[j]) == vis.bcols.end()) vis.bcols.push_back(cs[j]);
                }
            }
            for (int e : vis.in_edges) {
                const int b = p == 0 ? q->src[e] : q->dst[e];
                vis.level = std::max(vis.level, lvl[b] + 1);
            }
            lvl[vis.inst] = vis.level;
            q->lvl[p][vis.inst] = vis.level;
            // every row of a large instance without a selection starts alive: its first
            // probe streams the edge's hash column in a launch of its own
            vis.first = p == 0 && !vis.in_edges.empty() && q->sel[vis.inst].empty() && !q->sel_dev[vis.inst] &&
                        n[vis.inst] >= pt::kFirstMinRows;
            // scan tasks: tiles of kTileWords words, each run by a cluster of kCluster CTAs
            const int64_t words = (n[vis.inst] + 31) / 32;
            vis.grid = std::max<int64_t>(1, (words + kTileWords - 1) / kTileWords);
            const int64_t ctas = vis.grid * kCluster;
            int64_t wpw = (words + ctas * kScanWarps - 1) / (ctas * kScanWarps);
            wpw = std::max<int64_t>(32, (wpw + 31) / 32 * 32);
            vis.wpw = (int)wpw;
            q->levels[p] = std::max(q->levels[p], vis.level + 1);
            q->visits[p].push_back(vis);
        }
    }
    // layout
    size_t off = 0;
    bool has_edge[kMaxInst] = {};
    for (int e = 0; e < E; ++e) has_edge[q->edges[e].t0] = has_edge[q->edges[e].t1] = true;
    for (int v = 0; v < T; ++v) {
        const size_t wb = al(std::max<size_t>((size_t)((n[v] + 31) / 32) * 4, 16));
        for (int p = 0; p < 2; ++p) {
            q->o_surv[p][v] = off;
            off += wb;
        }
        q->o_sel[v] = off;
        if (!q->sel[v].empty()) off += wb;
        bool first = false;
        for (const QVisit& vis : q->visits[0])
            if (vis.inst == v) first = vis.first;
        q->o_mid[v] = off;  // whole 256-row tiles: the first probe writes 8 words at a time
        if (first) off += al((size_t)((n[v] + 255) / 256) * 32);
        q->o_first[v] = off;
        if (first) off += al(16);
        q->o_ids[v] = off;
        if (has_edge[v]) off += al(std::max<size_t>((size_t)n[v] * 4, 16));
        q->o_seg[v] = off;
        if (has_edge[v]) {
            int64_t g = 1;
            for (const QVisit& vis : q->visits[0])
                if (vis.inst == v) g = vis.grid;
            off += al((size_t)g * kCluster * kScanWarps * 4);
        }
    }
    for (int e = 0; e < E; ++e) {
        q->filt_words[e] = max_filter_words(n[q->edges[e].t0], n[q->edges[e].t1], f);
        for (int p = 0; p < 2; ++p) {
            q->o_filt[p][e] = off;
            off += al((size_t)q->filt_words[e] * 4);
        }
    }
    q->bytes = std::max<size_t>(off, kAl);
    return PT_OK;
}

pt::ColRef colref(pt_server* S, const Query* q, int inst, int c, bool hashed) {
    const Col& col = S->tables[q->table[inst]].cols[c];
    pt::ColRef r{};
    if (hashed) {
        r.p = col.hashed;
        r.dtype = pt::kHashed;
    } else {
        r.p = col.key;
        r.dtype = col.dtype;
    }
    return r;
}

// Visit arguments of (query q, pass p, visit vis), with the batch's counters at meta.
void fill_args(pt_server* S, const Query* q, int p, const QVisit& vis, unsigned long long* meta_dev,
               pt::VisitArgs& a) {
    std::memset(&a, 0, sizeof a);
    const int v = vis.inst;
    unsigned char* base = S->arena + q->base;
    unsigned long long* counts = meta_dev + p * kMetaWordsPerPass;
    unsigned long long* stats = counts + kMaxInst;
    int64_t* nblocks = (int64_t*)(counts + 4 * kMaxInst);
    a.n = S->tables[q->table[v]].n;
    if (p == 0)
        a.in_bits = q->sel_dev[v] ? q->sel_dev[v] : q->sel[v].empty() ? nullptr : (const uint32_t*)(base + q->o_sel[v]);
    else
        a.in_bits = (const uint32_t*)(base + q->o_surv[0][v]);
    if (vis.first) {  // the first-probe pass writes these, the scan reads them
        a.in_bits = (const uint32_t*)(base + q->o_mid[v]);
        a.first_in = (const int32_t*)(base + q->o_first[v]);
    }
    a.out_bits = (uint32_t*)(base + q->o_surv[p][v]);
    a.count = counts + v;
    a.stats = stats + 3 * v;
    a.n_in = (int)vis.in_edges.size();
    a.n_out = (int)vis.out_edges.size();
    a.words_per_warp = vis.wpw;
    a.total_warps = (int)(vis.grid * kCluster * kScanWarps);
    a.smem_words = kFilterSmem / 4;
    a.cluster = kCluster;
    for (int i = 0; i < a.n_in; ++i) {
        const int e = vis.in_edges[i];
        const pt_edge& ed = q->edges[e];
        const int32_t* cs = ed.t0 == v ? ed.c0 : ed.c1;
        const int b = p == 0 ? q->src[e] : q->dst[e];
        pt::ProbeEdge& pe = a.in[i];
        pe.ncols = ed.ncols;
        pe.edge_id = e;
        pe.col[0] = colref(S, q, v, cs[0], true);
        pe.col[1] = ed.ncols == 2 ? colref(S, q, v, cs[1], false) : pe.col[0];
        pe.filter = (const uint32_t*)(base + q->o_filt[p][e]);
        pe.nblocks = nblocks + e;
        pe.build_count = counts + b;
        pe.build_rows = S->tables[q->table[b]].n;
        pe.build_level = q->lvl[p][b];
    }
    for (int i = 0; i < a.n_out; ++i) {
        const int e = vis.out_edges[i];
        const pt_edge& ed = q->edges[e];
        const int32_t* cs = ed.t0 == v ? ed.c0 : ed.c1;
        const int other = ed.t0 == v ? ed.t1 : ed.t0;
        pt::BuildEdge& be = a.out[i];
        be.ncols = ed.ncols;
        be.edge_id = e;
        be.col[0] = colref(S, q, v, cs[0], true);
        be.col[1] = ed.ncols == 2 ? colref(S, q, v, cs[1], false) : be.col[0];
        be.filter = (uint32_t*)(base + q->o_filt[p][e]);
        be.nblocks = nblocks + e;
        be.probe_rows = S->tables[q->table[other]].n;
    }
    // build-sector accounting by the keys' own width (not their hash columns)
    a.n_bcols = (int)vis.bcols.size();
    for (int i = 0; i < a.n_bcols; ++i) a.bcol[i] = colref(S, q, v, vis.bcols[i], false);
    if (a.n_out > 0) {
        a.ids = (uint32_t*)(base + q->o_ids[v]);
        a.seg_count = (uint32_t*)(base + q->o_seg[v]);
    }
}

int launch_index(int p, int level, int kind) { return (p * kMaxLevels + level) * kLaunchesPerLevel + kind; }

// The batch's launch sequence for (forward levels, backward levels); the
// kernels read their task ranges from the slot's descriptor buffer.
pt_status enqueue_batch_launches(pt_server* S, Slot& sl, int lf, int lb) {
    const pt::VisitArgs* visits = (const pt::VisitArgs*)(sl.d_desc + S->dl.o_visits);
    const pt::BatchTask* tasks = (const pt::BatchTask*)(sl.d_desc + S->dl.o_tasks);
    const int32_t* ranges = (const int32_t*)(sl.d_desc + S->dl.o_ranges);
    for (int p = 0; p < 2; ++p) {
        const int L = p == 0 ? lf : lb;
        for (int l = 0; l < L; ++l) {
            if (p == 0) {
                // a pair over the same tasks: filters that fit the budget are probed from
                // shared memory, the others with all of L1 (each launch returns at once
                // from the other's tasks)
                const int32_t* rf = ranges + 2 * launch_index(p, l, 0);
                SRV_CUDA(pt::launch_probe_first_batch(visits, tasks, rf, S->fcfg, kFirstSmem / 4, kFirstSmem / 4, 1,
                                                      S->first_grid, kFirstSmem, sl.stream));
                SRV_CUDA(pt::launch_probe_first_batch(visits, tasks, rf, S->fcfg, 0, kFirstSmem / 4, 2,
                                                      S->first_grid0, 0, sl.stream));
            }
            SRV_CUDA(pt::launch_scan_batch(visits, tasks, ranges + 2 * launch_index(p, l, 1), S->fcfg, kCluster,
                                           S->scan_grid, kScanWarps * 32, S->scan_smem, sl.stream));
            SRV_CUDA(pt::launch_size_clear_batch(visits, tasks, ranges + 2 * launch_index(p, l, 2), kClearParts,
                                                 S->fcfg, S->clear_grid, 512, sl.stream));
            SRV_CUDA(pt::launch_insert_batch(visits, tasks, ranges + 2 * launch_index(p, l, 3), kInsertParts, S->fcfg,
                                             S->insert_grid, 512, sl.stream));
        }
    }
    return PT_OK;
}

pt_status graph_for(pt_server* S, Slot& sl, int lf, int lb, cudaGraphExec_t* out) {
    auto key = std::make_pair(lf, lb);
    auto it = sl.graphs.find(key);
    if (it != sl.graphs.end()) {
        *out = it->second;
        return PT_OK;
    }
    SRV_CUDA(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
    pt_status st = enqueue_batch_launches(S, sl, lf, lb);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(sl.stream, &g);
    if (st != PT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    sl.graphs[key] = ex;
    *out = ex;
    return PT_OK;
}

// Build the descriptors of a batch in the slot's pinned buffer, upload them
// and the queries' selections, and launch the batch's graph.
pt_status launch_batch(pt_server* S, Slot& sl) {
    const DescLayout& L = S->dl;
    unsigned char* h = sl.h_desc;
    pt::VisitArgs* hv = (pt::VisitArgs*)(h + L.o_visits);
    int32_t* ranges = (int32_t*)(h + L.o_ranges);
    pt::BatchTask* tasks = (pt::BatchTask*)(h + L.o_tasks);
    unsigned long long* meta_h = (unsigned long long*)(h + L.o_meta);
    unsigned long long* meta_d = (unsigned long long*)(sl.d_desc + L.o_meta);
    const int nq = (int)sl.batch.size();
    std::memset(meta_h, 0, (size_t)nq * 2 * kMetaWordsPerPass * 8);
    std::memset(ranges, 0, sizeof(int32_t) * 2 * 2 * kMaxLevels * kLaunchesPerLevel);

    int lf = 0, lb = 0, nv = 0, nt = 0;
    // visit index of (query i, pass p, visit j)
    std::vector<std::vector<int>> vidx[2];
    for (int p = 0; p < 2; ++p) vidx[p].resize(nq);
    for (int i = 0; i < nq; ++i) {
        Query* q = sl.batch[i];
        lf = std::max(lf, q->levels[0]);
        lb = std::max(lb, q->levels[1]);
        for (int p = 0; p < 2; ++p)
            for (const QVisit& vis : q->visits[p]) {
                if (nv >= L.max_visits) return fail(PT_ERR_INVALID, "batch exceeds %d visits", L.max_visits);
                fill_args(S, q, p, vis, meta_d + (size_t)i * 2 * kMetaWordsPerPass, hv[nv]);
                vidx[p][i].push_back(nv++);
            }
    }
    for (int p = 0; p < 2; ++p) {
        const int Lp = p == 0 ? lf : lb;
        for (int l = 0; l < Lp; ++l) {
            // first probes, part-major across queries: queries whose first probe
            // streams the same hash column read its rows at about the same time
            int32_t* rf = ranges + 2 * launch_index(p, l, 0);
            rf[0] = nt;
            int64_t pmax = 0;
            for (int i = 0; i < nq; ++i)
                for (const QVisit& vis : sl.batch[i]->visits[p])
                    if (vis.level == l && vis.first)
                        pmax = std::max(pmax, pt::first_parts(S->tables[sl.batch[i]->table[vis.inst]].n));
            for (int64_t g = 0; g < pmax; ++g)
                for (int i = 0; i < nq; ++i)
                    for (size_t j = 0; j < sl.batch[i]->visits[p].size(); ++j) {
                        const QVisit& vis = sl.batch[i]->visits[p][j];
                        if (vis.level != l || !vis.first) continue;
                        if (g >= pt::first_parts(S->tables[sl.batch[i]->table[vis.inst]].n)) continue;
                        if (nt >= L.max_tasks) return fail(PT_ERR_INVALID, "batch exceeds %d tasks", L.max_tasks);
                        tasks[nt++] = pt::BatchTask{vidx[p][i][j], (int32_t)g};
                    }
            rf[1] = nt - rf[0];
            // scans: tile-major across queries, so the queries' tasks on the same
            // rows of a shared table run close together (their column reads hit L2)
            int32_t* r = ranges + 2 * launch_index(p, l, 1);
            r[0] = nt;
            int64_t gmax = 0;
            for (int i = 0; i < nq; ++i)
                for (size_t j = 0; j < sl.batch[i]->visits[p].size(); ++j)
                    if (sl.batch[i]->visits[p][j].level == l) gmax = std::max(gmax, sl.batch[i]->visits[p][j].grid);
            for (int64_t g = 0; g < gmax; ++g)
                for (int i = 0; i < nq; ++i)
                    for (size_t j = 0; j < sl.batch[i]->visits[p].size(); ++j) {
                        const QVisit& vis = sl.batch[i]->visits[p][j];
                        if (vis.level != l || g >= vis.grid) continue;
                        if (nt >= L.max_tasks) return fail(PT_ERR_INVALID, "batch exceeds %d tasks", L.max_tasks);
                        tasks[nt++] = pt::BatchTask{vidx[p][i][j], (int32_t)g};
                    }
            r[1] = nt - r[0];
            for (int kind = 2; kind <= 3; ++kind) {
                const int parts = kind == 2 ? kClearParts : kInsertParts;
                int32_t* rr = ranges + 2 * launch_index(p, l, kind);
                rr[0] = nt;
                for (int part = 0; part < parts; ++part)
                    for (int i = 0; i < nq; ++i)
                        for (size_t j = 0; j < sl.batch[i]->visits[p].size(); ++j) {
                            const QVisit& vis = sl.batch[i]->visits[p][j];
                            if (vis.level != l || vis.out_edges.empty()) continue;
                            if (nt >= L.max_tasks) return fail(PT_ERR_INVALID, "batch exceeds %d tasks", L.max_tasks);
                            tasks[nt++] = pt::BatchTask{vidx[p][i][j], part};
                        }
                rr[1] = nt - rr[0];
            }
        }
    }
    // selections of the batch's queries, then the descriptors, then the graph
    for (Query* q : sl.batch)
        for (int v = 0; v < q->n_inst; ++v)
            if (!q->sel[v].empty())
                SRV_CUDA(cudaMemcpyAsync(S->arena + q->base + q->o_sel[v], q->sel[v].data(), q->sel[v].size() * 4,
                                         cudaMemcpyHostToDevice, sl.stream));
    SRV_CUDA(cudaMemcpyAsync(sl.d_desc, h, L.o_tasks + (size_t)nt * sizeof(pt::BatchTask), cudaMemcpyHostToDevice,
                             sl.stream));
    SRV_CUDA(cudaMemcpyAsync(sl.d_desc + L.o_meta, h + L.o_meta, (size_t)nq * 2 * kMetaWordsPerPass * 8,
                             cudaMemcpyHostToDevice, sl.stream));
    cudaGraphExec_t ex = nullptr;
    pt_status st = graph_for(S, sl, lf, lb, &ex);
    if (st != PT_OK) return st;
    SRV_CUDA(cudaGraphLaunch(ex, sl.stream));
    SRV_CUDA(cudaMemcpyAsync(h + L.o_meta, sl.d_desc + L.o_meta, (size_t)nq * 2 * kMetaWordsPerPass * 8,
                             cudaMemcpyDeviceToHost, sl.stream));
    SRV_CUDA(cudaEventRecord(sl.done, sl.stream));
    sl.busy = true;
    S->batches++;
    S->batched_queries += nq;
    return PT_OK;
}

void finish_batch(pt_server* S, Slot& sl, pt_status st) {
    const double t = now_s();
    const unsigned long long* meta = (const unsigned long long*)(sl.h_desc + S->dl.o_meta);
    for (size_t i = 0; i < sl.batch.size(); ++i) {
        Query* q = sl.batch[i];
        for (int p = 0; p < 2; ++p)
            for (int v = 0; v < q->n_inst; ++v) q->count[p][v] = (int64_t)meta[(i * 2 + p) * kMetaWordsPerPass + v];
        q->state = kDone;
        q->result = st;
        q->t_done = t;
        S->latencies.push_back(q->t_done - q->t_submit);
        S->last_done = t;
        S->completed++;
    }
    sl.batch.clear();
    sl.busy = false;
}

void worker_loop(pt_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool inflight = false;
        for (int si = 0; si < S->max_inflight; ++si) {
            Slot& sl = S->slots[si];
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) {
                inflight = true;
                continue;
            }
            finish_batch(S, sl, e == cudaSuccess ? PT_OK : PT_ERR_CUDA);
            if (e != cudaSuccess) {
                S->fatal = PT_ERR_CUDA;
                S->fatal_msg = cudaGetErrorString(e);
            }
            S->done_cv.notify_all();
        }
        for (int si = 0; si < S->max_inflight && !S->pending.empty(); ++si) {
            Slot& sl = S->slots[si];
            if (sl.busy) continue;
            // admit in arrival order while memory and the batch size allow
            while (!S->pending.empty() && (int)sl.batch.size() < S->max_batch) {
                Query* q = S->pending.front();
                size_t off = 0;
                if (!S->alloc.alloc(q->bytes, &off)) break;
                q->base = off;
                q->state = kRunning;
                q->t_start = now_s();
                sl.batch.push_back(q);
                S->pending.pop_front();
            }
            if (sl.batch.empty()) break;
            pt_status st = launch_batch(S, sl);
            if (st != PT_OK) {
                finish_batch(S, sl, st);
                S->done_cv.notify_all();
            } else {
                inflight = true;
            }
        }
        if (!inflight && S->pending.empty()) {
            S->cv.wait(lk);
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

pt_status pt_server_create(pt_server** out, const pt_filter_cfg* cfg, int64_t arena_bytes, int32_t max_batch,
                           int32_t max_inflight) {
    if (!out || !cfg) return fail(PT_ERR_INVALID, "out or cfg is NULL");
    *out = nullptr;
    if (cfg->block_bits != 256 && cfg->block_bits != 512) return fail(PT_ERR_INVALID, "block_bits %d", cfg->block_bits);
    if (cfg->k < 1 || cfg->k > 16) return fail(PT_ERR_INVALID, "k %d", cfg->k);
    if (cfg->bits_per_key < 1 || cfg->bits_per_key > 64) return fail(PT_ERR_INVALID, "bits_per_key %d", cfg->bits_per_key);
    if (arena_bytes < (1 << 20)) return fail(PT_ERR_INVALID, "arena_bytes too small");
    if (max_batch < 1 || max_batch > 256) return fail(PT_ERR_INVALID, "max_batch %d (1..256)", max_batch);
    if (max_inflight < 1 || max_inflight > kMaxSlots) return fail(PT_ERR_INVALID, "max_inflight %d (1..%d)", max_inflight, kMaxSlots);
    std::unique_ptr<pt_server> S(new (std::nothrow) pt_server());
    if (!S) return fail(PT_ERR_OOM, "host allocation");
    S->fcfg = pt::FilterCfg{cfg->bits_per_key, cfg->k, cfg->block_bits, 0, cfg->seed};
    S->max_batch = max_batch;
    S->max_inflight = max_inflight;
    SRV_CUDA(cudaGetDevice(&S->device));
    SRV_CUDA(cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device));
    void* arena = nullptr;
    if (cudaMalloc(&arena, (size_t)arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(PT_ERR_OOM, "server arena of %lld bytes", (long long)arena_bytes);
    }
    S->arena = (unsigned char*)arena;
    S->arena_bytes = (size_t)arena_bytes;
    S->alloc.reset(S->arena_bytes);
    *out = S.release();
    return PT_OK;
}

pt_status pt_server_register_table(pt_server* S, int64_t n_rows, int32_t n_cols, const pt_column* cols,
                                   int32_t* table_id) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    if (S->started) return fail(PT_ERR_STATE, "tables are registered before pt_server_start");
    if (n_rows < 0 || n_rows > 0x7FFFFFFFll) return fail(PT_ERR_INVALID, "n_rows %lld", (long long)n_rows);
    if (n_cols < 1 || n_cols > 16 || !cols) return fail(PT_ERR_INVALID, "n_cols %d", n_cols);
    ResTable t;
    t.n = n_rows;
    for (int j = 0; j < n_cols; ++j) {
        if (cols[j].dtype != PT_I32 && cols[j].dtype != PT_I64) return fail(PT_ERR_INVALID, "column %d dtype", j);
        if (n_rows > 0 && !cols[j].data) return fail(PT_ERR_INVALID, "column %d data is NULL", j);
        Col c;
        c.dtype = cols[j].dtype;
        const size_t bytes = (size_t)n_rows * (c.dtype == PT_I32 ? 4 : 8);
        if (cols[j].mem == PT_MEM_HOST && bytes) {
            if (cudaMalloc(&c.owned, bytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(PT_ERR_OOM, "resident copy of a host column");
            }
            SRV_CUDA(cudaMemcpy(c.owned, cols[j].data, bytes, cudaMemcpyHostToDevice));
            c.key = c.owned;
        } else {
            c.key = cols[j].data;
        }
        t.cols.push_back(c);
    }
    S->tables.push_back(t);
    if (table_id) *table_id = (int32_t)S->tables.size() - 1;
    return PT_OK;
}

pt_status pt_server_start(pt_server* S) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    if (S->started) return fail(PT_ERR_STATE, "already started");
    SRV_CUDA(cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking));
    // resident hash columns
    for (ResTable& t : S->tables)
        for (Col& c : t.cols) {
            if (t.n == 0) continue;
            void* p = nullptr;
            if (cudaMalloc(&p, (size_t)t.n * 8) != cudaSuccess) {
                cudaGetLastError();
                return fail(PT_ERR_OOM, "hash column of %lld rows", (long long)t.n);
            }
            c.hashed = (uint64_t*)p;
            SRV_CUDA(pt::launch_hash_column(c.key, c.dtype, t.n, S->fcfg.seed, c.hashed, S->copy_stream));
        }
    SRV_CUDA(cudaStreamSynchronize(S->copy_stream));
    // descriptor buffers: visits, task ranges, tasks, per-query counters
    DescLayout& L = S->dl;
    L.max_visits = S->max_batch * 2 * kMaxInst;
    int64_t max_grid = 1;
    for (const ResTable& t : S->tables)
        max_grid = std::max<int64_t>(max_grid, ((t.n + 31) / 32 + kTileWords - 1) / kTileWords);
    int64_t max_first = 1;
    for (const ResTable& t : S->tables) max_first = std::max<int64_t>(max_first, pt::first_parts(t.n));
    const int64_t mt = (int64_t)S->max_batch * 2 * kMaxInst * (max_grid + max_first + kClearParts + kInsertParts);
    L.max_tasks = (int)std::min<int64_t>(mt, 1 << 24);
    L.o_visits = 0;
    L.o_ranges = al((size_t)L.max_visits * sizeof(pt::VisitArgs));
    L.o_tasks = L.o_ranges + al(sizeof(int32_t) * 2 * 2 * kMaxLevels * kLaunchesPerLevel);
    L.o_meta = L.o_tasks + al((size_t)L.max_tasks * sizeof(pt::BatchTask));
    L.bytes = L.o_meta + al((size_t)S->max_batch * 2 * kMetaWordsPerPass * 8);
    for (int si = 0; si < S->max_inflight; ++si) {
        Slot& sl = S->slots[si];
        SRV_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        SRV_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        void* d = nullptr;
        if (cudaMalloc(&d, L.bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(PT_ERR_OOM, "descriptor buffer");
        }
        sl.d_desc = (unsigned char*)d;
        void* hp = nullptr;
        if (cudaMallocHost(&hp, L.bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(PT_ERR_OOM, "pinned descriptor buffer");
        }
        sl.h_desc = (unsigned char*)hp;
    }
    // launch shapes (fixed: the graphs replay them for every batch)
    S->scan_smem = (size_t)kFilterSmem + (size_t)kScanWarps * pt::scan_warp_smem_bytes(kMaxInst - 1);
    SRV_CUDA(pt::scan_batch_set_smem_limit(S->fcfg.block_bits, S->scan_smem));
    const int fit = std::max(1, pt::scan_batch_max_ctas_per_sm(S->fcfg.block_bits, kScanWarps * 32, S->scan_smem));
    S->scan_grid = S->num_sms * fit / kCluster * kCluster;
    S->clear_grid = S->num_sms * 2;
    S->insert_grid = S->num_sms * 2;
    S->first_grid = S->num_sms * std::max(1, pt::probe_first_batch_max_ctas_per_sm(S->fcfg.block_bits, kFirstSmem));
    S->first_grid0 = S->num_sms * std::max(1, pt::probe_first_batch_max_ctas_per_sm(S->fcfg.block_bits, 0));
    S->started = true;
    S->worker = std::thread(worker_loop, S);
    return PT_OK;
}

pt_status pt_server_submit(pt_server* S, int32_t n_inst, const int32_t* table_ids, const uint32_t* const* sel_bitmaps,
                           int32_t sel_mem, int32_t n_edges, const pt_edge* edges, uint64_t* ticket) {
    if (!S || !table_ids || !ticket) return fail(PT_ERR_INVALID, "NULL argument");
    if (!S->started) return fail(PT_ERR_STATE, "pt_server_start has not run");
    if (n_inst < 1 || n_inst > kMaxInst) return fail(PT_ERR_INVALID, "n_inst %d (1..%d)", n_inst, kMaxInst);
    if (sel_mem != PT_MEM_HOST && sel_mem != PT_MEM_DEVICE) return fail(PT_ERR_INVALID, "sel_mem %d", sel_mem);
    if (n_edges < 0 || n_edges > kMaxQEdges || (n_edges > 0 && !edges)) return fail(PT_ERR_INVALID, "n_edges %d", n_edges);
    std::unique_ptr<Query> q(new Query());
    q->n_inst = n_inst;
    for (int v = 0; v < n_inst; ++v) {
        if (table_ids[v] < 0 || table_ids[v] >= (int)S->tables.size()) return fail(PT_ERR_INVALID, "table id %d", table_ids[v]);
        q->table[v] = table_ids[v];
        if (sel_bitmaps && sel_bitmaps[v]) {
            if (sel_mem == PT_MEM_DEVICE) {
                if ((uintptr_t)sel_bitmaps[v] % 16) return fail(PT_ERR_INVALID, "device selection %d not 16-byte aligned", v);
                q->sel_dev[v] = sel_bitmaps[v];
            } else {
                const size_t w = (size_t)((S->tables[table_ids[v]].n + 31) / 32);
                q->sel[v].assign(sel_bitmaps[v], sel_bitmaps[v] + w);
                if (w == 0) q->sel[v].push_back(0);
            }
        }
    }
    for (int e = 0; e < n_edges; ++e) {
        const pt_edge& x = edges[e];
        if (x.flags) return fail(PT_ERR_UNSUPPORTED, "edge %d flags", e);
        if (x.ncols < 1 || x.ncols > 2) return fail(PT_ERR_INVALID, "edge %d ncols", e);
        if (x.t0 < 0 || x.t0 >= n_inst || x.t1 < 0 || x.t1 >= n_inst || x.t0 == x.t1)
            return fail(PT_ERR_INVALID, "edge %d instances", e);
        for (int j = 0; j < x.ncols; ++j) {
            const int nc0 = (int)S->tables[q->table[x.t0]].cols.size(), nc1 = (int)S->tables[q->table[x.t1]].cols.size();
            if (x.c0[j] < 0 || x.c0[j] >= nc0 || x.c1[j] < 0 || x.c1[j] >= nc1) return fail(PT_ERR_INVALID, "edge %d columns", e);
        }
        q->edges[e] = x;
    }
    q->n_edges = n_edges;
    pt_status st = plan_query(S, q.get());
    if (st != PT_OK) return st;
    if (q->bytes > S->arena_bytes) return fail(PT_ERR_OOM, "query needs %zu bytes, the arena has %zu", q->bytes, S->arena_bytes);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != PT_OK) return fail(S->fatal, "server failed: %s", S->fatal_msg.c_str());
    q->ticket = S->next_ticket++;
    q->t_submit = now_s();
    if (S->first_submit == 0) S->first_submit = q->t_submit;
    *ticket = q->ticket;
    S->pending.push_back(q.get());
    S->queries[q->ticket] = std::move(q);
    S->cv.notify_all();
    return PT_OK;
}

pt_status pt_server_poll(pt_server* S, uint64_t ticket, int32_t* done, pt_status* result) {
    if (!S || !done) return fail(PT_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->queries.find(ticket);
    if (it == S->queries.end()) return fail(PT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->state == kDone;
    if (result) *result = it->second->result;
    return PT_OK;
}

pt_status pt_server_wait(pt_server* S, uint64_t ticket, pt_status* result) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->queries.find(ticket);
    if (it == S->queries.end()) return fail(PT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    Query* q = it->second.get();
    S->done_cv.wait(lk, [&] { return q->state == kDone; });
    if (result) *result = q->result;
    return PT_OK;
}

pt_status pt_server_survivors(pt_server* S, uint64_t ticket, int32_t inst, uint32_t* bitmap_out, int64_t* count_out) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    Query* q = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->queries.find(ticket);
        if (it == S->queries.end()) return fail(PT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
        q = it->second.get();
        if (q->state != kDone) return fail(PT_ERR_STATE, "ticket %llu is not done", (unsigned long long)ticket);
        if (q->result != PT_OK) return fail(q->result, "the query failed");
    }
    if (inst < 0 || inst >= q->n_inst) return fail(PT_ERR_INVALID, "instance %d", inst);
    if (count_out) *count_out = q->count[1][inst];
    const size_t bytes = (size_t)((S->tables[q->table[inst]].n + 31) / 32) * 4;
    if (bitmap_out && bytes) {
        SRV_CUDA(cudaMemcpyAsync(bitmap_out, S->arena + q->base + q->o_surv[1][inst], bytes, cudaMemcpyDefault,
                                 S->copy_stream));
        SRV_CUDA(cudaStreamSynchronize(S->copy_stream));
    }
    return PT_OK;
}

pt_status pt_server_release(pt_server* S, uint64_t ticket) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->queries.find(ticket);
    if (it == S->queries.end()) return fail(PT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->state != kDone) return fail(PT_ERR_STATE, "ticket %llu is not done", (unsigned long long)ticket);
    if (it->second->state == kDone && it->second->t_start > 0) S->alloc.release(it->second->base, it->second->bytes);
    S->queries.erase(it);
    S->cv.notify_all();
    return PT_OK;
}

pt_status pt_server_stats(pt_server* S, double* p50_ms, double* p99_ms, double* qps, int64_t* completed) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        if (l.empty()) return 0.0;
        size_t i = (size_t)std::min<double>(l.size() - 1, std::max(0.0, std::ceil(p * l.size()) - 1));
        return l[i] * 1e3;
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (qps) *qps = (S->completed && S->last_done > S->first_submit) ? S->completed / (S->last_done - S->first_submit) : 0.0;
    if (completed) *completed = S->completed;
    return PT_OK;
}

pt_status pt_server_reset_stats(pt_server* S) {
    if (!S) return fail(PT_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies.clear();
    S->completed = 0;
    S->first_submit = S->last_done = 0;
    S->batches = S->batched_queries = 0;
    return PT_OK;
}

pt_status pt_server_destroy(pt_server* S) {
    if (!S) return PT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (int si = 0; si < kMaxSlots; ++si) {
        Slot& sl = S->slots[si];
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        for (auto& g : sl.graphs) cudaGraphExecDestroy(g.second);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.d_desc) cudaFree(sl.d_desc);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
    }
    for (ResTable& t : S->tables)
        for (Col& c : t.cols) {
            if (c.owned) cudaFree(c.owned);
            if (c.hashed) cudaFree(c.hashed);
        }
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    if (S->arena) cudaFree(S->arena);
    delete S;
    return PT_OK;
}

}  // extern "C"
