// Internal interface between the host runtime (pt_runtime.cu) and the
// device kernels (pt_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pt {

constexpr int kMaxIn = 8;         // incoming edges of one visit
constexpr int kMaxOut = 8;        // outgoing edges of one visit
constexpr int kMaxBuildCols = 8;  // distinct build columns of one visit
constexpr int kRoundWords = 128;  // bitmap words (32 rows each) a scan warp takes per round
constexpr int kChunkWords = 32;   // granularity of a scan warp's chunk of words (dense input)
constexpr int kSparseChunkWords = 8;  // the same for an input bitmap (no dense sub-rounds to keep whole)
constexpr int kDrain = 128;       // a probe stage runs once its queue holds this many rows
constexpr int kQueueCap = kDrain + 256;  // row-id queue in front of a probe stage (per warp): room for
                                         // a drain's worth plus 8 dense words (256 rows) or a sparse sub-round
constexpr int kScanMaxThreads = 256;  // scan CTA size limit (launch bounds)
constexpr int kScanMinBlocks = 2;     // scan CTAs per SM the register budget allows
constexpr int kScanSparseMinBlocks = 3;  // the same for the scan of a visit with an input bitmap
constexpr int kFirstThreads = 256;    // first-probe CTA size (launch bounds)
constexpr int kFirstMinBlocks = 3;    // first-probe CTAs per SM the register budget allows
constexpr int kFirstTileRows = 256;   // rows a first-probe warp takes at a time (8 bitmap words)
constexpr int64_t kFirstMinRows = 1 << 20;  // smaller visits keep their first probe in the scan kernel
constexpr int kListThreads = 256;     // backward list-probe CTA size (launch bounds)
constexpr int kListMinBlocks = 3;     // its CTAs per SM the register budget allows
constexpr int kListRows = 4;          // listed survivors per lane of a batch

// Word offset of stage s's queue inside a warp's queue area, and the area's size.
__host__ __device__ inline int qoff(int s) { return s * kQueueCap; }
__host__ __device__ inline int scan_queue_words(int n_in) { return n_in * kQueueCap; }

// Shared memory a scan CTA needs besides its filter budget: per warp, one
// queue per incoming edge, the round's survivor words and the last row
// that entered each stage.
__host__ __device__ inline size_t scan_warp_smem_bytes(int n_in) {
    return (size_t)(scan_queue_words(n_in) + kRoundWords + kMaxIn) * 4;
}

constexpr int32_t kHashed = 2;  // column dtype: uint64 values that already are H(key)

struct ColRef {
    const void* p;
    int32_t dtype;  // 0 = int32, 1 = int64, kHashed = precomputed key hashes
    int32_t pad;
};

// Fill out[i] = H(key[i]) for a resident column (dtype 0 or 1).
cudaError_t launch_hash_column(const void* keys, int32_t dtype, int64_t n, uint64_t seed, uint64_t* out,
                               cudaStream_t s);

// An incoming edge of a visit: the visit's key column(s) on the edge and
// the filter the other end built earlier in the same pass.
struct ProbeEdge {
    ColRef col[2];
    int32_t ncols;
    int32_t edge_id;
    const uint32_t* filter;
    const int64_t* nblocks;                   // written by the builder's size/clear kernel
    const unsigned long long* build_count;    // survivors of the building visit
    int64_t build_rows;                       // rows of the building table
    int32_t build_level;                      // the building visit's level in this pass's DAG
    int32_t pad;
    const uint64_t* hin;                      // backward list probe: this edge's key hash of every
                                              // listed survivor (slot-aligned with list_ids), or nullptr
                                              // (the list kernel then gathers and hashes the keys)
};

// An outgoing edge: the visit's key column(s) and the filter it builds.
struct BuildEdge {
    ColRef col[2];
    int32_t ncols;
    int32_t edge_id;
    uint32_t* filter;
    int64_t* nblocks;
    int64_t probe_rows;  // rows of the table at the other end (size rule)
    uint64_t* hout;      // the insert also stores each survivor's key hash here (slot-aligned with
                         // ids), for the backward pass's probe of this edge; nullptr: not stored
};

struct FilterCfg {
    int32_t bits_per_key;
    int32_t k;
    int32_t block_bits;
    int32_t probe_order;  // order of a visit's incoming probes: 0 = builder level, then LIP, then
                          // edge id; 1 = LIP, then edge id; 2 = edge id (results never depend on it)
    uint64_t seed;
};

// Everything one visit (table, pass) needs.  Passed by value as a kernel
// parameter (well under the 4 KB parameter limit).
struct VisitArgs {
    int64_t n;                       // rows
    const uint32_t* in_bits;         // input bitmap or nullptr (= all rows)
    uint32_t* out_bits;              // survivor bitmap
    uint32_t* ids;                   // compacted survivor row ids (nullptr: not needed by any later step)
    uint32_t* seg_count;             // survivors per scan warp (segment), nullptr if ids is
    unsigned long long* count;       // total survivors (zeroed before the pass)
    unsigned long long* stats;       // [0] probe sectors, [1] build sectors (zeroed before the pass);
                                     // [2] the part of [0] a first-probe pass read (only with one)
    int32_t n_in;
    int32_t n_out;
    int32_t n_bcols;
    int32_t words_per_warp;          // bitmap words per scan warp; segment s starts at row s*32*wpw
    int32_t smem_words;              // shared-memory filter budget of one CTA (uint32 words)
    int32_t total_warps;             // scan warps launched (= segments)
    int32_t cluster;                 // CTAs per thread-block cluster of the scan (1, 2 or 4)
    int32_t level_lo;                // the scan probes only the incoming edges whose build_level is
    int32_t level_hi;                // >= level_lo and, unless level_hi is 0, < level_hi (an early
                                     // scan takes the edges whose builders finish first)
    int32_t insert_sizes;            // 1: no size/clear launch -- the scan (or list probe) zeroes the
                                     // outgoing filters' words of the previous run (out[].nblocks
                                     // still holds its sizes) and the insert sizes the filters
    int32_t n_clear_extra;           // out[n_out .. n_out + n_clear_extra): filters of the table's
                                     // next-pass visit (only filter and nblocks set) whose words of
                                     // the previous run this visit's scan zeroes as well
    int32_t insert_bsec;             // 1: the insert counts the build columns' sectors holding a
                                     // survivor into stats[1] (no scan ran for the visit)
    const int32_t* first_in;         // in[] index of the edge a first-probe pass already tested
                                     // (in_bits then holds its survivors), or nullptr
    const uint32_t* list_ids;        // backward list probe: the forward survivors' ids, in segments
                                     // of words_per_warp * 32 slots (total_warps segments)
    const uint32_t* list_seg;        // survivors per forward segment
    ProbeEdge in[kMaxIn];
    BuildEdge out[kMaxOut];
    ColRef bcol[kMaxBuildCols];
};

// One task of a batched launch: part `part` of visit `visit` (an index into
// the launch's VisitArgs array).  For scans, part is the CTA index in the
// visit's grid; for size/clear and insert, one of the launch's `parts`.
struct BatchTask {
    int32_t visit;
    int32_t part;
};

// Launchers (return the launch error, if any).
//
// launch_probe_first: the first probe (in probe order) of a visit whose rows
// are all alive (a.in_bits is ignored).  Records the in[] index of that edge
// at *first, writes the rows that pass it to `mid` (ceil(n/32) words) and adds
// its key sectors to a.stats[2] and a.stats[0].  The filter is copied into
// shared memory when it fits smem_words; smem is the dynamic shared memory
// of the launch (>= smem_words * 4).
// gate 0 runs always; gate 1 only if the filter fits gate_words, gate 2 only
// if it does not (a pair of launches, with and without the shared-memory
// budget, of which exactly one does the work: a filter that cannot fit
// leaves the whole L1 to the probes through it).
cudaError_t launch_probe_first(const VisitArgs& a, const FilterCfg& f, uint32_t* mid, int32_t* first,
                               int32_t smem_words, int32_t gate_words, int32_t gate, int grid, int block,
                               size_t smem, cudaStream_t s);
int probe_first_max_ctas_per_sm(int block_bits, int block, size_t smem);
int insert_max_ctas_per_sm(int block_bits, int block);  // resident insert CTAs of `block` threads
// Parts a batched first probe of a visit of n rows is split into (host and
// device agree on it): about kFirstTilesPerPart tiles each.
constexpr int64_t kFirstTilesPerPart = 1024;
__host__ __device__ inline int64_t first_parts(int64_t n) {
    const int64_t tiles = (n + kFirstTileRows - 1) / kFirstTileRows;
    const int64_t p = (tiles + kFirstTilesPerPart - 1) / kFirstTilesPerPart;
    return p < 1 ? 1 : p;
}
// launch_probe_first_batch: the first probes of a batch's visits (task t is
// part tasks[t].part of visit tasks[t].visit); a visit's in_bits receives the
// rows that pass and first_in the in[] index of the edge it took.  The filter
// goes to shared memory when it fits smem_words; gate and gate_words as for
// launch_probe_first, per task.
cudaError_t launch_probe_first_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                                     const FilterCfg& f, int32_t smem_words, int32_t gate_words, int32_t gate,
                                     int grid, size_t smem, cudaStream_t s);
int probe_first_batch_max_ctas_per_sm(int block_bits, size_t smem);
// pdl: launch with programmatic stream serialization (the kernel may start
// while the previous kernel on the stream runs; it waits for that kernel's
// results with griddepcontrol.wait before touching memory).
cudaError_t launch_scan(const VisitArgs& a, const FilterCfg& f, int grid, int block, size_t smem,
                        cudaStream_t s, bool pdl = false);
cudaError_t launch_size_clear(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s);
// launch_pass_through: for a backward visit that probes nothing (its survivors
// are its forward ones), zero its filters' words of the previous run and add
// its build columns' sectors (from a.out_bits) to a.stats[1].
cudaError_t launch_pass_through(const VisitArgs& a, const FilterCfg& f, int grid, cudaStream_t s, bool pdl);
cudaError_t launch_insert(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s,
                          bool pdl = false);
// launch_probe_list: a backward visit over the forward survivors listed at
// a.list_ids / a.list_seg, probing with the stored hashes in[].hin; writes
// a.out_bits (every word of the table), a.ids / a.seg_count (same segment
// geometry), a.count and a.stats.  grid * block / 32 warps walk the
// a.total_warps segments.
cudaError_t launch_probe_list(const VisitArgs& a, const FilterCfg& f, int grid, size_t smem, cudaStream_t s,
                              bool pdl = false);
cudaError_t probe_list_set_smem_limit(int block_bits, size_t smem);

// Batched launches read their task range {first, count} from device memory
// (range[0], range[1]) so that one captured graph serves every batch.
cudaError_t launch_scan_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                              const FilterCfg& f, int cluster, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_size_clear_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                                    int parts, const FilterCfg& f, int grid, int block, cudaStream_t s);
cudaError_t launch_insert_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range, int parts,
                                const FilterCfg& f, int grid, int block, cudaStream_t s);
int scan_batch_max_ctas_per_sm(int block_bits, int block, size_t smem);
cudaError_t scan_batch_set_smem_limit(int block_bits, size_t smem);

// Join phase: a slot of the device hash table that sums row weights per key
// (state 0 empty, 1 claimed, 2 ready; zero-filled before a build).
struct JoinSlot {
    unsigned long long a, b;  // the key (b = 0 for a one-column key)
    unsigned long long sum;   // summed weights of the rows with that key
    unsigned state;
    unsigned pad;
};
// w[r] = bit r of `bits` (n rows).
cudaError_t launch_join_init(const uint32_t* bits, int64_t n, unsigned long long* w, int num_sms, cudaStream_t s);
// Sum w over the rows of each key (c0, c1 when ncols == 2) into `table`
// (mask + 1 slots, a power of two); *err: 1 = a wait on a claimed slot ran
// out, 2 = the table is full.
cudaError_t launch_join_build(const ColRef& c0, const ColRef& c1, int32_t ncols, const unsigned long long* w, int64_t n,
                              JoinSlot* table, uint64_t mask, int32_t* err, int num_sms, cudaStream_t s);
// w[r] *= the sum under row r's key (0 when absent).
cudaError_t launch_join_probe(const ColRef& c0, const ColRef& c1, int32_t ncols, unsigned long long* w, int64_t n,
                              const JoinSlot* table, uint64_t mask, int num_sms, cudaStream_t s);
// *out += sum of w (out zeroed by the caller).
cudaError_t launch_join_sum(const unsigned long long* w, int64_t n, unsigned long long* out, int num_sms,
                            cudaStream_t s);

// Message returned by pt_last_error(NULL) (calls that have no context).
void set_global_error(const char* msg);

// CTAs of the scan kernel (sparse: the one for visits with an input bitmap)
// that fit on one SM for this shape.
int scan_max_ctas_per_sm(int block_bits, int block, size_t smem, bool sparse);
cudaError_t scan_set_smem_limit(int block_bits, size_t smem);

}  // namespace pt
