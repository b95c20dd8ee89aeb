// pt_visit_static: one transfer visit that allocates no memory.
//
// Some callers cannot call cudaMalloc: engines that hand all device memory
// to their own pool up front and forbid other allocations, latency-bound
// paths where an allocation (which can synchronize the device) is not
// acceptable, and hosts that must not fail with an out-of-memory error
// mid-query.  For
// them this entry point runs the same three kernels as a planned context
// (scan, size/clear, insert) for a single visit, with every input and
// output supplied by the caller and the kernels' scratch -- the compacted
// row ids, the per-warp segment lengths and the counters -- taken from a
// fixed array in device memory that is part of the library image.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pt.h"
#include "pt_internal.h"

namespace {

constexpr int64_t kStaticMaxWarps = 16384;  // >= SMs x 64 resident warps on any current GPU
constexpr size_t kCounterBytes = 256;       // survivor count, two sector counters, a zero word
constexpr size_t kSegBytes = (size_t)kStaticMaxWarps * 4;
constexpr size_t kIdsBytes = (size_t)PT_STATIC_MAX_ROWS * 4;
constexpr size_t kScratchBytes = kCounterBytes + kSegBytes + kIdsBytes;

// The scratch every call shares (about 4.1 MB on every GPU that loads the
// library, kept until the process exits).
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

pt_status fail(pt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pt::set_global_error(buf);
    return st;
}

// Device address of the scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current.
pt_status scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PT_ERR_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return fail(PT_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PT_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

pt_status check_col(const pt_column& c, int64_t n, const char* what, int i) {
    if (c.dtype != PT_I32 && c.dtype != PT_I64) return fail(PT_ERR_INVALID, "%s %d: dtype %d", what, i, c.dtype);
    if (c.mem != PT_MEM_DEVICE) return fail(PT_ERR_INVALID, "%s %d: columns must be device memory", what, i);
    if (n > 0 && !c.data) return fail(PT_ERR_INVALID, "%s %d: data is NULL", what, i);
    if (!aligned(c.data, c.dtype == PT_I32 ? 4 : 8)) return fail(PT_ERR_INVALID, "%s %d: misaligned column", what, i);
    return PT_OK;
}

pt::ColRef ref(const pt_column& c) {
    pt::ColRef r{};
    r.p = c.data;
    r.dtype = c.dtype;
    return r;
}

}  // namespace

extern "C" pt_status pt_visit_static(const pt_filter_cfg* cfg, void* cuda_stream, int64_t n_rows,
                                     const uint32_t* in_bits, int32_t n_in, const pt_static_probe* in,
                                     int32_t n_out, const pt_static_build* out, uint32_t* out_bits,
                                     int64_t* count_out) {
    if (!cfg) return fail(PT_ERR_INVALID, "cfg is NULL");
    if (cfg->block_bits != 256 && cfg->block_bits != 512) return fail(PT_ERR_INVALID, "block_bits %d", cfg->block_bits);
    if (cfg->k < 1 || cfg->k > 16) return fail(PT_ERR_INVALID, "k %d", cfg->k);
    if (cfg->bits_per_key < 1 || cfg->bits_per_key > 64) return fail(PT_ERR_INVALID, "bits_per_key %d", cfg->bits_per_key);
    if (n_rows < 0 || n_rows > PT_STATIC_MAX_ROWS)
        return fail(PT_ERR_INVALID, "n_rows %lld exceeds the allocation-free limit of %d rows", (long long)n_rows,
                    PT_STATIC_MAX_ROWS);
    if (n_in < 0 || n_in > pt::kMaxIn || (n_in > 0 && !in)) return fail(PT_ERR_INVALID, "n_in %d", n_in);
    if (n_out < 0 || n_out > pt::kMaxOut || (n_out > 0 && !out)) return fail(PT_ERR_INVALID, "n_out %d", n_out);
    if (n_rows > 0 && !out_bits) return fail(PT_ERR_INVALID, "out_bits is NULL");
    pt_status st;
    for (int i = 0; i < n_in; ++i) {
        if (in[i].ncols < 1 || in[i].ncols > 2) return fail(PT_ERR_INVALID, "probe %d: ncols %d", i, in[i].ncols);
        for (int j = 0; j < in[i].ncols; ++j)
            if ((st = check_col(in[i].col[j], n_rows, "probe", i)) != PT_OK) return st;
        if (!in[i].filter || !aligned(in[i].filter, 16) || !in[i].nblocks)
            return fail(PT_ERR_INVALID, "probe %d: filter and nblocks must be 16-byte aligned device pointers", i);
    }
    const pt::FilterCfg f{cfg->bits_per_key, cfg->k, cfg->block_bits, 0, cfg->seed};
    for (int i = 0; i < n_out; ++i) {
        if (out[i].ncols < 1 || out[i].ncols > 2) return fail(PT_ERR_INVALID, "build %d: ncols %d", i, out[i].ncols);
        for (int j = 0; j < out[i].ncols; ++j)
            if ((st = check_col(out[i].col[j], n_rows, "build", i)) != PT_OK) return st;
        if (!out[i].filter || !aligned(out[i].filter, 16) || !out[i].nblocks_out)
            return fail(PT_ERR_INVALID, "build %d: filter and nblocks_out must be 16-byte aligned device pointers", i);
        const int64_t m = n_rows < out[i].probe_rows ? n_rows : out[i].probe_rows;
        int64_t need = (m * f.bits_per_key + f.block_bits - 1) / f.block_bits;
        if (need < 1) need = 1;
        if (out[i].probe_rows < 0 || out[i].capacity_blocks < need)
            return fail(PT_ERR_INVALID, "build %d: filter holds %lld blocks, the size rule may need %lld",
                        i, (long long)out[i].capacity_blocks, (long long)need);
    }

    void* scratch = nullptr;
    if ((st = scratch_for_current_device(&scratch)) != PT_OK) return st;
    unsigned char* base = (unsigned char*)scratch;
    unsigned long long* counters = (unsigned long long*)base;  // [0] count, [1..2] sectors, [3] zero
    uint32_t* seg = (uint32_t*)(base + kCounterBytes);
    uint32_t* ids = (uint32_t*)(base + kCounterBytes + kSegBytes);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "device query: %s", cudaGetErrorString(e));

    // Launch shape within the default 48 KB of shared memory per CTA (46 KB
    // dynamic plus the kernel's static part), so no kernel attribute is
    // changed: the most warps (8, 4, 2 or 1) whose per-warp queues fit, and
    // the rest of the 46 KB for filters.
    constexpr size_t kStaticSmem = 46 * 1024;
    int warps_per_cta = 8;
    while (warps_per_cta > 1 && (size_t)warps_per_cta * pt::scan_warp_smem_bytes(n_in) > kStaticSmem) warps_per_cta /= 2;
    const int block = warps_per_cta * 32;
    const size_t queues = (size_t)warps_per_cta * pt::scan_warp_smem_bytes(n_in);
    if (queues > kStaticSmem) return fail(PT_ERR_UNSUPPORTED, "%d incoming filters need more shared memory than 46 KB", n_in);
    const size_t filt = n_in > 0 ? (kStaticSmem - queues) / 16 * 16 : 0;
    const size_t smem = filt + queues;
    int fit = pt::scan_max_ctas_per_sm(cfg->block_bits, block, smem, in_bits != nullptr);
    if (fit < 1) fit = 1;
    const int64_t n_words = (n_rows + 31) / 32;
    int64_t grid = (n_words + pt::kChunkWords - 1) / pt::kChunkWords;
    grid = (grid + warps_per_cta - 1) / warps_per_cta;
    if (grid < 1) grid = 1;
    if (grid > (int64_t)sms * fit) grid = (int64_t)sms * fit;
    while (grid * warps_per_cta > kStaticMaxWarps) --grid;
    const int total_warps = (int)(grid * warps_per_cta);
    int64_t wpw = (n_words + total_warps - 1) / total_warps;
    wpw = (wpw + pt::kChunkWords - 1) / pt::kChunkWords * pt::kChunkWords;
    if (wpw < pt::kChunkWords) wpw = pt::kChunkWords;

    pt::VisitArgs a;
    std::memset(&a, 0, sizeof a);
    a.n = n_rows;
    a.in_bits = in_bits;
    a.out_bits = out_bits;
    a.count = counters + 0;
    a.stats = counters + 1;
    a.n_in = n_in;
    a.n_out = n_out;
    a.words_per_warp = (int32_t)wpw;
    a.total_warps = total_warps;
    a.smem_words = (int32_t)(filt / 4);
    for (int i = 0; i < n_in; ++i) {
        pt::ProbeEdge& pe = a.in[i];
        pe.ncols = in[i].ncols;
        pe.edge_id = i;  // probed in the order given: every build count reads the zero word
        pe.col[0] = ref(in[i].col[0]);
        pe.col[1] = in[i].ncols == 2 ? ref(in[i].col[1]) : pe.col[0];
        pe.filter = in[i].filter;
        pe.nblocks = in[i].nblocks;
        pe.build_count = counters + 3;
        pe.build_rows = 1;
    }
    for (int i = 0; i < n_out; ++i) {
        pt::BuildEdge& be = a.out[i];
        be.ncols = out[i].ncols;
        be.edge_id = i;
        be.col[0] = ref(out[i].col[0]);
        be.col[1] = out[i].ncols == 2 ? ref(out[i].col[1]) : be.col[0];
        be.filter = out[i].filter;
        be.nblocks = out[i].nblocks_out;
        be.probe_rows = out[i].probe_rows;
        for (int j = 0; j < out[i].ncols; ++j) {
            const void* p = out[i].col[j].data;
            bool dup = false;
            for (int b = 0; b < a.n_bcols; ++b) dup |= a.bcol[b].p == p;
            if (!dup && a.n_bcols < pt::kMaxBuildCols) a.bcol[a.n_bcols++] = ref(out[i].col[j]);
        }
    }
    if (n_out > 0) {
        a.ids = ids;
        a.seg_count = seg;
    }

    // The counters start every call at zero; the ids and segment lengths are
    // written by the scan before the insert reads them.
    e = cudaMemsetAsync(counters, 0, kCounterBytes, stream);
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    e = pt::launch_scan(a, f, (int)grid, block, smem, stream);
    if (e != cudaSuccess) return fail(PT_ERR_CUDA, "scan launch: %s", cudaGetErrorString(e));
    if (n_out > 0) {
        int64_t words = 0;
        for (int i = 0; i < n_out; ++i) {
            const int64_t w = out[i].capacity_blocks * (cfg->block_bits / 32);
            words = w > words ? w : words;
        }
        int64_t gc = (words / 4 + 511) / 512;
        if (gc < 1) gc = 1;
        if (gc > (int64_t)sms * 4) gc = (int64_t)sms * 4;
        e = pt::launch_size_clear(a, f, (int)gc, 512, stream);
        if (e != cudaSuccess) return fail(PT_ERR_CUDA, "size/clear launch: %s", cudaGetErrorString(e));
        int gi = total_warps / 16 + 1;
        if (gi > sms * 4) gi = sms * 4;
        e = pt::launch_insert(a, f, gi, 512, stream);
        if (e != cudaSuccess) return fail(PT_ERR_CUDA, "insert launch: %s", cudaGetErrorString(e));
    }
    if (count_out) {
        e = cudaMemcpyAsync(count_out, counters, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return fail(PT_ERR_CUDA, "count copy: %s", cudaGetErrorString(e));
    }
    return PT_OK;
}
