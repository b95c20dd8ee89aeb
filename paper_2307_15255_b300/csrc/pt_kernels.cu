// Device kernels of one predicate-transfer visit (Section 3.2, "Filter
// Transformation"): scan (probe + survivor bitmap + compaction), size and
// clear of the outgoing filters, and insert.
//
// A visit runs as three launches on the context's stream:
//   1. pt_scan_kernel    -- streams the input bitmap and the probed key
//      columns; for every row still alive it hashes the key and tests the
//      incoming filter (held in shared memory when it fits the CTA's
//      budget, else read through L1/L2); __ballot_sync turns the 32 lanes'
//      verdicts into one survivor word; survivors are compacted into
//      per-warp segments of row ids with __popc prefix ranks.
//   2. pt_size_clear_kernel -- reads the survivor count on the device (no
//      host synchronization), sizes every outgoing filter and zeroes the
//      blocks it will use.
//   3. pt_insert_kernel  -- walks the compacted ids, gathers the outgoing
//      key(s), hashes them and sets k bits with word-level atomicOr.
#include <cooperative_groups.h>

#include "pt_internal.h"

namespace pt {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hash_key(uint64_t x, uint64_t seed) { return mix64((x ^ seed) + kGamma); }

// Loads of data a kernel reads once (key columns, bitmaps, row lists): through
// the read-only path without allocating in L1, which is left to the filters
// probed through it.  Volatile, so that none moves above a kernel's
// griddepcontrol.wait.
__device__ __forceinline__ int32_t ld_once(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_once(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ long long ld_once(const long long* p) {
    long long v;
    asm volatile("ld.global.nc.L1::no_allocate.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned long long ld_once(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.nc.L1::no_allocate.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
// Key of row r as u64; int32 values are sign-extended.
__device__ __forceinline__ uint64_t load_key(const ColRef& c, uint32_t r) {
    if (c.dtype == 0) return (uint64_t)(int64_t)ld_once(reinterpret_cast<const int32_t*>(c.p) + r);
    return (uint64_t)ld_once(reinterpret_cast<const long long*>(c.p) + r);
}

// Hash of row r's key on an edge.  A first column of dtype kHashed already
// holds H(x) of its key (precomputed for resident tables), so only the
// composite step, if any, is left.
__device__ __forceinline__ uint64_t edge_hash(const ColRef& c0, const ColRef& c1, int ncols, uint32_t r,
                                              uint64_t seed) {
    const uint64_t a = load_key(c0, r);
    const uint64_t h = c0.dtype == kHashed ? a : hash_key(a, seed);
    if (ncols == 2) return mix64(h ^ load_key(c1, r));
    return h;
}

// 32-byte sectors of a column holding at least one set row of a 32-row
// word: 8 rows per sector for int32 (4 sectors), 4 rows for int64 (8).
__device__ __forceinline__ uint32_t sectors_of(uint32_t m, int32_t dtype) {
    if (dtype == 0) {
        m |= m >> 4;
        m |= m >> 2;
        m |= m >> 1;
        return __popc(m & 0x01010101u);
    }
    m |= m >> 2;
    m |= m >> 1;
    return __popc(m & 0x11111111u);
}

// The k bit positions of a key, written so that the index arithmetic runs on
// the multiply-add pipe and only the final shift and AND use the integer ALU
// (the scan is bound by the ALU pipe otherwise).  With lo = (uint32)h and
// h2 = (lo >> 16) | 1, a_i = lo + i*h2 agrees with (h1 + i*h2) mod B in its
// low log2(B) bits; a_i << (32 - log2 B) puts that bit index in the top
// log2(B) bits, so its word inside the block is mulhi(a_i << .., B/32) and
// its bit inside the word is a_i & 31 (the wrap-mode funnel shift uses the
// low 5 bits of the shift amount).
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t mul_hi(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t rot_r(uint32_t x, uint32_t n) {
    uint32_t d;
    asm("shf.r.wrap.b32 %0, %1, %1, %2;" : "=r"(d) : "r"(x), "r"(n));
    return d;
}
__device__ __forceinline__ void red_or_shared(uint32_t saddr, uint32_t v) {
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t saddr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr));
    return v;
}

// Block-wide copy of n16 16-byte chunks from global into shared memory, with
// four independent loads per thread in flight (a filter copy then costs one
// or two L2 round trips, not one per chunk a thread moves).
__device__ __forceinline__ void copy_to_smem(uint4* dst, const uint4* __restrict__ src, uint32_t n16) {
    constexpr uint32_t U = 4;
    uint32_t t = threadIdx.x;
    for (; t + (U - 1) * blockDim.x < n16; t += U * blockDim.x) {
        uint4 v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) v[u] = __ldg(src + t + u * blockDim.x);
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) dst[t + u * blockDim.x] = v[u];
    }
    for (; t < n16; t += blockDim.x) dst[t] = __ldg(src + t);
}

// Address in CTA `rank` of this cluster of the shared-memory location at
// (this CTA's) shared-window address `addr`, and a load through it.
__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
    return d;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel on its stream still
// runs.  grid_dependency_wait() returns once that kernel has completed and its
// memory operations are visible (at once for a kernel launched without the
// attribute); allow_dependents() lets the next such kernel on the stream
// launch once every CTA of this one has called it or exited.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <int B>
struct BlockBits {
    static constexpr uint32_t LOGB = B == 256 ? 8 : 9;
    static constexpr uint32_t SCALE = 1u << (32 - LOGB);
    static constexpr uint32_t WPB = B / 32;
};

// Probe one key in a filter held in shared memory at byte address sbase
// (shared window): all k bits of its block set?  KT > 0 fixes k at compile
// time; KT == 0 reads it at run time.
template <int B, int KT>
__device__ __forceinline__ bool probe_shared(uint32_t sbase, uint32_t nb, uint64_t h, int k) {
    using BB = BlockBits<B>;
    const uint32_t lo = (uint32_t)h;
    const uint32_t blk = mad_lo(mul_hi((uint32_t)(h >> 32), nb), B / 8, sbase);  // byte address of the block
    const uint32_t h2 = (lo >> 16) | 1u;
    const int kk = KT > 0 ? KT : k;
    uint32_t ok = 0xFFFFFFFFu;
#pragma unroll 4
    for (int i = 0; i < kk; ++i) {
        const uint32_t ai = mad_lo((uint32_t)i, h2, lo);
        const uint32_t wi = mul_hi(mad_lo(ai, BB::SCALE, 0u), BB::WPB);
        ok &= rot_r(lds_u32(mad_lo(wi, 4u, blk)), ai);
    }
    return ok & 1u;
}

template <int B, int KT>
__device__ __forceinline__ bool probe_global(const uint32_t* __restrict__ f, uint32_t nb, uint64_t h, int k) {
    using BB = BlockBits<B>;
    const uint32_t lo = (uint32_t)h;
    const uint32_t* blk = f + (size_t)mul_hi((uint32_t)(h >> 32), nb) * BB::WPB;
    const uint32_t h2 = (lo >> 16) | 1u;
    const int kk = KT > 0 ? KT : k;
    uint32_t ok = 0xFFFFFFFFu;
#pragma unroll 4
    for (int i = 0; i < kk; ++i) {
        const uint32_t ai = mad_lo((uint32_t)i, h2, lo);
        const uint32_t wi = mul_hi(mad_lo(ai, BB::SCALE, 0u), BB::WPB);
        ok &= rot_r(__ldg(blk + wi), ai);
    }
    return ok & 1u;
}

// Probes of R keys at once.  In shared memory, every key tests its k bits
// (measured faster than skipping loads, which costs branches on an
// ALU-bound stream).  Through L1/L2, in two steps: step 1 tests bit 0 of
// every key -- a key that is not in the filter fails it with probability
// 1 - (fill of its block), about 78% at 16 bits per key -- and step 2 tests
// bits 1..k-1 only for the keys that passed, so lanes whose key failed
// issue no load and take no L1 tag lookup.  The verdicts equal the
// one-key probes above: all k bits set.
template <int B, int KT, int R>
__device__ __forceinline__ void probe_shared_n(uint32_t sbase, uint32_t nb, const uint64_t* h, int k, bool* pass) {
#pragma unroll
    for (int i = 0; i < R; ++i) pass[i] = probe_shared<B, KT>(sbase, nb, h[i], k);
}

template <int B, int KT, int R>
__device__ __forceinline__ void probe_global_n(const uint32_t* __restrict__ f, uint32_t nb, const uint64_t* h, int k,
                                               bool* pass) {
    using BB = BlockBits<B>;
    uint32_t lo[R], bi[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        lo[i] = (uint32_t)h[i];
        bi[i] = mul_hi((uint32_t)(h[i] >> 32), nb);
        const uint32_t w0 = mul_hi(mad_lo(lo[i], BB::SCALE, 0u), BB::WPB);
        pass[i] = rot_r(__ldg(f + (size_t)bi[i] * BB::WPB + w0), lo[i]) & 1u;
    }
    const int kk = KT > 0 ? KT : k;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        if (pass[i]) {
            const uint32_t* blk = f + (size_t)bi[i] * BB::WPB;
            const uint32_t h2 = (lo[i] >> 16) | 1u;
            uint32_t ok = 0xFFFFFFFFu;
#pragma unroll 4
            for (int t = 1; t < kk; ++t) {
                const uint32_t at = mad_lo((uint32_t)t, h2, lo[i]);
                ok &= rot_r(__ldg(blk + mul_hi(mad_lo(at, BB::SCALE, 0u), BB::WPB)), at);
            }
            pass[i] = ok & 1u;
        }
    }
}

// probe_global_n for rows of which only some are live: a row that is not
// live issues no load and does not pass.
template <int B, int KT, int R>
__device__ __forceinline__ void probe_global_live(const uint32_t* __restrict__ f, uint32_t nb, const uint64_t* h,
                                                  int k, const bool* live, bool* pass) {
    using BB = BlockBits<B>;
    uint32_t lo[R], bi[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        lo[i] = (uint32_t)h[i];
        bi[i] = mul_hi((uint32_t)(h[i] >> 32), nb);
        pass[i] = false;
        if (live[i]) {
            const uint32_t w0 = mul_hi(mad_lo(lo[i], BB::SCALE, 0u), BB::WPB);
            pass[i] = rot_r(__ldg(f + (size_t)bi[i] * BB::WPB + w0), lo[i]) & 1u;
        }
    }
    const int kk = KT > 0 ? KT : k;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        if (pass[i]) {
            const uint32_t* blk = f + (size_t)bi[i] * BB::WPB;
            const uint32_t h2 = (lo[i] >> 16) | 1u;
            uint32_t ok = 0xFFFFFFFFu;
#pragma unroll 4
            for (int t = 1; t < kk; ++t) {
                const uint32_t at = mad_lo((uint32_t)t, h2, lo[i]);
                ok &= rot_r(__ldg(blk + mul_hi(mad_lo(at, BB::SCALE, 0u), BB::WPB)), at);
            }
            pass[i] = ok & 1u;
        }
    }
}

// Probe a filter spread over the CTAs of a cluster of 2^lc CTAs: block j is
// block j >> lc of the part held by CTA j & (2^lc - 1), at byte address
// sbase in every CTA's shared window.
template <int B, int KT>
__device__ __forceinline__ bool probe_cluster(uint32_t sbase, uint32_t lc, uint32_t nb, uint64_t h, int k) {
    using BB = BlockBits<B>;
    const uint32_t lo = (uint32_t)h;
    const uint32_t j = mul_hi((uint32_t)(h >> 32), nb);
    const uint32_t blk = mapa_u32(mad_lo(j >> lc, B / 8, sbase), j & ((1u << lc) - 1u));
    const uint32_t h2 = (lo >> 16) | 1u;
    const int kk = KT > 0 ? KT : k;
    uint32_t ok = 0xFFFFFFFFu;
#pragma unroll 4
    for (int i = 0; i < kk; ++i) {
        const uint32_t ai = mad_lo((uint32_t)i, h2, lo);
        const uint32_t wi = mul_hi(mad_lo(ai, BB::SCALE, 0u), BB::WPB);
        ok &= rot_r(ld_cluster_u32(mad_lo(wi, 4u, blk)), ai);
    }
    return ok & 1u;
}

// ---------------------------------------------------------------------------
// 1. scan: probe every incoming filter, write the survivor bitmap, compact
//
// Each warp owns a contiguous chunk of bitmap words and walks it in rounds
// of 128 words (4096 rows): one coalesced load brings four input words per
// lane.  Rows still alive wait in a per-warp queue in front of each probe
// stage (incoming edges in probe order); a stage runs once its queue holds
// kDrain rows, kDrain/32 rows per lane, so every probe works on densely
// packed live rows and each lane has independent key loads in flight.
// Survivors of a stage are appended, in row order, to the next stage's
// queue; survivors of the last stage set their bit in the round's output
// words in shared memory, which are stored at the end of the round.  The
// queues are not emptied at round ends: on a sparse input they fill over
// several rounds, so the stages keep running full batches, and rows queued
// in an earlier round set their output bit directly in the bitmap.  After
// the chunk's last round the queues are flushed, and the survivors' row
// ids are compacted into the warp's segment of the id array from its
// finished output words.
//
// Sector accounting: rows enter every stage in ascending row order, so the
// key sectors a stage reads are the rows whose sector differs from that of
// the row that entered the same stage before them.
// ---------------------------------------------------------------------------
// Shared state of one scan CTA besides the dynamic filter/queue area.
struct ScanShared {
    ProbeEdge pe[kMaxIn];  // incoming edges in probe order
    int32_t off[kMaxIn];   // word offset of the filter in smem, or -1: probe from global
    uint32_t nb[kMaxIn];
    uint32_t split[kMaxIn];  // 1: the filter is spread over the cluster (this CTA holds its part)
    int32_t n_in;            // edges this kernel probes (a first-probe pass may have taken one)
    unsigned long long sum[3];  // the CTA's survivors and key sectors (see warp_to_cta)
};

// Counters that every warp of a grid adds to (a visit's survivor count and its
// sector accounting) are summed per CTA in shared memory first, and one thread
// of the CTA adds the sums to the global counters: atomics on one address are
// serialised at one L2 slice, about 2 ns apiece on B300 (measured: three
// counters added by each of 3552 warps took 7.9 us, by each of 444 CTAs 1.9 us).
// Lane 0 of each warp calls warp_to_cta; after a __syncthreads, thread 0 calls
// cta_to_global, which also clears the CTA's sum for the block's next task.
__device__ __forceinline__ void warp_to_cta(unsigned long long* s, unsigned long long v) {
    if (v) atomicAdd(s, v);
}
__device__ __forceinline__ void cta_to_global(unsigned long long* s, unsigned long long* g) {
    if (*s) atomicAdd(g, *s);
    *s = 0;
}

// With a.insert_sizes, zero this visit's outgoing filters as the previous run
// left them (out[e].nblocks blocks each; the words past them are still zero
// from the run before, or from the allocation), in 16-byte stores spread over
// the visit's n_ctas CTAs.  The insert, which follows on the same stream,
// then sizes the filters and sets their bits.  a.n_clear_extra more entries
// of out[] are filters the table's next-pass visit builds, when that visit
// runs no scan of its own (its insert follows later in the same run).
__device__ __forceinline__ void clear_previous_filters(const VisitArgs& a, int block_bits, int64_t cta, int64_t n_ctas) {
    if (!a.insert_sizes) return;
    const size_t tid = (size_t)cta * blockDim.x + threadIdx.x, stride = (size_t)n_ctas * blockDim.x;
    for (int e = 0; e < a.n_out + a.n_clear_extra; ++e) {
        uint4* p = reinterpret_cast<uint4*>(a.out[e].filter);
        const size_t n16 = (size_t)*a.out[e].nblocks * (size_t)(block_bits / 128);
        for (size_t i = tid; i < n16; i += stride) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Probe order (mode 0, the default): incoming edges by ascending level of the
// building visit (its longest path from a source of the pass's DAG: filters
// finished earlier come first), then ascending survivors/rows of the building
// visit (LIP-style, Section 3.2 "Transfer Schedule"), then edge id.  Mode 1
// leaves the level out (the LIP ratio, then edge id); mode 2 is edge id alone
// (unordered).  in[skip] is left out (skip < 0: none), and so is every edge
// whose build_level is outside [a.level_lo, a.level_hi) (level_hi 0: no upper
// bound).  Writes the in[]
// indexes to ord and returns their number; nbs[i] receives in[i]'s filter
// size in blocks (every count and size is loaded at once: one round trip).
// One thread.  In mode 0 the first edge depends only on the counts of the
// lowest-level builders, so it can be taken while higher-level builders
// still run (their sizes are then not read by the caller).
__device__ __forceinline__ int lip_order(const VisitArgs& a, int skip, int mode, int* ord, uint32_t* nbs) {
    unsigned long long c[kMaxIn];
    int m = 0;
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i) {
        c[i] = i < a.n_in ? *a.in[i].build_count : 0ull;
        nbs[i] = i < a.n_in ? (uint32_t)*a.in[i].nblocks : 0u;
        const bool in_range = i < a.n_in && a.in[i].build_level >= a.level_lo &&
                              (a.level_hi == 0 || a.in[i].build_level < a.level_hi);
        if (in_range && i != skip) ord[m++] = i;
    }
    for (int i = 1; i < m; ++i) {
        const int x = ord[i];
        int j = i - 1;
        while (j >= 0) {
            const int y = ord[j];
            const int32_t lx = mode == 0 ? a.in[x].build_level : 0, ly = mode == 0 ? a.in[y].build_level : 0;
            const unsigned long long lhs = mode == 2 ? 0ull : c[x] * (unsigned long long)a.in[y].build_rows;
            const unsigned long long rhs = mode == 2 ? 0ull : c[y] * (unsigned long long)a.in[x].build_rows;
            if (lx < ly || (lx == ly && (lhs < rhs || (lhs == rhs && a.in[x].edge_id < a.in[y].edge_id)))) {
                ord[j + 1] = ord[j];
                --j;
            } else {
                break;
            }
        }
        ord[j + 1] = x;
    }
    return m;
}

// One CTA of a visit's scan: `cta` is its index in the visit's grid of
// total_warps / (blockDim.x / 32) CTAs.  Every thread of the block calls it.
// DENSE = false leaves out the dense sub-round path (visits whose input is a
// bitmap rarely have 32 full words in a row), which frees registers for a
// third CTA per SM.
template <int B, int KT, bool DENSE>
__device__ __forceinline__ void scan_cta(const VisitArgs& a, const FilterCfg& f, int64_t cta, uint32_t crank,
                                         uint32_t* smem, ScanShared& sh) {
    ProbeEdge* s_pe = sh.pe;
    int32_t* s_off = sh.off;
    uint32_t* s_nb = sh.nb;
    uint32_t* s_split = sh.split;
    const uint32_t C = a.cluster > 1 ? (uint32_t)a.cluster : 1u;
    const uint32_t lc = __ffs(C) - 1;  // C is 1, 2 or 4
    constexpr uint32_t WPB = B / 32;
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t sfilt = (uint32_t)__cvta_generic_to_shared(smem);  // shared-window address of the filters

    clear_previous_filters(a, B, cta, a.total_warps / (blockDim.x >> 5));
    if (threadIdx.x == 0) {
        int ord[kMaxIn];
        uint32_t nbs[kMaxIn];
        const int m = lip_order(a, a.first_in ? *a.first_in : -1, f.probe_order, ord, nbs);
        sh.n_in = m;
        sh.sum[0] = sh.sum[1] = sh.sum[2] = 0;
        // Shared-memory placement, greedily in probe order: a whole copy in
        // every CTA when it fits, else (in a cluster) 1/C of it in each CTA of
        // the cluster, else probed from global memory.  Every CTA of a cluster
        // computes the same placement from the same counts.
        int32_t used = 0;
        for (int i = 0; i < m; ++i) {
            const ProbeEdge& pe = a.in[ord[i]];
            s_pe[i] = pe;
            const uint32_t nb = nbs[ord[i]];
            s_nb[i] = nb;
            s_split[i] = 0;
            const int64_t words = (int64_t)nb * WPB;
            const int64_t part = (int64_t)((nb + C - 1) >> lc) * WPB;
            if (used + words <= a.smem_words) {
                s_off[i] = used;
                used += (int32_t)words;
            } else if (C > 1 && used + part <= a.smem_words) {
                s_off[i] = used;
                s_split[i] = 1;
                used += (int32_t)part;
            } else {
                s_off[i] = -1;
            }
        }
    }
    __syncthreads();
    const int n_in = sh.n_in;
    for (int i = 0; i < n_in; ++i) {
        if (s_off[i] < 0) continue;
        const uint4* src = reinterpret_cast<const uint4*>(s_pe[i].filter);
        uint4* dst = reinterpret_cast<uint4*>(smem + s_off[i]);
        if (!s_split[i]) {
            copy_to_smem(dst, src, s_nb[i] * (WPB / 4));
        } else {
            // this CTA's part: blocks crank, crank + C, crank + 2C, ...
            const uint32_t nl = (s_nb[i] + C - 1 - crank) >> lc;
            for (uint32_t t = threadIdx.x; t < nl * (WPB / 4); t += blockDim.x) {
                const uint32_t l = t / (WPB / 4), piece = t % (WPB / 4);
                dst[t] = __ldg(src + (size_t)((l << lc) + crank) * (WPB / 4) + piece);
            }
        }
    }
    __syncthreads();
    if (C > 1) cooperative_groups::this_cluster().sync();  // every part in place before any probe

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t* wsm = smem + a.smem_words + warp * (uint32_t)(scan_warp_smem_bytes(n_in) / 4);
    uint32_t* queue = wsm;                             // row-id queues, stage s at qoff(s)
    uint32_t* obm = wsm + scan_queue_words(n_in);      // [kRoundWords] survivors of the round
    uint32_t* last_in = obm + kRoundWords;             // [kMaxIn] last row that entered stage s

    const int64_t gw = cta * (blockDim.x >> 5) + warp;
    const int64_t n_words = (a.n + 31) >> 5;
    const int64_t w_begin = gw * a.words_per_warp;
    const int64_t w_end = min(n_words, w_begin + a.words_per_warp);
    const uint32_t tail_bits = (uint32_t)(a.n & 31);
    const int k = f.k;
    const uint64_t seed = f.seed;
    constexpr uint32_t kNoRow = 0xFFFFFFFFu;  // rows are below 2^31

    if (lane < (uint32_t)kMaxIn) last_in[lane] = kNoRow;
    unsigned long long psec = 0;  // per lane; reduced at the end
    // queue lengths (warp-uniform), 16 bits per stage: stages 0-3 in qlo, 4-7 in qhi
    uint64_t qlo = 0, qhi = 0;
    auto qget = [&](int s) -> uint32_t {
        return (uint32_t)((s < 4 ? qlo : qhi) >> (16 * (s & 3))) & 0xFFFFu;
    };
    auto qset = [&](int s, uint32_t v) {
        const uint64_t clear = ~(0xFFFFull << (16 * (s & 3))), put = (uint64_t)v << (16 * (s & 3));
        if (s < 4)
            qlo = (qlo & clear) | put;
        else
            qhi = (qhi & clear) | put;
    };
    __syncwarp();

    // Run stage s on the first cnt (<= kDrain) rows of its queue.  Survivors
    // of the last stage set their bit in obm when they belong to the round
    // starting at row round_row0, else (rows queued in an earlier round)
    // directly in the output bitmap.
    auto run_stage = [&](int s, uint32_t cnt, uint32_t round_row0) {
        uint32_t* q = queue + qoff(s);
        const ColRef c0 = s_pe[s].col[0];
        const ColRef c1 = s_pe[s].col[1];
        const int ncols = s_pe[s].ncols;
        const uint32_t sh0 = c0.dtype == 0 ? 3u : 2u, sh1 = c1.dtype == 0 ? 3u : 2u;  // log2 rows per sector
        const int32_t off = s_off[s];
        const uint32_t nb = s_nb[s];
        const uint32_t split = s_split[s];
        const uint32_t* fg = s_pe[s].filter;
        const bool last = s == n_in - 1;
        uint32_t* nq = queue + qoff(s + 1);
        uint32_t nn = last ? 0u : qget(s + 1);
        const uint32_t prev0 = last_in[s];
        // key sectors: a row whose sector differs from the previous row's entering
        // this stage (stage 0's are counted from the input words instead)
        auto count_sectors = [&](uint32_t r, uint32_t prev) {
            if (s == 0) return;
            psec += (r >> sh0) != (prev >> sh0);
            if (ncols == 2) psec += (r >> sh1) != (prev >> sh1);
        };
        auto emit = [&](bool pass, uint32_t r) {
            const uint32_t m = __ballot_sync(FULL, pass);
            if (pass) {
                if (!last)
                    nq[nn + __popc(m & lt_mask)] = r;
                else if (r >= round_row0)
                    atomicOr(obm + ((r - round_row0) >> 5), 1u << (r & 31));
                else
                    atomicOr(a.out_bits + (r >> 5), 1u << (r & 31));
            }
            nn += __popc(m);
        };
        if (cnt == (uint32_t)kDrain) {
            // a full batch: kDrain/32 rows per lane, independent gathers in flight
            constexpr int R = kDrain / 32;
            uint32_t r[R];
            uint64_t h[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint32_t idx = lane + 32u * i;
                r[i] = q[idx];
                count_sectors(r[i], idx == 0 ? prev0 : q[idx - 1]);
            }
#pragma unroll
            for (int i = 0; i < R; ++i) h[i] = edge_hash(c0, c1, ncols, r[i], seed);
            bool pass[R];
            if (off >= 0 && !split) {
                probe_shared_n<B, KT, R>(sfilt + 4u * (uint32_t)off, nb, h, k, pass);
            } else if (off >= 0) {
#pragma unroll
                for (int i = 0; i < R; ++i) pass[i] = probe_cluster<B, KT>(sfilt + 4u * (uint32_t)off, lc, nb, h[i], k);
            } else {
                probe_global_n<B, KT, R>(fg, nb, h, k, pass);
            }
            const uint32_t last_row = q[cnt - 1];
            // keep the unprocessed tail of the queue (fewer than kQueueCap - kDrain rows) at its front
            const uint32_t rest = qget(s) - cnt;
            constexpr int RT = (kQueueCap - kDrain) / 32;
            uint32_t keep[RT];
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const uint32_t idx = lane + 32u * i;
                keep[i] = idx < rest ? q[cnt + idx] : 0u;
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const uint32_t idx = lane + 32u * i;
                if (idx < rest) q[idx] = keep[i];
            }
            if (lane == 0) last_in[s] = last_row;
            qset(s, rest);
#pragma unroll
            for (int i = 0; i < R; ++i) emit(pass[i], r[i]);
        } else {
            // the rest of the queue (cnt < kDrain is the whole queue): one batch
            // with the lanes past its end idle, so that its gathers are in flight
            // together rather than one 32-row group after another
            constexpr int R = kDrain / 32;
            uint32_t r[R];
            bool live[R];
            uint64_t h[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint32_t idx = lane + 32u * i;
                live[i] = idx < cnt;
                r[i] = live[i] ? q[idx] : 0u;
                if (live[i]) count_sectors(r[i], idx == 0 ? prev0 : q[idx - 1]);
            }
#pragma unroll
            for (int i = 0; i < R; ++i) h[i] = live[i] ? edge_hash(c0, c1, ncols, r[i], seed) : 0ull;
            bool pass[R];
            if (off >= 0 && !split) {
                probe_shared_n<B, KT, R>(sfilt + 4u * (uint32_t)off, nb, h, k, pass);
            } else if (off >= 0) {
#pragma unroll
                for (int i = 0; i < R; ++i)
                    pass[i] = live[i] && probe_cluster<B, KT>(sfilt + 4u * (uint32_t)off, lc, nb, h[i], k);
            } else {
                probe_global_live<B, KT, R>(fg, nb, h, k, live, pass);
            }
            const uint32_t last_row = q[cnt - 1];
            __syncwarp();
            if (lane == 0) last_in[s] = last_row;
            qset(s, 0u);
#pragma unroll
            for (int i = 0; i < R; ++i) emit(pass[i] && live[i], r[i]);
        }
        if (!last) qset(s + 1, nn);
        __syncwarp();
    };

    // After stage s ran: later stages whose queue reached kDrain run too.
    auto cascade = [&](int s, uint32_t round_row0) {
        for (int t = s + 1; t < n_in; ++t) {
            if (qget(t) < (uint32_t)kDrain) break;
            run_stage(t, kDrain, round_row0);
        }
    };

    // Input word w (lane-specific), masked to the table's rows; 0 past the chunk.
    auto load_word = [&](int64_t w) -> uint32_t {
        uint32_t x = 0;
        if (w < w_end) {
            x = a.in_bits ? ld_once(a.in_bits + w) : FULL;
            if (w == n_words - 1 && tail_bits) x &= (1u << tail_bits) - 1u;
        }
        return x;
    };
    // Dense sub-rounds (32 words, every row alive) read stage 0's single key
    // column straight from memory: lane l takes rows lane + 32*j, so word j's
    // survivors are one ballot.  The keys of the next 8 words are loaded
    // before the current 8 are hashed, and the first 8 of the next dense
    // sub-round before the current one's last 8, so a warp keeps its key
    // loads in flight.
    const bool dense_ok = DENSE && n_in > 0 && s_pe[0].ncols == 1;
    const ColRef d_col = s_pe[0].col[0];
    auto load8 = [&](uint32_t row0, uint64_t* kv) {
        if (d_col.dtype == 0) {
            const int32_t* p = reinterpret_cast<const int32_t*>(d_col.p) + row0 + lane;
#pragma unroll
            for (int i = 0; i < 8; ++i) kv[i] = (uint64_t)(int64_t)ld_once(p + 32 * i);
        } else {
            const long long* p = reinterpret_cast<const long long*>(d_col.p) + row0 + lane;
#pragma unroll
            for (int i = 0; i < 8; ++i) kv[i] = (uint64_t)ld_once(p + 32 * i);
        }
    };
    uint64_t kn[8];  // prefetched keys (valid when have_pref)
    bool have_pref = false;
    constexpr int NS = kRoundWords / 32;  // sub-rounds of 32 words per round
    const int32_t d00 = n_in > 0 ? s_pe[0].col[0].dtype : 0, d01 = n_in > 0 ? s_pe[0].col[1].dtype : 0;
    const bool two0 = n_in > 0 && s_pe[0].ncols == 2;

    uint32_t win[NS], win_next[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) win[q] = load_word(w_begin + 32 * q + lane);
    for (int64_t rb = w_begin; rb < w_end; rb += kRoundWords) {
        const uint32_t round_row0 = (uint32_t)(rb * 32);
        const int64_t rb_next = rb + kRoundWords;
#pragma unroll
        for (int q = 0; q < NS; ++q) win_next[q] = load_word(rb_next + 32 * q + lane);
        if (n_in == 0) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int64_t wl = rb + 32 * q + lane;
                if (wl < w_end) a.out_bits[wl] = win[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                obm[32 * q + lane] = 0u;
                psec += sectors_of(win[q], d00);  // every input row enters stage 0
                if (two0) psec += sectors_of(win[q], d01);
            }
            __syncwarp();
#pragma unroll 1
            for (int q = 0; q < NS; ++q) {
                const int64_t sb = rb + 32 * q;  // first word of the sub-round
                if (sb >= w_end) break;
                const int nw = (int)min((int64_t)32, w_end - sb);
                uint32_t wq = win[0], wn = win[NS > 1 ? 1 : 0];
#pragma unroll
                for (int t = 1; t < NS; ++t)
                    if (q == t) {
                        wq = win[t];
                        wn = t + 1 < NS ? win[t + 1 < NS ? t + 1 : 0] : win_next[0];
                    }
                if (NS == 1) wn = win_next[0];
                const uint32_t sub_row0 = round_row0 + 1024u * q;
                const bool dense = dense_ok && nw == 32 && __all_sync(FULL, wq == FULL);
                if (dense) {
                    // rows still waiting for stage 0 move on first, so that every
                    // stage keeps receiving its rows in ascending order
                    if (qget(0) > 0) {
                        run_stage(0, qget(0), round_row0);
                        cascade(0, round_row0);
                    }
                    const int32_t off = s_off[0];
                    const uint32_t nb = s_nb[0];
                    const uint32_t* fg = s_pe[0].filter;
                    const bool last = n_in == 1;
                    uint32_t* nbm = obm + 32 * q;
                    if (!have_pref) load8(sub_row0, kn);
                    const bool next_dense = sb + 64 <= w_end && __all_sync(FULL, wn == FULL);
#pragma unroll 1
                    for (int g = 0; g < 32; g += 8) {
                        uint64_t h[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) h[i] = kn[i];
                        if (g + 8 < 32)
                            load8(sub_row0 + 32u * (g + 8), kn);
                        else if (next_dense)
                            load8(sub_row0 + 1024u, kn);
                        if (d_col.dtype != kHashed) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) h[i] = hash_key(h[i], seed);
                        }
                        bool pass[8];
                        if (off >= 0 && !s_split[0]) {
                            probe_shared_n<B, KT, 8>(sfilt + 4u * (uint32_t)off, nb, h, k, pass);
                        } else if (off >= 0) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) pass[i] = probe_cluster<B, KT>(sfilt + 4u * (uint32_t)off, lc, nb, h[i], k);
                        } else {
                            probe_global_n<B, KT, 8>(fg, nb, h, k, pass);
                        }
                        uint32_t mk[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            mk[i] = __ballot_sync(FULL, pass[i]);
                            if (last && lane == 0) nbm[g + i] = mk[i];
                        }
                        if (!last) {
                            // queue the survivors of all 8 words for stage 1 at once (prefix
                            // of the words' popcounts + rank inside the word), then drain it
                            uint32_t q1 = qget(1);
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                if (pass[i]) queue[qoff(1) + q1 + __popc(mk[i] & lt_mask)] = sub_row0 + 32u * (g + i) + lane;
                                q1 += __popc(mk[i]);
                            }
                            qset(1, q1);
                            __syncwarp();
                            while (qget(1) >= (uint32_t)kDrain) {
                                run_stage(1, kDrain, round_row0);
                                cascade(1, round_row0);
                            }
                        }
                    }
                    have_pref = next_dense;
                } else {
                    // Sparse sub-round: every lane appends the rows of its own word
                    // (a warp prefix sum of the popcounts gives each lane its place),
                    // when the queue has room for all of them; else one word at a time.
                    const uint32_t c = __popc(wq);
                    uint32_t incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= (uint32_t)o) incl += t;
                    }
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t q0 = qget(0);
                    if (q0 + total <= (uint32_t)kQueueCap) {
                        uint32_t pos = q0 + incl - c;
                        uint32_t m = wq;
                        const uint32_t row = sub_row0 + 32u * lane;
                        while (m) {
                            queue[pos++] = row + (uint32_t)(__ffs(m) - 1);
                            m &= m - 1u;
                        }
                        qset(0, q0 + total);
                        __syncwarp();
                        while (qget(0) >= (uint32_t)kDrain) {
                            run_stage(0, kDrain, round_row0);
                            cascade(0, round_row0);
                        }
                    } else {
                        uint32_t nz = __ballot_sync(FULL, wq != 0u);
                        while (nz) {
                            const int j = __ffs(nz) - 1;
                            nz &= nz - 1u;
                            const uint32_t m = __shfl_sync(FULL, wq, j);
                            const uint32_t qj = qget(0);
                            if ((m >> lane) & 1u) queue[qj + __popc(m & lt_mask)] = sub_row0 + 32u * j + lane;
                            qset(0, qj + __popc(m));
                            __syncwarp();
                            if (qj + __popc(m) >= (uint32_t)kDrain) {
                                run_stage(0, kDrain, round_row0);
                                cascade(0, round_row0);
                            }
                        }
                    }
                }
            }
            // rows still queued stay queued (their survivors will be set in
            // the output bitmap directly); store the round's survivor words
            __syncwarp();
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int64_t wl = rb + 32 * q + lane;
                if (wl < w_end) a.out_bits[wl] = obm[32 * q + lane];
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) win[q] = win_next[q];
    }
    // the rows still queued go through their remaining stages
    for (int s = 0; s < n_in; ++s) {
        while (qget(s) > 0) {
            run_stage(s, min(qget(s), (uint32_t)kDrain), kNoRow);
            cascade(s, kNoRow);
        }
    }
    __syncwarp();

    // Compaction of the chunk's survivors from its finished output words
    // (read past L1: some bits were set by atomics): lane l takes word l of
    // each group of 32, a warp prefix sum of the popcounts places its rows.
    uint32_t local = 0;  // per lane; reduced below
    unsigned long long bsec = 0;
    int64_t seg_pos = w_begin * 32;  // next free slot of this warp's id segment
    constexpr int CB = 8;  // groups of 32 words loaded at once (independent loads in flight)
    for (int64_t g0 = w_begin; g0 < w_end; g0 += 32 * CB) {
        uint32_t owb[CB];
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            const int64_t wl = g0 + 32 * j + lane;
            owb[j] = wl < w_end ? __ldcg(a.out_bits + wl) : 0u;
        }
#pragma unroll 1
        for (int j = 0; j < CB; ++j) {
        const int64_t g = g0 + 32 * j;
        if (g >= w_end) break;
        const int64_t wl = g + lane;
        const uint32_t ow = owb[j];
        const uint32_t c = __popc(ow);
        local += c;
        if (a.ids) {
            for (int b = 0; b < a.n_bcols; ++b) bsec += sectors_of(ow, a.bcol[b].dtype);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            uint32_t* dst = a.ids + seg_pos + (incl - c);
            const uint32_t row = (uint32_t)(wl * 32);
            uint32_t m = ow;
            while (m) {
                *dst++ = row + (uint32_t)(__ffs(m) - 1);
                m &= m - 1u;
            }
            seg_pos += __shfl_sync(FULL, incl, 31);
        }
        }
    }

    allow_dependents();  // the next kernel on the stream may launch; it waits for this grid's end
    local = __reduce_add_sync(FULL, local);
    psec = __reduce_add_sync(FULL, (unsigned)psec);
    bsec = __reduce_add_sync(FULL, (unsigned)bsec);
    if (lane == 0) {
        if (a.seg_count && gw < a.total_warps) a.seg_count[gw] = local;
        warp_to_cta(&sh.sum[0], local);
        warp_to_cta(&sh.sum[1], psec);
        warp_to_cta(&sh.sum[2], bsec);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cta_to_global(&sh.sum[0], a.count);
        cta_to_global(&sh.sum[1], a.stats + 0);
        cta_to_global(&sh.sum[2], a.stats + 1);
    }
    // no CTA of a cluster leaves (or reuses its shared memory) while another may still read its part
    if (C > 1) cooperative_groups::this_cluster().sync();
}

template <int B, int KT>
__global__ void __launch_bounds__(kScanMaxThreads, kScanMinBlocks) pt_scan_kernel(const VisitArgs a, const FilterCfg f) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ ScanShared sh;
    grid_dependency_wait();
    scan_cta<B, KT, true>(a, f, blockIdx.x, a.cluster > 1 ? cluster_rank() : 0u, smem, sh);
}

// The scan of a visit with an input bitmap (selection, backward pass, or the
// survivors of a first-probe pass): no dense path, three CTAs per SM.
template <int B, int KT>
__global__ void __launch_bounds__(kScanMaxThreads, kScanSparseMinBlocks)
    pt_scan_sparse_kernel(const VisitArgs a, const FilterCfg f) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ ScanShared sh;
    grid_dependency_wait();
    scan_cta<B, KT, false>(a, f, blockIdx.x, a.cluster > 1 ? cluster_rank() : 0u, smem, sh);
}

// Copy a visit's arguments from global memory into shared memory (all threads).
__device__ __forceinline__ void load_visit(VisitArgs& dst, const VisitArgs* src) {
    static_assert(sizeof(VisitArgs) % 8 == 0, "VisitArgs is copied in 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (unsigned i = threadIdx.x; i < sizeof(VisitArgs) / 8; i += blockDim.x) d[i] = s[i];
}

// Batched scan: one launch runs the scans of many visits (of many queries);
// task t is CTA tasks[t].part of visit tasks[t].visit.  Tasks of one launch
// must not depend on each other.
template <int B, int KT>
__global__ void __launch_bounds__(kScanMaxThreads, kScanMinBlocks)
    pt_scan_batch_kernel(const VisitArgs* visits, const BatchTask* task_base, const int32_t* range, const FilterCfg f) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ ScanShared sh;
    __shared__ __align__(16) VisitArgs s_a;
    const BatchTask* tasks = task_base + range[0];
    const int32_t n = range[1];
    // tasks are per cluster (the CTAs of a cluster share the task's filters);
    // without clusters a cluster is one CTA
    uint32_t C = 1, rank = 0;
    {
        const unsigned int cs = cooperative_groups::this_cluster().num_blocks();
        if (cs > 1) {
            C = cs;
            rank = cluster_rank();
        }
    }
    for (int32_t t = blockIdx.x / C; t < n; t += gridDim.x / C) {
        const BatchTask task = tasks[t];
        load_visit(s_a, visits + task.visit);
        __syncthreads();
        scan_cta<B, KT, true>(s_a, f, (int64_t)task.part * C + rank, rank, smem, sh);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 1a. first probe of a visit that starts with every row alive
//
// A visit with no input bitmap (a forward-pass visit of a table without a
// local predicate) tests its first filter in probe order on every row, so
// that stage is a plain stream over the edge's key column(s): no queue and
// no compaction.  This kernel runs that stage alone with a small register
// footprint -- four 256-thread CTAs per SM instead of the scan kernel's two
// -- so that twice the warps cover the key loads and the filter reads.  It
// writes the rows that pass as a bitmap; the scan kernel then runs the
// remaining probes with that bitmap as its input (the probe order, and so
// the sector accounting, is the same as in one kernel).
//
// Warp w takes tiles of 256 rows (8 bitmap words) w, w + W, w + 2W, ...
// (W warps in the grid); lane l holds rows l + 32 i (i < 8) of a tile, so a
// key load of the warp is one coalesced access of 32 rows and the tile's 8
// survivor words are 8 ballots.  The keys of the warp's next tile are
// loaded before the current tile is hashed.
// ---------------------------------------------------------------------------
struct FirstShared {
    ProbeEdge pe;
    uint32_t nb;
    int32_t fit, run;
    unsigned long long sum;  // the CTA's key sectors (see warp_to_cta)
};

// CTA `cta` of the n_ctas a visit's first probe is split into (every thread of
// the block calls it; it returns at once when the gate says the other launch of
// a pair has the filter).
template <int B, int KT>
__device__ __forceinline__ void probe_first_cta(const VisitArgs& a, const FilterCfg& f, uint32_t* __restrict__ mid,
                                                int32_t* first, const int32_t smem_words, const int32_t gate_words,
                                                const int32_t gate, const int64_t cta, const int64_t n_ctas,
                                                uint32_t* smem, FirstShared& fs) {
    ProbeEdge& s_pe = fs.pe;
    uint32_t& s_nb = fs.nb;
    int32_t& s_fit = fs.fit;
    int32_t& s_run = fs.run;
    constexpr uint32_t WPB = B / 32;
    constexpr int R = kFirstTileRows / 32;  // rows per lane of a tile
    const uint32_t FULL = 0xFFFFFFFFu;
    if (threadIdx.x == 0) {
        int ord[kMaxIn];
        uint32_t nbs[kMaxIn];
        lip_order(a, -1, f.probe_order, ord, nbs);
        s_pe = a.in[ord[0]];
        s_nb = nbs[ord[0]];
        s_fit = (int64_t)s_nb * WPB <= (int64_t)smem_words;
        // gate 1: run only if the filter fits gate_words; 2: only if it does not
        const bool fits = (int64_t)s_nb * WPB <= (int64_t)gate_words;
        s_run = gate == 0 || (gate == 1) == fits;
        if (cta == 0 && s_run) *first = ord[0];
        fs.sum = 0;
    }
    __syncthreads();
    if (!s_run) return;  // the other launch of the pair has this filter
    const uint32_t nb = s_nb;
    const bool in_smem = s_fit != 0;
    if (in_smem) {
        const uint4* src = reinterpret_cast<const uint4*>(s_pe.filter);
        uint4* dst = reinterpret_cast<uint4*>(smem);
        copy_to_smem(dst, src, nb * (WPB / 4));
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const int64_t n = a.n;
    const int64_t n_words = (n + 31) >> 5;
    const int64_t n_tiles = (n + kFirstTileRows - 1) / kFirstTileRows;
    const int64_t n_full = n / kFirstTileRows;  // tiles with every row inside the table
    const int64_t W = n_ctas * (blockDim.x >> 5);
    const int64_t gw = cta * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const ColRef c0 = s_pe.col[0], c1 = s_pe.col[1];
    const int ncols = s_pe.ncols;
    const uint32_t* fg = s_pe.filter;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int k = f.k;
    const uint64_t seed = f.seed;

    // the R rows of a lane, with the filter's location branched on once
    auto probe = [&](const uint64_t* h, bool* pass) {
        if (in_smem)
            probe_shared_n<B, KT, R>(sbase, nb, h, k, pass);
        else
            probe_global_n<B, KT, R>(fg, nb, h, k, pass);
    };
    // the tile's survivor words: word i is ballot i; lanes 0..7 store one each
    // (every lane holds all 8 ballots; lane 0 stores them as two 16-byte
    // writes: the tile's words start 32-byte aligned, and the bitmap's
    // allocation covers whole tiles, so the last tile's words past the table
    // land in its padding, which no reader looks at)
    static_assert(R == 8, "a tile is 8 bitmap words");
    auto store = [&](int64_t t, const bool* pass) {
        uint32_t m[R];
#pragma unroll
        for (int i = 0; i < R; ++i) m[i] = __ballot_sync(FULL, pass[i]);
        if (lane == 0) {
            uint4* dst = reinterpret_cast<uint4*>(mid + t * R);
            dst[0] = make_uint4(m[0], m[1], m[2], m[3]);
            dst[1] = make_uint4(m[4], m[5], m[6], m[7]);
        }
    };

    if (ncols == 1 && c0.dtype != 0) {
        // one 64-bit column (int64 keys, or precomputed hashes): keys prefetched a tile ahead
        const long long* col = reinterpret_cast<const long long*>(c0.p);
        const bool hashed = c0.dtype == kHashed;
        auto load = [&](int64_t t, uint64_t* kv) {
            const int64_t r0 = t * kFirstTileRows + lane;
            if (t < n_full) {
#pragma unroll
                for (int i = 0; i < R; ++i) kv[i] = (uint64_t)ld_once(col + r0 + 32 * i);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) kv[i] = r0 + 32 * i < n ? (uint64_t)ld_once(col + r0 + 32 * i) : 0ull;
            }
        };
        uint64_t kv[R];
        if (gw < n_tiles) load(gw, kv);
        for (int64_t t = gw; t < n_tiles; t += W) {
            uint64_t h[R];
#pragma unroll
            for (int i = 0; i < R; ++i) h[i] = kv[i];
            if (t + W < n_tiles) load(t + W, kv);
            if (!hashed) {
                if (seed == 0) {  // x ^ 0 = x: two integer-ALU operations per key fewer
#pragma unroll
                    for (int i = 0; i < R; ++i) h[i] = mix64(h[i] + kGamma);
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) h[i] = hash_key(h[i], seed);
                }
            }
            bool pass[R];
            probe(h, pass);
            if (t >= n_full) {  // the ragged last tile: rows past the table do not pass
                const int64_t r0 = t * kFirstTileRows + lane;
#pragma unroll
                for (int i = 0; i < R; ++i) pass[i] = pass[i] && r0 + 32 * i < n;
            }
            store(t, pass);
        }
    } else {
        // int32 keys or a composite key: no prefetch
        for (int64_t t = gw; t < n_tiles; t += W) {
            const int64_t r0 = t * kFirstTileRows + lane;
            uint64_t h[R];
            bool live[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                live[i] = r0 + 32 * i < n;
                h[i] = live[i] ? edge_hash(c0, c1, ncols, (uint32_t)(r0 + 32 * i), seed) : 0ull;
            }
            bool pass[R];
            probe(h, pass);
#pragma unroll
            for (int i = 0; i < R; ++i) pass[i] = pass[i] && live[i];
            store(t, pass);
        }
    }

    // key sectors this stage read: every sector of the edge's column(s)
    unsigned long long psec = 0;
    for (int64_t w = cta * blockDim.x + threadIdx.x; w < n_words; w += n_ctas * blockDim.x) {
        const uint32_t tail = (uint32_t)(n & 31);
        const uint32_t alive = (w == n_words - 1 && tail) ? (1u << tail) - 1u : FULL;
        psec += sectors_of(alive, c0.dtype);
        if (ncols == 2) psec += sectors_of(alive, c1.dtype);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) psec += __shfl_xor_sync(FULL, psec, o);
    if (lane == 0) warp_to_cta(&fs.sum, psec);
    __syncthreads();
    if (threadIdx.x == 0 && fs.sum) {
        atomicAdd(a.stats + 0, fs.sum);
        atomicAdd(a.stats + 2, fs.sum);
        fs.sum = 0;
    }
}

template <int B, int KT>
__global__ void __launch_bounds__(kFirstThreads, kFirstMinBlocks)
    pt_probe_first_kernel(const VisitArgs a, const FilterCfg f, uint32_t* __restrict__ mid, int32_t* first,
                          const int32_t smem_words, const int32_t gate_words, const int32_t gate) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FirstShared fs;
    probe_first_cta<B, KT>(a, f, mid, first, smem_words, gate_words, gate, blockIdx.x, gridDim.x, smem, fs);
}

// Batched first probes: task t is part tasks[t].part of the first_parts(n)
// parts of visit tasks[t].visit's first probe.  The visit's in_bits is the
// bitmap the probe writes and first_in the slot of the edge it takes (the
// visit's scan then reads them as its input); its rows all start alive.
template <int B, int KT>
__global__ void __launch_bounds__(kFirstThreads, kFirstMinBlocks)
    pt_probe_first_batch_kernel(const VisitArgs* visits, const BatchTask* task_base, const int32_t* range,
                                const FilterCfg f, const int32_t smem_words, const int32_t gate_words,
                                const int32_t gate) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FirstShared fs;
    __shared__ __align__(16) VisitArgs s_a;
    const BatchTask* tasks = task_base + range[0];
    const int32_t n = range[1];
    for (int32_t t = blockIdx.x; t < n; t += gridDim.x) {
        const BatchTask task = tasks[t];
        load_visit(s_a, visits + task.visit);
        __syncthreads();
        probe_first_cta<B, KT>(s_a, f, const_cast<uint32_t*>(s_a.in_bits), const_cast<int32_t*>(s_a.first_in),
                               smem_words, gate_words, gate, task.part, first_parts(s_a.n), smem, fs);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 1b. a backward visit over the forward pass's compacted survivors
//
// The backward pass reverses every edge and starts each table from what
// survived its forward visit (Section 3.2, "Transfer Schedule").  So the
// filters a table probes in the backward pass are on exactly the edges it
// built in the forward pass, and the forward insert stored, beside each
// survivor's row id, the hash of its key on each of those edges (a one-way
// edge, which builds in one pass only, is the exception: its keys are
// gathered and hashed here).  This kernel therefore reads no input bitmap,
// and no key column for the other edges: warp w walks
// forward segment s = w, w + W, ... -- row ids and hashes in coalesced 4-
// and 8-byte loads, kListRows per lane at a time -- probes the incoming
// filters in probe order (shared memory when they fit, else L1/L2), and
// writes the survivors' ids into backward segment s (same geometry).  The
// rows of segment s are the bitmap words of segment s, which only this
// warp touches: it zero-fills them, then ORs in its survivors, one atomicOr
// per word run of 32 listed rows.
//
// Sector accounting equals a scan's: listed rows are in ascending order, so
// a stage's sectors are the rows alive at that stage whose sector differs
// from the previous such row's (segments hold whole sectors).
// ---------------------------------------------------------------------------
namespace {
// Sectors of this group of 32 ascending rows: each live row whose sector
// (row >> sh0, and row >> sh1 for a second column) differs from that of the
// previous live row -- in this group, else `last` -- counts.  Returns the
// last live row (every lane calls it).
__device__ __forceinline__ uint32_t group_sectors(bool live, uint32_t r, uint32_t sh0, uint32_t sh1, int ncols,
                                                  uint32_t last, unsigned long long& cnt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, live);
    const uint32_t below = m & ((1u << lane) - 1u);
    const uint32_t pr = __shfl_sync(0xFFFFFFFFu, r, below ? 31 - __clz(below) : 0);
    const uint32_t prev = below ? pr : last;
    if (live) {
        cnt += (r >> sh0) != (prev >> sh0);
        if (ncols == 2) cnt += (r >> sh1) != (prev >> sh1);
    }
    const uint32_t top = __shfl_sync(0xFFFFFFFFu, r, m ? 31 - __clz(m) : 0);
    return m ? top : last;
}
__device__ __forceinline__ uint32_t sector_shift(int32_t dtype) { return dtype == 0 ? 3u : 2u; }
}  // namespace

template <int B, int KT>
__global__ void __launch_bounds__(kListThreads, kListMinBlocks)
    pt_probe_list_kernel(const VisitArgs a, const FilterCfg f) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ ScanShared sh;
    __shared__ uint32_t s_last[kListThreads / 32][kMaxIn + 1];  // per warp: last row of each stage; [kMaxIn]: survivors
    grid_dependency_wait();
    constexpr uint32_t WPB = B / 32;
    constexpr int R = kListRows;
    const uint32_t FULL = 0xFFFFFFFFu;
    constexpr uint32_t kNoRow = 0xFFFFFFFFu;  // rows are below 2^31

    clear_previous_filters(a, B, blockIdx.x, gridDim.x);
    if (threadIdx.x == 0) {
        int ord[kMaxIn];
        uint32_t nbs[kMaxIn];
        const int m = lip_order(a, -1, f.probe_order, ord, nbs);
        sh.n_in = m;
        sh.sum[0] = sh.sum[1] = sh.sum[2] = 0;
        int32_t used = 0;
        for (int i = 0; i < m; ++i) {
            sh.pe[i] = a.in[ord[i]];
            const uint32_t nb = nbs[ord[i]];
            sh.nb[i] = nb;
            sh.split[i] = 0;
            const int64_t words = (int64_t)nb * WPB;
            if (used + words <= a.smem_words) {
                sh.off[i] = used;
                used += (int32_t)words;
            } else {
                sh.off[i] = -1;
            }
        }
    }
    __syncthreads();
    const int n_in = sh.n_in;
    for (int i = 0; i < n_in; ++i)
        if (sh.off[i] >= 0)
            copy_to_smem(reinterpret_cast<uint4*>(smem + sh.off[i]), reinterpret_cast<const uint4*>(sh.pe[i].filter),
                         sh.nb[i] * (WPB / 4));
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t* last = s_last[warp];
    const uint32_t sfilt = (uint32_t)__cvta_generic_to_shared(smem);
    const int64_t n_words = (a.n + 31) >> 5;
    const size_t seg_rows = (size_t)a.words_per_warp * 32;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int k = f.k;
    unsigned long long psec = 0, bsec = 0;  // per lane; reduced at the end
    uint32_t total = 0;                     // warp-uniform

    for (int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; seg < a.total_warps; seg += W) {
        // the segment's output words: zero, then OR in the survivors below
        const int64_t w0 = seg * a.words_per_warp, w1 = min(n_words, w0 + a.words_per_warp);
        for (int64_t w = w0 + lane; w < w1; w += 32) a.out_bits[w] = 0u;
        if (lane <= (uint32_t)kMaxIn) last[lane] = kNoRow;
        __syncwarp();
        const uint32_t cnt = a.list_seg[seg];
        const size_t slot0 = (size_t)seg * seg_rows;
        const uint32_t* ids = a.list_ids + slot0;
        uint32_t ocnt = 0;  // warp-uniform
        for (uint32_t b = 0; b < cnt; b += 32u * R) {
            uint32_t r[R];
            bool live[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint32_t idx = b + lane + 32u * i;
                live[i] = idx < cnt;
                r[i] = live[i] ? ld_once(ids + idx) : kNoRow;
            }
            for (int s = 0; s < n_in; ++s) {
                const ProbeEdge& pe = sh.pe[s];
                uint64_t h[R];
                if (pe.hin) {  // the hashes the forward insert stored
                    const unsigned long long* hin = reinterpret_cast<const unsigned long long*>(pe.hin) + slot0;
#pragma unroll
                    for (int i = 0; i < R; ++i) h[i] = live[i] ? ld_once(hin + b + lane + 32u * i) : 0ull;
                } else {       // an edge the forward pass did not build on (one-way): gather and hash
#pragma unroll
                    for (int i = 0; i < R; ++i) h[i] = live[i] ? edge_hash(pe.col[0], pe.col[1], pe.ncols, r[i], f.seed) : 0ull;
                }
                // key sectors of the rows that reach this stage
                const uint32_t sh0 = sector_shift(pe.col[0].dtype), sh1 = sector_shift(pe.col[1].dtype);
                uint32_t lr = last[s];
#pragma unroll
                for (int i = 0; i < R; ++i) lr = group_sectors(live[i], r[i], sh0, sh1, pe.ncols, lr, psec);
                __syncwarp();
                if (lane == 0) last[s] = lr;
                bool pass[R];
                if (sh.off[s] >= 0) {
                    probe_shared_n<B, KT, R>(sfilt + 4u * (uint32_t)sh.off[s], sh.nb[s], h, k, pass);
                } else {
                    probe_global_live<B, KT, R>(pe.filter, sh.nb[s], h, k, live, pass);
                }
#pragma unroll
                for (int i = 0; i < R; ++i) live[i] = live[i] && pass[i];
            }
            // survivors: ids into the backward segment, bits into the bitmap,
            // build-column sectors
            uint32_t lb = last[kMaxIn];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const uint32_t m = __ballot_sync(FULL, live[i]);
                if (m == 0) continue;  // (warp-uniform) no survivor in this group of 32: nothing to write
                if (a.ids && live[i]) a.ids[slot0 + ocnt + __popc(m & lt_mask)] = r[i];
                ocnt += __popc(m);
                // word runs: rows ascend across lanes, so equal words are adjacent
                const uint32_t wd = r[i] >> 5;
                uint32_t val = live[i] ? 1u << (r[i] & 31) : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v2 = __shfl_down_sync(FULL, val, o);
                    const uint32_t w2 = __shfl_down_sync(FULL, wd, o);
                    if (lane + o < 32 && w2 == wd) val |= v2;
                }
                const uint32_t wprev = __shfl_up_sync(FULL, wd, 1);
                if ((lane == 0 || wprev != wd) && val) atomicOr(a.out_bits + wd, val);
                // build sectors: one count per distinct build column
                const uint32_t below = m & lt_mask;
                const uint32_t pr = __shfl_sync(FULL, r[i], below ? 31 - __clz(below) : 0);
                const uint32_t prev = below ? pr : lb;
                if (live[i])
                    for (int c = 0; c < a.n_bcols; ++c) {
                        const uint32_t shc = sector_shift(a.bcol[c].dtype);
                        bsec += (r[i] >> shc) != (prev >> shc);
                    }
                const uint32_t top = __shfl_sync(FULL, r[i], m ? 31 - __clz(m) : 0);
                if (m) lb = top;
            }
            __syncwarp();
            if (lane == 0) last[kMaxIn] = lb;
            __syncwarp();
        }
        if (lane == 0 && a.seg_count) a.seg_count[seg] = ocnt;
        total += ocnt;
    }
    allow_dependents();  // the next kernel on the stream may launch; it waits for this grid's end
    psec = __reduce_add_sync(FULL, (unsigned)psec);
    bsec = __reduce_add_sync(FULL, (unsigned)bsec);
    if (lane == 0) {
        warp_to_cta(&sh.sum[0], total);
        warp_to_cta(&sh.sum[1], psec);
        warp_to_cta(&sh.sum[2], bsec);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cta_to_global(&sh.sum[0], a.count);
        cta_to_global(&sh.sum[1], a.stats + 0);
        cta_to_global(&sh.sum[2], a.stats + 1);
    }
}

// ---------------------------------------------------------------------------
// 2. size + clear the outgoing filters from the device-side survivor count
// ---------------------------------------------------------------------------
// The size rule: max(1, ceil(min(c, n_probe) * bits_per_key / block_bits)).
__device__ __forceinline__ int64_t filter_blocks(unsigned long long c, int64_t n_probe, const FilterCfg& f) {
    const int64_t n_est = min((int64_t)c, n_probe);
    const int64_t nb = (n_est * f.bits_per_key + f.block_bits - 1) / f.block_bits;
    return nb < 1 ? 1 : nb;
}

// Part `part` of `nparts` of a visit's size/clear (thread t of the part zeroes
// every (nparts * blockDim)-th 16-byte chunk from (part * blockDim + t)).
__device__ __forceinline__ void size_clear_part(const VisitArgs& a, const FilterCfg& f, int64_t part, int64_t nparts) {
    const unsigned long long c = *a.count;
    const size_t tid = (size_t)part * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)nparts * blockDim.x;
#pragma unroll
    for (int e = 0; e < kMaxOut; ++e) {
        if (e >= a.n_out) break;
        const int64_t nb = filter_blocks(c, a.out[e].probe_rows, f);
        if (tid == 0) *a.out[e].nblocks = nb;
        uint4* p = reinterpret_cast<uint4*>(a.out[e].filter);
        const size_t n16 = (size_t)nb * (size_t)(f.block_bits / 128);
        for (size_t i = tid; i < n16; i += stride) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void __launch_bounds__(512) pt_size_clear_kernel(const VisitArgs a, const FilterCfg f) {
    size_clear_part(a, f, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(512)
    pt_size_clear_batch_kernel(const VisitArgs* visits, const BatchTask* task_base, const int32_t* range,
                               const int32_t parts, const FilterCfg f) {
    __shared__ __align__(16) VisitArgs s_a;
    const BatchTask* tasks = task_base + range[0];
    const int32_t n = range[1];
    for (int32_t t = blockIdx.x; t < n; t += gridDim.x) {
        const BatchTask task = tasks[t];
        load_visit(s_a, visits + task.visit);
        __syncthreads();
        size_clear_part(s_a, f, task.part, parts);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 3. insert the survivors' outgoing keys
// ---------------------------------------------------------------------------
// A filter of at most kTinyWords words that more rows build than its probe
// side has is built in each CTA's shared memory and then ORed into the global
// one word by word: many rows inserting into a few blocks (a foreign key into
// a tiny table, whose probe side caps the filter's size) otherwise pile
// thousands of atomics onto one L2 line, which serialises them (measured: D1's
// backward insert into N's 2-block filter, 7373 rows, took 11 us more than its
// CTAs ran).  A few rows into a small filter go straight to it.
constexpr int kTinyWords = 128;
struct InsertShared {
    uint32_t nb[kMaxOut];    // this run's filter sizes
    unsigned long long sum;  // the CTA's build sectors (with a.insert_bsec; see warp_to_cta)
    uint32_t tiny[kMaxOut][kTinyWords];  // the CTA's part of each tiny filter
    uint32_t repeat[kMaxOut];  // 1: more rows build the filter than the probe side has (see below)
};

// Part `part` of `nparts` of a visit's insert: warp w of the part takes the
// segments s = part * warps + w, then every (nparts * warps)-th one.
template <int B, int KT>
__device__ __forceinline__ void insert_part(const VisitArgs& a, const FilterCfg& f, int64_t part, int64_t nparts,
                                            InsertShared& ish) {
    using BB = BlockBits<B>;
    uint32_t* s_nb = ish.nb;
    if (threadIdx.x == 0) ish.sum = 0;
#pragma unroll
    for (int e = 0; e < kMaxOut; ++e)
        if (threadIdx.x == (unsigned)e && e < a.n_out) {
            ish.repeat[e] = (int64_t)*a.count > a.out[e].probe_rows;
            if (a.insert_sizes) {
                // the scan zeroed the previous run's words; this run's size, from the count
                // (the size rule with the block size known here: a shift, not a division)
                const int64_t n_est = min((int64_t)*a.count, a.out[e].probe_rows);
                const int64_t nb = max((int64_t)1, (n_est * f.bits_per_key + B - 1) / B);
                s_nb[e] = (uint32_t)nb;
                if (part == 0) *a.out[e].nblocks = nb;
            } else {
                s_nb[e] = (uint32_t)*a.out[e].nblocks;
            }
        }
    __syncthreads();
    // tiny filters: this CTA's shared copies start empty
    bool any_tiny = false;
    auto tiny_edge = [&](int e) { return ish.repeat[e] != 0 && s_nb[e] * BB::WPB <= (uint32_t)kTinyWords; };
    for (int e = 0; e < a.n_out; ++e) any_tiny |= tiny_edge(e);
    if (any_tiny) {
        for (int e = 0; e < a.n_out; ++e)
            if (tiny_edge(e))
                for (uint32_t w = threadIdx.x; w < s_nb[e] * BB::WPB; w += blockDim.x) ish.tiny[e][w] = 0u;
        __syncthreads();
    }

    const uint32_t lane = threadIdx.x & 31;
    const int64_t gw = part * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t n_warps = nparts * (blockDim.x >> 5);
    const size_t seg_rows = (size_t)a.words_per_warp * 32;
    const int k = f.k;
    const uint64_t seed = f.seed;
    // with more warps than segments, the ways-th part of every segment's
    // batches goes to a different warp (more gathers in flight)
    const int64_t ways = max((int64_t)1, n_warps / a.total_warps);
    unsigned long long bsec = 0;  // per lane (with a.insert_bsec)

    for (int64_t t = gw; t < a.total_warps * ways; t += n_warps) {
        const int64_t s = t % a.total_warps;
        const uint32_t cnt = a.seg_count[s];
        const uint32_t* ids = a.ids + (size_t)s * seg_rows;
        // four survivors per lane at a time: four independent key gathers in flight
        for (uint32_t base = 128u * (uint32_t)(t / a.total_warps); base < cnt; base += 128u * (uint32_t)ways) {
            uint32_t r[4], live_mask[4];
            bool live[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t idx = base + lane + 32u * i;
                live[i] = idx < cnt;
                live_mask[i] = __ballot_sync(0xFFFFFFFFu, live[i]);
                r[i] = live[i] ? ld_once(ids + idx) : 0u;
            }
            if (a.insert_bsec) {
                // build sectors holding a survivor: rows ascend with the slot (i, then
                // lane), so a row counts when its sector differs from the previous
                // slot's row's -- the slot before `base` is ids[base - 1], or none at
                // the segment's start (segments hold whole sectors)
                const uint32_t before = base > 0 ? ld_once(ids + base - 1) : 0xFFFFFFFFu;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, r[i], 1);
                    const uint32_t wrap = __shfl_sync(0xFFFFFFFFu, r[i > 0 ? i - 1 : 0], 31);
                    const uint32_t prev = lane > 0 ? up : (i > 0 ? wrap : before);
                    if (live[i])
                        for (int c = 0; c < a.n_bcols; ++c) {
                            const uint32_t shc = a.bcol[c].dtype == 0 ? 3u : 2u;
                            bsec += (r[i] >> shc) != (prev >> shc);
                        }
                }
            }
#pragma unroll
            for (int e = 0; e < kMaxOut; ++e) {
                if (e >= a.n_out) break;
                const BuildEdge& be = a.out[e];
                const bool dedup = a.n > be.probe_rows;
                const bool tiny = tiny_edge(e);  // (warp-uniform)
                const bool repeat = ish.repeat[e] != 0;
                uint64_t h[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) h[i] = live[i] ? edge_hash(be.col[0], be.col[1], be.ncols, r[i], seed) : 0ull;
                if (be.hout) {
                    // kept for the backward pass, which probes this edge with the same key
                    unsigned long long* ho = reinterpret_cast<unsigned long long*>(be.hout) + (size_t)s * seg_rows;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (live[i]) ho[base + lane + 32u * i] = h[i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!live[i]) continue;
                    // lanes holding the same hash set the same bits: only the lowest one
                    // does.  Keys repeat when the building table has more rows than the
                    // other end (foreign keys, skewed ones piling atomics on a few words);
                    // the smaller side's keys are mostly distinct, and the match would
                    // only cost time
                    if (dedup) {
                        const uint32_t peers = __match_any_sync(live_mask[i], h[i]);
                        if (lane != (uint32_t)(__ffs(peers) - 1)) continue;
                    }
                    const uint32_t lo = (uint32_t)h[i];
                    const uint32_t bi = mul_hi((uint32_t)(h[i] >> 32), s_nb[e]);
                    const uint32_t h2 = (lo >> 16) | 1u;
                    if (tiny) {
                        // the CTA's shared copy (merged into the filter at the end)
                        const uint32_t sblk = (uint32_t)__cvta_generic_to_shared(ish.tiny[e]) + 4u * bi * BB::WPB;
                        for (int t = 0; t < k; ++t) {
                            const uint32_t at = mad_lo((uint32_t)t, h2, lo);
                            red_or_shared(sblk + 4u * mul_hi(mad_lo(at, BB::SCALE, 0u), BB::WPB), 1u << (at & 31));
                        }
                        continue;
                    }
                    uint32_t* blk = be.filter + (size_t)bi * BB::WPB;
                    if (KT > 0) {
                        // bits that share a word go out in one atomicOr
                        uint32_t w[KT > 0 ? KT : 1], m[KT > 0 ? KT : 1];
#pragma unroll
                        for (int t = 0; t < KT; ++t) {
                            const uint32_t at = mad_lo((uint32_t)t, h2, lo);
                            w[t] = mul_hi(mad_lo(at, BB::SCALE, 0u), BB::WPB);
                            m[t] = 1u << (at & 31);
                        }
#pragma unroll
                        for (int t = 1; t < KT; ++t)
#pragma unroll
                            for (int u = 0; u < t; ++u)
                                if (m[t] && w[t] == w[u] && m[u]) {
                                    m[u] |= m[t];
                                    m[t] = 0;
                                }
                        if (repeat) {
                            // more rows than the probe side has, so keys repeat, and a skewed
                            // one many times: a repeated key usually finds its bits set
                            // already, so read its words (from L2, where the atomics land) and
                            // skip the atomics that would change nothing, so that a hot key's
                            // block is not hit by one atomic per row (with fewer rows the
                            // extra read only adds latency: 18 -> 20 us on a 20k-row build)
                            uint32_t cur[KT > 0 ? KT : 1];
#pragma unroll
                            for (int t = 0; t < KT; ++t) cur[t] = m[t] ? __ldcg(blk + w[t]) : 0u;
#pragma unroll
                            for (int t = 0; t < KT; ++t)
                                if (m[t] & ~cur[t]) atomicOr(blk + w[t], m[t] & ~cur[t]);
                        } else {
#pragma unroll
                            for (int t = 0; t < KT; ++t)
                                if (m[t]) atomicOr(blk + w[t], m[t]);
                        }
                    } else {
                        for (int t = 0; t < k; ++t) {
                            const uint32_t at = mad_lo((uint32_t)t, h2, lo);
                            uint32_t* wp = blk + mul_hi(mad_lo(at, BB::SCALE, 0u), BB::WPB);
                            const uint32_t bit = 1u << (at & 31);
                            if (!repeat || !(__ldcg(wp) & bit)) atomicOr(wp, bit);
                        }
                    }
                }
            }
        }
    }
    if (any_tiny) {
        // the CTA's parts of tiny filters, one atomic per word that has a bit set
        __syncthreads();
        for (int e = 0; e < a.n_out; ++e) {
            const uint32_t words = s_nb[e] * BB::WPB;
            if (!tiny_edge(e)) continue;
            for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
                const uint32_t v = ish.tiny[e][w];
                if (v) atomicOr(a.out[e].filter + w, v);
            }
        }
    }
    if (a.insert_bsec) {  // (the same for every thread of the CTA)
        bsec = __reduce_add_sync(0xFFFFFFFFu, (unsigned)bsec);
        if (lane == 0) warp_to_cta(&ish.sum, bsec);
        __syncthreads();
        if (threadIdx.x == 0) cta_to_global(&ish.sum, a.stats + 1);
    }
}

// A backward visit that probes nothing (a source of the reversed DAG) keeps
// its forward survivors, so no scan runs for it: this kernel does the two
// things such a scan would have done for its builds -- zero its filters' words
// of the previous run, and count the build columns' sectors holding a
// survivor, from the survivor words.
__global__ void __launch_bounds__(512) pt_pass_through_kernel(const VisitArgs a, const FilterCfg f) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    grid_dependency_wait();
    clear_previous_filters(a, f.block_bits, blockIdx.x, gridDim.x);
    // the survivor words in 16-byte loads, four of them in flight per thread (the
    // bitmap's allocation is 16-byte aligned; words past the table are zero)
    const int64_t n_words = (a.n + 31) >> 5, n16 = (n_words + 3) >> 2;
    const uint4* w4 = reinterpret_cast<const uint4*>(a.out_bits);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long bsec = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = i + u * stride < n16 ? __ldcs(w4 + i + u * stride) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t w0 = (i + u * stride) * 4;
            const uint32_t m[4] = {v[u].x, w0 + 1 < n_words ? v[u].y : 0u, w0 + 2 < n_words ? v[u].z : 0u,
                                   w0 + 3 < n_words ? v[u].w : 0u};
            for (int c = 0; c < a.n_bcols; ++c)
#pragma unroll
                for (int j = 0; j < 4; ++j) bsec += sectors_of(m[j], a.bcol[c].dtype);
        }
    }
    allow_dependents();
    bsec = __reduce_add_sync(0xFFFFFFFFu, (unsigned)bsec);
    if ((threadIdx.x & 31) == 0) warp_to_cta(&s_sum, bsec);
    __syncthreads();
    if (threadIdx.x == 0) cta_to_global(&s_sum, a.stats + 1);
}

template <int B, int KT>
__global__ void __launch_bounds__(512) pt_insert_kernel(const VisitArgs a, const FilterCfg f) {
    __shared__ InsertShared ish;
    grid_dependency_wait();
    insert_part<B, KT>(a, f, blockIdx.x, gridDim.x, ish);
    allow_dependents();
}

template <int B, int KT>
__global__ void __launch_bounds__(512)
    pt_insert_batch_kernel(const VisitArgs* visits, const BatchTask* task_base, const int32_t* range,
                           const int32_t parts, const FilterCfg f) {
    __shared__ InsertShared ish;
    __shared__ __align__(16) VisitArgs s_a;
    const BatchTask* tasks = task_base + range[0];
    const int32_t n = range[1];
    for (int32_t t = blockIdx.x; t < n; t += gridDim.x) {
        const BatchTask task = tasks[t];
        load_visit(s_a, visits + task.visit);
        __syncthreads();
        insert_part<B, KT>(s_a, f, task.part, parts, ish);
        __syncthreads();
    }
}

}  // namespace

namespace {
template <typename K, typename... Args>
cudaError_t launch_ex(K kernel, int cluster, bool pdl, int grid, int block, size_t smem, cudaStream_t s,
                      Args... args) {
    if (cluster <= 1 && !pdl) {
        kernel<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    unsigned n = 0;
    if (cluster > 1) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = cluster;
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    if (pdl) {
        at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
}  // namespace

cudaError_t launch_scan(const VisitArgs& a, const FilterCfg& f, int grid, int block, size_t smem,
                        cudaStream_t s, bool pdl) {
    const int c = a.cluster;
    if (a.in_bits) {
        if (f.block_bits == 512) {
            if (f.k == 4) return launch_ex(pt_scan_sparse_kernel<512, 4>, c, pdl, grid, block, smem, s, a, f);
            return launch_ex(pt_scan_sparse_kernel<512, 0>, c, pdl, grid, block, smem, s, a, f);
        }
        if (f.k == 4) return launch_ex(pt_scan_sparse_kernel<256, 4>, c, pdl, grid, block, smem, s, a, f);
        return launch_ex(pt_scan_sparse_kernel<256, 0>, c, pdl, grid, block, smem, s, a, f);
    }
    if (f.block_bits == 512) {
        if (f.k == 4) return launch_ex(pt_scan_kernel<512, 4>, c, pdl, grid, block, smem, s, a, f);
        return launch_ex(pt_scan_kernel<512, 0>, c, pdl, grid, block, smem, s, a, f);
    }
    if (f.k == 4) return launch_ex(pt_scan_kernel<256, 4>, c, pdl, grid, block, smem, s, a, f);
    return launch_ex(pt_scan_kernel<256, 0>, c, pdl, grid, block, smem, s, a, f);
}

cudaError_t launch_probe_first(const VisitArgs& a, const FilterCfg& f, uint32_t* mid, int32_t* first,
                               int32_t smem_words, int32_t gate_words, int32_t gate, int grid, int block,
                               size_t smem, cudaStream_t s) {
    if (f.block_bits == 512) {
        if (f.k == 4) pt_probe_first_kernel<512, 4><<<grid, block, smem, s>>>(a, f, mid, first, smem_words, gate_words, gate);
        else pt_probe_first_kernel<512, 0><<<grid, block, smem, s>>>(a, f, mid, first, smem_words, gate_words, gate);
    } else {
        if (f.k == 4) pt_probe_first_kernel<256, 4><<<grid, block, smem, s>>>(a, f, mid, first, smem_words, gate_words, gate);
        else pt_probe_first_kernel<256, 0><<<grid, block, smem, s>>>(a, f, mid, first, smem_words, gate_words, gate);
    }
    return cudaGetLastError();
}

cudaError_t launch_probe_first_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                                     const FilterCfg& f, int32_t smem_words, int32_t gate_words, int32_t gate,
                                     int grid, size_t smem, cudaStream_t s) {
    const int block = kFirstThreads;
    if (f.block_bits == 512) {
        if (f.k == 4)
            pt_probe_first_batch_kernel<512, 4><<<grid, block, smem, s>>>(visits, tasks, range, f, smem_words, gate_words, gate);
        else
            pt_probe_first_batch_kernel<512, 0><<<grid, block, smem, s>>>(visits, tasks, range, f, smem_words, gate_words, gate);
    } else {
        if (f.k == 4)
            pt_probe_first_batch_kernel<256, 4><<<grid, block, smem, s>>>(visits, tasks, range, f, smem_words, gate_words, gate);
        else
            pt_probe_first_batch_kernel<256, 0><<<grid, block, smem, s>>>(visits, tasks, range, f, smem_words, gate_words, gate);
    }
    return cudaGetLastError();
}

int probe_first_batch_max_ctas_per_sm(int block_bits, size_t smem) {
    int n = 0, m = 0;
    if (block_bits == 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_probe_first_batch_kernel<512, 4>, kFirstThreads, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_probe_first_batch_kernel<512, 0>, kFirstThreads, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_probe_first_batch_kernel<256, 4>, kFirstThreads, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_probe_first_batch_kernel<256, 0>, kFirstThreads, smem);
    }
    return n < m ? n : m;
}

int probe_first_max_ctas_per_sm(int block_bits, int block, size_t smem) {
    int n = 0, m = 0;
    if (block_bits == 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_probe_first_kernel<512, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_probe_first_kernel<512, 0>, block, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_probe_first_kernel<256, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_probe_first_kernel<256, 0>, block, smem);
    }
    return n < m ? n : m;
}

int insert_max_ctas_per_sm(int block_bits, int block) {
    int n = 0, m = 0;
    if (block_bits == 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_insert_kernel<512, 4>, block, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_insert_kernel<512, 0>, block, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_insert_kernel<256, 4>, block, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_insert_kernel<256, 0>, block, 0);
    }
    return n < m ? n : m;
}

cudaError_t launch_pass_through(const VisitArgs& a, const FilterCfg& f, int grid, cudaStream_t s, bool pdl) {
    return launch_ex(pt_pass_through_kernel, 1, pdl, grid, 512, 0, s, a, f);
}

cudaError_t launch_size_clear(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s) {
    pt_size_clear_kernel<<<grid, block, 0, s>>>(a, f);
    return cudaGetLastError();
}

cudaError_t launch_insert(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s, bool pdl) {
    if (f.block_bits == 512) {
        if (f.k == 4) return launch_ex(pt_insert_kernel<512, 4>, 1, pdl, grid, block, 0, s, a, f);
        return launch_ex(pt_insert_kernel<512, 0>, 1, pdl, grid, block, 0, s, a, f);
    }
    if (f.k == 4) return launch_ex(pt_insert_kernel<256, 4>, 1, pdl, grid, block, 0, s, a, f);
    return launch_ex(pt_insert_kernel<256, 0>, 1, pdl, grid, block, 0, s, a, f);
}

cudaError_t launch_probe_list(const VisitArgs& a, const FilterCfg& f, int grid, size_t smem, cudaStream_t s,
                              bool pdl) {
    const int block = kListThreads;
    if (f.block_bits == 512) {
        if (f.k == 4) return launch_ex(pt_probe_list_kernel<512, 4>, 1, pdl, grid, block, smem, s, a, f);
        return launch_ex(pt_probe_list_kernel<512, 0>, 1, pdl, grid, block, smem, s, a, f);
    }
    if (f.k == 4) return launch_ex(pt_probe_list_kernel<256, 4>, 1, pdl, grid, block, smem, s, a, f);
    return launch_ex(pt_probe_list_kernel<256, 0>, 1, pdl, grid, block, smem, s, a, f);
}

cudaError_t probe_list_set_smem_limit(int block_bits, size_t smem) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if (block_bits == 512) {
        if ((e = cudaFuncSetAttribute(pt_probe_list_kernel<512, 4>, at, (int)smem)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(pt_probe_list_kernel<512, 0>, at, (int)smem);
    }
    if ((e = cudaFuncSetAttribute(pt_probe_list_kernel<256, 4>, at, (int)smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(pt_probe_list_kernel<256, 0>, at, (int)smem);
}

int scan_max_ctas_per_sm(int block_bits, int block, size_t smem, bool sparse) {
    int n = 0, m = 0;
    // every instantiation of a kernel has the same launch bounds; take the smallest fit
    if (sparse) {
        if (block_bits == 512) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_sparse_kernel<512, 4>, block, smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_sparse_kernel<512, 0>, block, smem);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_sparse_kernel<256, 4>, block, smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_sparse_kernel<256, 0>, block, smem);
        }
        return n < m ? n : m;
    }
    if (block_bits == 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_kernel<512, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_kernel<512, 0>, block, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_kernel<256, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_kernel<256, 0>, block, smem);
    }
    return n < m ? n : m;
}

cudaError_t scan_set_smem_limit(int block_bits, size_t smem) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if (block_bits == 512) {
        if ((e = cudaFuncSetAttribute(pt_scan_kernel<512, 4>, at, (int)smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(pt_scan_sparse_kernel<512, 4>, at, (int)smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(pt_scan_sparse_kernel<512, 0>, at, (int)smem)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(pt_scan_kernel<512, 0>, at, (int)smem);
    }
    if ((e = cudaFuncSetAttribute(pt_scan_kernel<256, 4>, at, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pt_scan_sparse_kernel<256, 4>, at, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pt_scan_sparse_kernel<256, 0>, at, (int)smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(pt_scan_kernel<256, 0>, at, (int)smem);
}

cudaError_t launch_scan_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                              const FilterCfg& f, int cluster, int grid, int block, size_t smem, cudaStream_t s) {
    if (f.block_bits == 512) {
        if (f.k == 4) return launch_ex(pt_scan_batch_kernel<512, 4>, cluster, false, grid, block, smem, s, visits, tasks, range, f);
        return launch_ex(pt_scan_batch_kernel<512, 0>, cluster, false, grid, block, smem, s, visits, tasks, range, f);
    }
    if (f.k == 4) return launch_ex(pt_scan_batch_kernel<256, 4>, cluster, false, grid, block, smem, s, visits, tasks, range, f);
    return launch_ex(pt_scan_batch_kernel<256, 0>, cluster, false, grid, block, smem, s, visits, tasks, range, f);
}

cudaError_t launch_size_clear_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range,
                                    int parts, const FilterCfg& f, int grid, int block, cudaStream_t s) {
    pt_size_clear_batch_kernel<<<grid, block, 0, s>>>(visits, tasks, range, parts, f);
    return cudaGetLastError();
}

cudaError_t launch_insert_batch(const VisitArgs* visits, const BatchTask* tasks, const int32_t* range, int parts,
                                const FilterCfg& f, int grid, int block, cudaStream_t s) {
    if (f.block_bits == 512) {
        if (f.k == 4) pt_insert_batch_kernel<512, 4><<<grid, block, 0, s>>>(visits, tasks, range, parts, f);
        else pt_insert_batch_kernel<512, 0><<<grid, block, 0, s>>>(visits, tasks, range, parts, f);
    } else {
        if (f.k == 4) pt_insert_batch_kernel<256, 4><<<grid, block, 0, s>>>(visits, tasks, range, parts, f);
        else pt_insert_batch_kernel<256, 0><<<grid, block, 0, s>>>(visits, tasks, range, parts, f);
    }
    return cudaGetLastError();
}

int scan_batch_max_ctas_per_sm(int block_bits, int block, size_t smem) {
    int n = 0, m = 0;
    if (block_bits == 512) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_batch_kernel<512, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_batch_kernel<512, 0>, block, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_batch_kernel<256, 4>, block, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, pt_scan_batch_kernel<256, 0>, block, smem);
    }
    return n < m ? n : m;
}

cudaError_t scan_batch_set_smem_limit(int block_bits, size_t smem) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if (block_bits == 512) {
        if ((e = cudaFuncSetAttribute(pt_scan_batch_kernel<512, 4>, at, (int)smem)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(pt_scan_batch_kernel<512, 0>, at, (int)smem);
    }
    if ((e = cudaFuncSetAttribute(pt_scan_batch_kernel<256, 4>, at, (int)smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(pt_scan_batch_kernel<256, 0>, at, (int)smem);
}

namespace {
__global__ void pt_hash_column_kernel(const void* keys, int32_t dtype, int64_t n, uint64_t seed, uint64_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        ColRef c{keys, dtype, 0};
        out[i] = hash_key(load_key(c, (uint32_t)i), seed);
    }
}
}  // namespace

cudaError_t launch_hash_column(const void* keys, int32_t dtype, int64_t n, uint64_t seed, uint64_t* out,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t grid = (n + 255) / 256;
    if (grid > 148 * 32) grid = 148 * 32;
    pt_hash_column_kernel<<<(int)grid, 256, 0, s>>>(keys, dtype, n, seed, out);
    return cudaGetLastError();
}

}  // namespace pt
