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

__device__ __forceinline__ uint64_t hash_pair(uint64_t a, uint64_t b, uint64_t seed) {
    return mix64(hash_key(a, seed) ^ b);
}

// Key of row r as u64; int32 values are sign-extended.
__device__ __forceinline__ uint64_t load_key(const ColRef& c, uint32_t r) {
    if (c.dtype == 0) return (uint64_t)(int64_t)__ldg(reinterpret_cast<const int32_t*>(c.p) + r);
    return (uint64_t)__ldg(reinterpret_cast<const long long*>(c.p) + r);
}

__device__ __forceinline__ uint64_t edge_hash(const ColRef& c0, const ColRef& c1, int ncols, uint32_t r,
                                              uint64_t seed) {
    const uint64_t a = load_key(c0, r);
    if (ncols == 2) return hash_pair(a, load_key(c1, r), seed);
    return hash_key(a, seed);
}

// Block of a hash: multiply-shift range reduction of its high word.
__device__ __forceinline__ uint32_t block_of(uint64_t h, uint32_t nblocks) {
    return __umulhi((uint32_t)(h >> 32), nblocks);
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

template <int B>
__device__ __forceinline__ bool probe_shared(const uint32_t* s_filt, uint32_t off, uint32_t nb, uint64_t h,
                                             int k) {
    constexpr uint32_t WPB = B / 32;
    const uint32_t base = off + block_of(h, nb) * WPB;
    const uint32_t lo = (uint32_t)h;
    const uint32_t h1 = lo & (B - 1), h2 = (lo >> 16) | 1u;
    bool ok = true;
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
        const uint32_t bit = (h1 + (uint32_t)i * h2) & (B - 1);
        ok &= ((s_filt[base + (bit >> 5)] >> (bit & 31)) & 1u) != 0;
    }
    return ok;
}

template <int B>
__device__ __forceinline__ bool probe_global(const uint32_t* __restrict__ f, uint32_t nb, uint64_t h, int k) {
    constexpr uint32_t WPB = B / 32;
    const uint32_t* blk = f + (size_t)block_of(h, nb) * WPB;
    const uint32_t lo = (uint32_t)h;
    const uint32_t h1 = lo & (B - 1), h2 = (lo >> 16) | 1u;
    bool ok = true;
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
        const uint32_t bit = (h1 + (uint32_t)i * h2) & (B - 1);
        ok &= ((__ldg(blk + (bit >> 5)) >> (bit & 31)) & 1u) != 0;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// 1. scan: probe every incoming filter, write the survivor bitmap, compact
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(1024) pt_scan_kernel(const VisitArgs a, const FilterCfg f) {
    extern __shared__ __align__(16) uint32_t s_filt[];
    __shared__ ProbeEdge s_pe[kMaxIn];     // incoming edges in probe order
    __shared__ int32_t s_off[kMaxIn];      // word offset in s_filt, or -1: probe from global
    __shared__ uint32_t s_nb[kMaxIn];
    constexpr int U = kWordsPerIter;
    constexpr uint32_t WPB = B / 32;

    if (threadIdx.x == 0) {
        // LIP-style order: ascending survivors/rows of the building visit, ties by edge id.
        int ord[kMaxIn];
        unsigned long long c[kMaxIn];
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) {
            ord[i] = i;
            c[i] = i < a.n_in ? *a.in[i].build_count : 0ull;
        }
        for (int i = 1; i < a.n_in; ++i) {
            const int x = ord[i];
            int j = i - 1;
            while (j >= 0) {
                const int y = ord[j];
                const unsigned long long lhs = c[x] * (unsigned long long)a.in[y].build_rows;
                const unsigned long long rhs = c[y] * (unsigned long long)a.in[x].build_rows;
                if (lhs < rhs || (lhs == rhs && a.in[x].edge_id < a.in[y].edge_id)) {
                    ord[j + 1] = ord[j];
                    --j;
                } else {
                    break;
                }
            }
            ord[j + 1] = x;
        }
        // Shared-memory placement, greedily in probe order.
        int32_t used = 0;
        for (int i = 0; i < a.n_in; ++i) {
            const ProbeEdge& pe = a.in[ord[i]];
            s_pe[i] = pe;
            const uint32_t nb = (uint32_t)*pe.nblocks;
            s_nb[i] = nb;
            const int64_t words = (int64_t)nb * WPB;
            if (used + words <= a.smem_words) {
                s_off[i] = used;
                used += (int32_t)words;
            } else {
                s_off[i] = -1;
            }
        }
    }
    __syncthreads();
    for (int i = 0; i < a.n_in; ++i) {
        if (s_off[i] < 0) continue;
        const uint4* src = reinterpret_cast<const uint4*>(s_pe[i].filter);
        uint4* dst = reinterpret_cast<uint4*>(s_filt + s_off[i]);
        const uint32_t n16 = s_nb[i] * (WPB / 4);
        for (uint32_t t = threadIdx.x; t < n16; t += blockDim.x) dst[t] = __ldg(src + t);
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t n_words = (a.n + 31) >> 5;
    const int64_t w_begin = gw * a.words_per_warp;
    const int64_t w_end = min(n_words, w_begin + a.words_per_warp);
    const uint32_t tail_bits = (uint32_t)(a.n & 31);
    const int k = f.k;
    const uint64_t seed = f.seed;

    uint32_t local = 0;
    unsigned long long psec = 0, bsec = 0;

    for (int64_t w0 = w_begin; w0 < w_end; w0 += U) {
        // input words: lane u loads word w0+u, then broadcast
        uint32_t mine = 0;
        if (lane < (uint32_t)U && w0 + lane < w_end) {
            const int64_t w = w0 + lane;
            mine = a.in_bits ? __ldg(a.in_bits + w) : 0xFFFFFFFFu;
            if (w == n_words - 1 && tail_bits) mine &= (1u << tail_bits) - 1u;
        }
        uint32_t alive[U];
#pragma unroll
        for (int u = 0; u < U; ++u) alive[u] = __shfl_sync(0xFFFFFFFFu, mine, u);

        for (int j = 0; j < a.n_in; ++j) {
            uint32_t any = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) any |= alive[u];
            if (!any) break;
            const ColRef c0 = s_pe[j].col[0];
            const ColRef c1 = s_pe[j].col[1];
            const int ncols = s_pe[j].ncols;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                psec += sectors_of(alive[u], c0.dtype);
                if (ncols == 2) psec += sectors_of(alive[u], c1.dtype);
            }
            uint64_t h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                h[u] = 0;
                if ((alive[u] >> lane) & 1u) {
                    const uint32_t r = (uint32_t)((w0 + u) * 32 + lane);
                    h[u] = edge_hash(c0, c1, ncols, r, seed);
                }
            }
            const int32_t off = s_off[j];
            const uint32_t nb = s_nb[j];
            if (off >= 0) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool live = (alive[u] >> lane) & 1u;
                    const bool pass = live && probe_shared<B>(s_filt, (uint32_t)off, nb, h[u], k);
                    alive[u] = __ballot_sync(0xFFFFFFFFu, pass);
                }
            } else {
                const uint32_t* fg = s_pe[j].filter;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool live = (alive[u] >> lane) & 1u;
                    const bool pass = live && probe_global<B>(fg, nb, h[u], k);
                    alive[u] = __ballot_sync(0xFFFFFFFFu, pass);
                }
            }
        }

        // survivor words: lane u stores word w0+u
        uint32_t outw = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (lane == (uint32_t)u) outw = alive[u];
        if (lane < (uint32_t)U && w0 + lane < w_end) a.out_bits[w0 + lane] = outw;

        if (a.ids) {
            uint32_t* seg = a.ids + (size_t)w_begin * 32;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t m = alive[u];
                if ((m >> lane) & 1u) seg[local + __popc(m & lt_mask)] = (uint32_t)((w0 + u) * 32 + lane);
                local += __popc(m);
            }
            for (int b = 0; b < a.n_bcols; ++b) {
                const int32_t dt = a.bcol[b].dtype;
#pragma unroll
                for (int u = 0; u < U; ++u) bsec += sectors_of(alive[u], dt);
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) local += __popc(alive[u]);
        }
    }

    if (lane == 0) {
        if (a.seg_count && gw < a.total_warps) a.seg_count[gw] = local;
        if (local) atomicAdd(a.count, (unsigned long long)local);
        if (psec) atomicAdd(a.stats + 0, psec);
        if (bsec) atomicAdd(a.stats + 1, bsec);
    }
}

// ---------------------------------------------------------------------------
// 2. size + clear the outgoing filters from the device-side survivor count
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) pt_size_clear_kernel(const VisitArgs a, const FilterCfg f) {
    const unsigned long long c = *a.count;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
#pragma unroll
    for (int e = 0; e < kMaxOut; ++e) {
        if (e >= a.n_out) break;
        const int64_t n_est = min((int64_t)c, a.out[e].probe_rows);
        int64_t nb = (n_est * f.bits_per_key + f.block_bits - 1) / f.block_bits;
        if (nb < 1) nb = 1;
        if (tid == 0) *a.out[e].nblocks = nb;
        uint4* p = reinterpret_cast<uint4*>(a.out[e].filter);
        const size_t n16 = (size_t)nb * (size_t)(f.block_bits / 128);
        for (size_t i = tid; i < n16; i += stride) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// ---------------------------------------------------------------------------
// 3. insert the survivors' outgoing keys
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(512) pt_insert_kernel(const VisitArgs a, const FilterCfg f) {
    constexpr uint32_t WPB = B / 32;
    __shared__ uint32_t s_nb[kMaxOut];
#pragma unroll
    for (int e = 0; e < kMaxOut; ++e)
        if (threadIdx.x == (unsigned)e && e < a.n_out) s_nb[e] = (uint32_t)*a.out[e].nblocks;
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const size_t seg_rows = (size_t)a.words_per_warp * 32;
    const int k = f.k;
    const uint64_t seed = f.seed;

    for (int64_t s = gw; s < a.total_warps; s += n_warps) {
        const uint32_t cnt = a.seg_count[s];
        const uint32_t* ids = a.ids + (size_t)s * seg_rows;
        for (uint32_t i = lane; i < cnt; i += 32) {
            const uint32_t r = ids[i];
#pragma unroll
            for (int e = 0; e < kMaxOut; ++e) {
                if (e >= a.n_out) break;
                const BuildEdge& be = a.out[e];
                const uint64_t h = edge_hash(be.col[0], be.col[1], be.ncols, r, seed);
                uint32_t* blk = be.filter + (size_t)block_of(h, s_nb[e]) * WPB;
                const uint32_t lo = (uint32_t)h;
                const uint32_t h1 = lo & (B - 1), h2 = (lo >> 16) | 1u;
                for (int t = 0; t < k; ++t) {
                    const uint32_t bit = (h1 + (uint32_t)t * h2) & (B - 1);
                    atomicOr(blk + (bit >> 5), 1u << (bit & 31));
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_scan(const VisitArgs& a, const FilterCfg& f, int grid, int block, size_t smem,
                        cudaStream_t s) {
    if (f.block_bits == 512)
        pt_scan_kernel<512><<<grid, block, smem, s>>>(a, f);
    else
        pt_scan_kernel<256><<<grid, block, smem, s>>>(a, f);
    return cudaGetLastError();
}

cudaError_t launch_size_clear(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s) {
    pt_size_clear_kernel<<<grid, block, 0, s>>>(a, f);
    return cudaGetLastError();
}

cudaError_t launch_insert(const VisitArgs& a, const FilterCfg& f, int grid, int block, cudaStream_t s) {
    if (f.block_bits == 512)
        pt_insert_kernel<512><<<grid, block, 0, s>>>(a, f);
    else
        pt_insert_kernel<256><<<grid, block, 0, s>>>(a, f);
    return cudaGetLastError();
}

int scan_max_ctas_per_sm(int block_bits, int block, size_t smem) {
    int n = 0;
    if (block_bits == 512)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_kernel<512>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pt_scan_kernel<256>, block, smem);
    return n;
}

cudaError_t scan_set_smem_limit(int block_bits, size_t smem) {
    if (block_bits == 512)
        return cudaFuncSetAttribute(pt_scan_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(pt_scan_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace pt
