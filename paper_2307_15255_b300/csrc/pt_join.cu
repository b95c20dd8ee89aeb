// Join phase (Section 3.3 of the paper): the size of the join of the rows
// that survived the transfer, counted without building a tuple.
//
// On an acyclic join graph (a forest of inner equi-joins), each tree is
// rooted at its largest table.  Every surviving row starts with weight 1.
// Bottom-up, a child's rows are aggregated by their key on the edge to
// the parent into a device hash table (key -> summed weight), and each
// parent row's weight is multiplied by the sum under its own key (0 when
// absent).  A tree's join size is its root's weight sum; the join's is the
// product over trees.  The host side (pt_join_count) is in pt_runtime.cu.
#include <algorithm>

#include "pt_internal.h"

namespace pt {

namespace {

// SplitMix64 output function, here only to spread keys over the slots.
__device__ __forceinline__ uint64_t spread(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t key_of(const ColRef& c, int64_t r) {
    if (c.dtype == 0) return (uint64_t)(int64_t)__ldg(reinterpret_cast<const int32_t*>(c.p) + r);
    return (uint64_t)__ldg(reinterpret_cast<const long long*>(c.p) + r);
}

constexpr unsigned kEmpty = 0, kClaimed = 1, kReady = 2;
constexpr int kSpinLimit = 1 << 20;  // a claimed slot is ready a few instructions later

__global__ void pt_join_init_kernel(const uint32_t* __restrict__ bits, int64_t n, unsigned long long* __restrict__ w) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        w[r] = (__ldg(bits + (r >> 5)) >> (r & 31)) & 1u;
}

// Add each weighted row's weight to its key's slot (open addressing, linear
// probing).  A slot is claimed by a CAS of its state, filled, then marked
// ready; a thread that meets a claimed slot waits (at most kSpinLimit
// polls) for it to be ready before comparing keys.  err: 1 = a wait ran
// out, 2 = the table is full.
__global__ void pt_join_build_kernel(ColRef c0, ColRef c1, int32_t ncols, const unsigned long long* __restrict__ w,
                                     int64_t n, JoinSlot* __restrict__ table, uint64_t mask, int32_t* err) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long wr = w[r];
        if (!wr) continue;
        const uint64_t a = key_of(c0, r), b = ncols == 2 ? key_of(c1, r) : 0ull;
        uint64_t i = spread(a ^ spread(b)) & mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= mask && !done; ++probe, i = (i + 1) & mask) {
            JoinSlot& s = table[i];
            const unsigned st = atomicCAS(&s.state, kEmpty, kClaimed);
            if (st == kEmpty) {
                s.a = a;
                s.b = b;
                __threadfence();
                atomicExch(&s.state, kReady);
                atomicAdd(&s.sum, wr);
                done = true;
                break;
            }
            int spins = 0;
            while (*(volatile unsigned*)&s.state != kReady && spins < kSpinLimit) ++spins;
            if (spins >= kSpinLimit) {
                atomicExch(err, 1);
                return;
            }
            __threadfence();
            if (*(volatile unsigned long long*)&s.a == a && *(volatile unsigned long long*)&s.b == b) {
                atomicAdd(&s.sum, wr);
                done = true;
            }
        }
        if (!done) {
            atomicExch(err, 2);
            return;
        }
    }
}

// Multiply each weighted row's weight by the summed weight under its key
// (0 when no child row has it).  The table is complete: every slot is empty
// or ready.
__global__ void pt_join_probe_kernel(ColRef c0, ColRef c1, int32_t ncols, unsigned long long* __restrict__ w,
                                     int64_t n, const JoinSlot* __restrict__ table, uint64_t mask) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long wr = w[r];
        if (!wr) continue;
        const uint64_t a = key_of(c0, r), b = ncols == 2 ? key_of(c1, r) : 0ull;
        uint64_t i = spread(a ^ spread(b)) & mask;
        unsigned long long sum = 0;
        for (uint64_t probe = 0; probe <= mask; ++probe, i = (i + 1) & mask) {
            const JoinSlot& s = table[i];
            if (s.state == kEmpty) break;
            if (s.a == a && s.b == b) {
                sum = s.sum;
                break;
            }
        }
        w[r] = wr * sum;
    }
}

__global__ void pt_join_sum_kernel(const unsigned long long* __restrict__ w, int64_t n, unsigned long long* out) {
    unsigned long long s = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        s += w[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

int grid_for(int64_t n, int num_sms) {
    const int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms * 8));
}

}  // namespace

cudaError_t launch_join_init(const uint32_t* bits, int64_t n, unsigned long long* w, int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pt_join_init_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(bits, n, w);
    return cudaGetLastError();
}

cudaError_t launch_join_build(const ColRef& c0, const ColRef& c1, int32_t ncols, const unsigned long long* w, int64_t n,
                              JoinSlot* table, uint64_t mask, int32_t* err, int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pt_join_build_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(c0, c1, ncols, w, n, table, mask, err);
    return cudaGetLastError();
}

cudaError_t launch_join_probe(const ColRef& c0, const ColRef& c1, int32_t ncols, unsigned long long* w, int64_t n,
                              const JoinSlot* table, uint64_t mask, int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pt_join_probe_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(c0, c1, ncols, w, n, table, mask);
    return cudaGetLastError();
}

cudaError_t launch_join_sum(const unsigned long long* w, int64_t n, unsigned long long* out, int num_sms,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pt_join_sum_kernel<<<grid_for(n, num_sms), 256, 0, s>>>(w, n, out);
    return cudaGetLastError();
}

}  // namespace pt
