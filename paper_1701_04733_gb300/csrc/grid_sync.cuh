// Bounded grid-wide barrier for cooperative launches (all blocks resident).
//
// bar points at 64 words (256 bytes) zeroed before the launch: bar[0 .. 15]
// hold a ring of 8 64-bit arrival counters, bar[32 .. 33] the release word.
// Barrier g (g = 1, 2, ... in every block) counts arrivals in ring slot
// (g - 1) % 8: each block adds 1, plus 2^32 if its flag is set, so the last
// block to arrive learns the grid's flag from the value its add returns.  It
// resets the slot barrier g + 4 will use (every block is past barrier g - 4,
// its previous user, and none can reach g + 4 before this release), computes
// a value (by default it reads one word), and publishes barrier number, flag
// and value in one 64-bit release word; the other blocks poll that word, so
// one load gives them the release and both results.  Every wait is bounded: on expiry the block sets
// *status to BTAS_ERR_TIMEOUT and the barrier returns false, as it does once
// any block has set the status.  No trap, no fault.
#pragma once

#include "common.cuh"

namespace btas {

struct GridSync {
    unsigned *bar;
    int *status;
    long long timeout_cycles;
};

namespace gsync {
__device__ __forceinline__ int ld_acquire_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
}  // namespace gsync

// flag: this block's contribution (ORed over the grid, returned in v0);
// value(): called by the last block to arrive, once every block's writes
// before the barrier are visible; its low 30 bits are published (v1).
// Returns false if the status word is set: the caller returns.
template <class ValueFn>
__device__ __forceinline__ bool grid_barrier_fn(const GridSync &g, unsigned &gen, bool flag, ValueFn value, int &v0,
                                                int &v1) {
    __shared__ int s_ok, s_v0, s_v1;
    const int any = __syncthreads_or(flag ? 1 : 0);
    ++gen;
    if (threadIdx.x == 0) {
        unsigned long long *ring = reinterpret_cast<unsigned long long *>(g.bar);
        unsigned long long *pub = reinterpret_cast<unsigned long long *>(g.bar + 32);
        unsigned long long word = 0;
        __threadfence();
        const unsigned long long prev = atomicAdd(ring + ((gen - 1) & 7), 1ull | ((unsigned long long)(any != 0) << 32));
        if ((unsigned)prev == gridDim.x - 1) {
            __threadfence();
            atomicExch(ring + ((gen + 3) & 7), 0ull);
            const unsigned f = ((prev >> 32) != 0 || any != 0) ? 1u : 0u;
            const unsigned v = (unsigned)value() & 0x3FFFFFFFu;
            word = (unsigned long long)gen | ((unsigned long long)f << 32) | ((unsigned long long)v << 33);
            __threadfence();
            gsync::st_release_u64(pub, word);
        } else {
            const long long t0 = clock64();
            for (unsigned it = 1;; ++it) {
                word = gsync::ld_acquire_u64(pub);
                if ((unsigned)word == gen) break;
                // another block gave up (status set) or this wait expires
                if ((it & 15) == 0 && gsync::ld_acquire_i32(g.status) != 0) break;
                if (clock64() - t0 > g.timeout_cycles) {
                    atomicCAS(g.status, 0, BTAS_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = (unsigned)word == gen;
        s_v0 = (int)((word >> 32) & 1u);
        s_v1 = (int)(word >> 33);
    }
    __syncthreads();
    v0 = s_v0;
    v1 = s_v1;
    return s_ok != 0;
}

// pval: optional word in [0, 2^30) read after all arrivals (v1).
__device__ __forceinline__ bool grid_barrier(const GridSync &g, unsigned &gen, bool flag, const int *pval, int &v0,
                                             int &v1) {
    return grid_barrier_fn(
        g, gen, flag, [pval]() -> unsigned { return pval ? (unsigned)gsync::ld_relaxed_i32(pval) : 0u; }, v0, v1);
}

}  // namespace btas
