// APSP by repeated squaring (Sec. III) for n <= 128 in ONE thread block
// (by default the library sends it n <= 64; see apsp_small_limit).
//
// For a small graph the general path is latency-bound: every squaring is a
// separate launch over a handful of tiles, with a host round trip for the
// change flag.  Here D lives in shared memory (two 128 x 128 int32 buffers,
// 128 KiB) and one block of 1024 threads runs the domain check and all
// squarings, each thread owning a 4 x 4 block of outputs: one launch, one
// read-back.  The arithmetic is that of the int32 product kernels (DPX
// add-min, INF absorption by the clamp at INF - 2^28), so the result is
// bit-identical to the general path.
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"

namespace btas {
namespace {

constexpr int kMaxN = 128, kLd = kMaxN, kThreads = 1024;
constexpr int kSmem = 2 * kMaxN * kLd * 4 + 64;

// info: [0] entries outside the domain, [1] largest finite weight,
// [2] squarings that changed D
__global__ void __launch_bounds__(kThreads, 1)
    apsp_small_kernel(const int *W, long long ldw, int n, int S, int early, int *D, long long ldd, int *info) {
    // W and D may be the same matrix: every load of W precedes every store to D
    extern __shared__ __align__(16) int sm[];
    int *const buf0 = sm, *const buf1 = sm + kMaxN * kLd;
    int *flags = sm + 2 * kMaxN * kLd;  // [0] bad, [1] max weight, [2..] changed per squaring
    const int tid = threadIdx.x;
    const int n4 = (n + 3) & ~3;
    if (tid < 16) flags[tid] = 0;
    __syncthreads();
    int bad = 0, mx = 0;
    for (int idx = tid; idx < n4 * n4; idx += kThreads) {
        const int i = idx / n4, j = idx % n4;
        int v = kInfI32;
        if (i < n && j < n) {
            v = W[(long long)i * ldw + j];
            const bool fin = v >= 0 && v <= BTAS_I32_FINITE_MAX;
            if ((!fin && v != kInfI32) || (i == j && v != 0)) ++bad;
            if (fin) mx = max(mx, v);
        }
        buf0[i * kLd + j] = v;
    }
    if (bad) atomicAdd(&flags[0], bad);
    atomicMax(&flags[1], mx);
    __syncthreads();
    if (flags[0] != 0) {
        if (tid == 0) {
            info[0] = flags[0];
            info[1] = flags[1];
            info[2] = 0;
        }
        return;
    }
    const int tx = tid & 31, ty = tid >> 5;
    const int i0 = ty * 4, j0 = tx * 4;
    const bool mine = i0 < n4 && j0 < n4;
    int cur = 0, done = 0;
    for (int s = 1; s <= S; ++s) {
        const int *in = cur ? buf1 : buf0;
        int *out = cur ? buf0 : buf1;
        bool ch = false;
        if (mine) {
            int acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = kInfI32;
            for (int k = 0; k < n4; k += 4) {
                int4 a[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = *reinterpret_cast<const int4 *>(in + (i0 + r) * kLd + k);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int4 b = *reinterpret_cast<const int4 *>(in + (k + q) * kLd + j0);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int av = q == 0 ? a[r].x : q == 1 ? a[r].y : q == 2 ? a[r].z : a[r].w;
                        acc[r][0] = __viaddmin_s32(av, b.x, acc[r][0]);
                        acc[r][1] = __viaddmin_s32(av, b.y, acc[r][1]);
                        acc[r][2] = __viaddmin_s32(av, b.z, acc[r][2]);
                        acc[r][3] = __viaddmin_s32(av, b.w, acc[r][3]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = i0 + r, j = j0 + c;
                    int v = clamp_i32<kMin>(acc[r][c]);
                    if (i >= n || j >= n) v = kInfI32;  // padding stays INF
                    ch |= v != in[i * kLd + j];
                    out[i * kLd + j] = v;
                }
        }
        if (__any_sync(0xffffffffu, ch) && tx == 0) flags[2 + (s & 7)] = 1;
        __syncthreads();
        const int changed = flags[2 + (s & 7)];
        // clear the slot used by squaring s + 4 before anyone reaches it
        if (tid == 0) flags[2 + ((s + 4) & 7)] = 0;
        cur ^= 1;
        done += changed;
        if (!changed && early) break;
        __syncthreads();
    }
    for (int idx = tid; idx < n * n; idx += kThreads) {
        const int i = idx / n, j = idx % n;
        D[(long long)i * ldd + j] = (cur ? buf1 : buf0)[i * kLd + j];
    }
    if (tid == 0) {
        info[0] = 0;
        info[1] = flags[1];
        info[2] = done;
    }
}

}  // namespace

int apsp_small_max_n() { return kMaxN; }

int apsp_small_limit() {
    // graphs up to this size take the one-block kernel, larger ones the
    // cooperative kernel, which is faster from n of about 72 on (one SM's DPX
    // rate against a few grid barriers per squaring); BTAS_APSP_SMALL_MAX_N
    // overrides it (0 .. 128)
    static const int dflt = 64;
    const char *e = getenv("BTAS_APSP_SMALL_MAX_N");
    if (!e || !*e) return dflt;
    const int v = atoi(e);
    return v < 0 ? 0 : v > kMaxN ? kMaxN : v;
}

cudaError_t launch_apsp_small(const int *W, long long ldw, int n, int S, bool early, int *D, long long ldd,
                              int *info, cudaStream_t st) {
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(apsp_small_kernel), kSmem);
    if (e != cudaSuccess) return e;
    apsp_small_kernel<<<1, kThreads, kSmem, st>>>(W, ldw, n, S, early ? 1 : 0, D, ldd, info);
    note_launch();
    return cudaGetLastError();
}

}  // namespace btas
