// APSP by repeated squaring (Sec. III) for mid-size graphs in ONE
// cooperative launch.
//
// Between the one-block kernel (n <= 128) and the tiled product kernels, a
// solve is bound by launches and host round trips: a few dozen tiles per
// squaring cannot fill the GPU, and every squaring waits for the previous
// one's change flag.  Here one cooperative grid runs the domain check and all
// squarings, separated by grid barriers.  Each squaring is split into (64 x
// 64 output tile, k-chunk) work items so that every SM has work; an item
// computes the tile's partial minimum over its k-chunk and merges it into
// the output with atomicMin -- exact, because (+) = min is associative,
// commutative and idempotent, and the INF clamp commutes with min.  The
// arithmetic per term is the int32 product's (DPX add-min), so results are
// bit-identical to the other paths.
//
// Squaring s reads X_{s-1} (X_0 = a pitch-n copy of W) and writes X_s into
// one of three rotating buffers; X_{s+1}'s buffer is reset to INF while
// squaring s is checked for change.  Every grid barrier wait is bounded (clock64); on
// expiry the kernel records BTAS_ERR_TIMEOUT and all blocks return.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace btas {
namespace {

constexpr int kT = 64, kThreads = 256, kKc = 32;  // tile edge, threads, k step

struct MidArgs {
    const int *W;
    long long ldw;
    int n;
    int S;
    int early;
    int *D;
    long long ldd;
    int *buf0, *buf1, *buf2;  // n x ldx each; columns n .. ldx-1 always hold INF
    long long ldx;            // round4(n): 16-byte rows for vector staging
    int kchunks;      // k-chunks per output tile
    int chunk;        // k-chunk length (multiple of kKc)
    unsigned *bar;    // [0] arrivals, [32] generation (separate 128-byte lines)
    int *info;        // [0] bad entries, [1] max weight, [2] squarings that changed, [3] status, [4..] changed[s]
    long long timeout_cycles;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier (sense by generation).  Returns false if the status
// word is set (timeout here or elsewhere): the caller returns.
__device__ bool grid_barrier(const MidArgs &a) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_u32(a.bar + 32);
        __threadfence();
        if (atomicAdd(a.bar, 1u) == gridDim.x - 1) {
            atomicExch(a.bar, 0u);
            __threadfence();
            atomicAdd(a.bar + 32, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(a.bar + 32) == g) {
                if (ld_acquire_i32(a.info + 3) != 0) break;
                if (clock64() - t0 > a.timeout_cycles) {
                    atomicCAS(a.info + 3, 0, BTAS_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ld_acquire_i32(a.info + 3) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int *bufp(const MidArgs &a, int i) { return i == 0 ? a.buf0 : i == 1 ? a.buf1 : a.buf2; }

__global__ void __launch_bounds__(kThreads) apsp_mid_kernel(const MidArgs a) {
    __shared__ __align__(16) int sa[kT][kKc + 4];
    __shared__ __align__(16) int sb[kKc][kT];
    const int n = a.n, tid = threadIdx.x;
    const long long ldx = a.ldx;
    const long long nx = (long long)n * ldx;
    const long long gthreads = (long long)gridDim.x * kThreads;
    const long long gtid = (long long)blockIdx.x * kThreads + tid;

    // phase 0: domain check, W -> X_0 (buf2), X_1's buffer to INF
    {
        int bad = 0, mx = 0;
        for (long long idx = gtid; idx < nx; idx += gthreads) {
            const int i = (int)(idx / ldx), j = (int)(idx % ldx);
            int v = kInfI32;
            if (j < n) {
                v = a.W[(long long)i * a.ldw + j];
                const bool fin = v >= 0 && v <= BTAS_I32_FINITE_MAX;
                if ((!fin && v != kInfI32) || (i == j && v != 0)) ++bad;
                if (fin) mx = max(mx, v);
            }
            a.buf2[idx] = v;
            a.buf0[idx] = kInfI32;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bad += __shfl_xor_sync(0xffffffffu, bad, o);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if ((tid & 31) == 0) {
            if (bad) atomicAdd(a.info + 0, bad);
            atomicMax(a.info + 1, mx);
        }
    }
    if (!grid_barrier(a)) return;
    if (ld_acquire_i32(a.info + 0) != 0) return;  // D untouched

    const int tiles = (n + kT - 1) / kT;
    const int items = tiles * tiles * a.kchunks;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4 x 4 outputs each
    const int *in = a.buf2;  // X_0
    int cur = 0, done = 0;   // X_s (s >= 1) lives in buf[(s - 1) % 3]
    for (int s = 1; s <= a.S; ++s) {
        int *out = bufp(a, cur);
        // phase A: partial products merged with atomicMin
        for (int it = blockIdx.x; it < items; it += gridDim.x) {
            const int tile = it / a.kchunks, kc = it % a.kchunks;
            const int bm = (tile / tiles) * kT, bn = (tile % tiles) * kT;
            const int k0 = kc * a.chunk, k1 = min(n, k0 + a.chunk);
            if (k0 >= k1) continue;
            int acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = kInfI32;
            for (int kb = k0; kb < k1; kb += kKc) {
                // stage A[bm.., kb..] (64 x 32) and B[kb.., bn..] (32 x 64) with
                // 16-byte loads, all issued before the shared-memory stores.  A
                // vector that starts inside the matrix ends inside the row (ldx
                // is a multiple of 4) and reads INF padding past column n-1;
                // k-chunks end on multiples of 32, so no vector crosses one.
                int4 va[2], vb[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int e = tid + q * kThreads;
                    const int ra = e >> 3, ca = (e & 7) * 4;  // A: 8 vectors per row
                    const int gi = bm + ra, gka = kb + ca;
                    va[q] = (gi < n && gka < k1) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gi * ldx + gka))
                                                 : make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
                    const int rb = e >> 4, cb = (e & 15) * 4;  // B: 16 vectors per row
                    const int gkb = kb + rb, gj = bn + cb;
                    vb[q] = (gkb < k1 && gj < n) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gkb * ldx + gj))
                                                 : make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int e = tid + q * kThreads;
                    *reinterpret_cast<int4 *>(&sa[e >> 3][(e & 7) * 4]) = va[q];
                    *reinterpret_cast<int4 *>(&sb[e >> 4][(e & 15) * 4]) = vb[q];
                }
                __syncthreads();
#pragma unroll 4
                for (int k = 0; k < kKc; ++k) {
                    int av[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) av[r] = sa[ty * 4 + r][k];
                    const int4 b = *reinterpret_cast<const int4 *>(&sb[k][tx * 4]);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][0] = __viaddmin_s32(av[r], b.x, acc[r][0]);
                        acc[r][1] = __viaddmin_s32(av[r], b.y, acc[r][1]);
                        acc[r][2] = __viaddmin_s32(av[r], b.z, acc[r][2]);
                        acc[r][3] = __viaddmin_s32(av[r], b.w, acc[r][3]);
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = bm + ty * 4 + r, j = bn + tx * 4 + c;
                    const int v = clamp_i32<kMin>(acc[r][c]);
                    if (i < n && j < n && v < kInfI32) atomicMin(out + (long long)i * ldx + j, v);
                }
        }
        if (!grid_barrier(a)) return;
        // phase B: change check of X_s against X_{s-1}; X_{s+1}'s buffer to INF
        {
            int *nxt = bufp(a, (cur + 1) % 3);
            bool ch = false;
            for (long long idx = gtid; idx < nx; idx += gthreads) {
                ch |= __ldcg(out + idx) != __ldcg(in + idx);
                if (s < a.S) nxt[idx] = kInfI32;
            }
            if (__any_sync(0xffffffffu, ch) && (tid & 31) == 0) atomicOr(a.info + 4 + s, 1);
        }
        if (!grid_barrier(a)) return;
        const int changed = ld_acquire_i32(a.info + 4 + s);
        done += changed;
        in = out;
        cur = (cur + 1) % 3;
        if (!changed && a.early) break;
    }
    // result: X_last -> D (W was read only in phase 0, so D may be W)
    for (long long idx = gtid; idx < (long long)n * n; idx += gthreads)
        a.D[(idx / n) * a.ldd + idx % n] = __ldcg(in + (idx / n) * ldx + idx % n);
    if (blockIdx.x == 0 && tid == 0) a.info[2] = done;
}

}  // namespace

int apsp_mid_max_n() { return 1024; }

size_t apsp_mid_workspace(long long n, int S) {
    const size_t mat = ((size_t)n * ((n + 3) & ~3LL) * 4 + 255) & ~size_t(255);
    return 3 * mat + 256 + (((size_t)(S + 8) * 4 + 255) & ~size_t(255));
}

cudaError_t launch_apsp_mid(const int *W, long long ldw, int n, int S, bool early, int *D, long long ldd, void *ws,
                            int *info_out_dev, cudaStream_t st) {
    // device facts and the kernel's occupancy, queried once per device
    DeviceInfo di{};
    int dev = 0;
    if (!current_device_info(&di, &dev)) return cudaErrorInvalidDevice;
    static std::mutex mu;
    static int cached_per_sm[64];
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && cached_per_sm[dev] > 0) {
            per_sm = cached_per_sm[dev];
        } else {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apsp_mid_kernel, kThreads, 0);
            if (e != cudaSuccess) return e;
            if (dev < 64) cached_per_sm[dev] = per_sm;
        }
    }
    const int sms = di.sms, clk_khz = di.clock_khz;
    const int tiles = (n + kT - 1) / kT;
    const int want = 2 * sms;
    int kchunks = std::max(1, std::min((n + kKc - 1) / kKc, (want + tiles * tiles - 1) / (tiles * tiles)));
    int chunk = ((n + kchunks - 1) / kchunks + kKc - 1) / kKc * kKc;
    kchunks = (n + chunk - 1) / chunk;
    const int grid = std::max(1, std::min(tiles * tiles * kchunks, std::min(want, per_sm * sms)));
    const long long ldx = (n + 3) & ~3LL;
    const size_t mat = ((size_t)n * ldx * 4 + 255) & ~size_t(255);
    char *base = static_cast<char *>(ws);
    MidArgs a{};
    a.W = W;
    a.ldw = ldw;
    a.n = n;
    a.S = S;
    a.early = early ? 1 : 0;
    a.D = D;
    a.ldd = ldd;
    a.ldx = ldx;
    a.buf0 = reinterpret_cast<int *>(base);
    a.buf1 = reinterpret_cast<int *>(base + mat);
    a.buf2 = reinterpret_cast<int *>(base + 2 * mat);
    a.bar = reinterpret_cast<unsigned *>(base + 3 * mat);
    a.info = info_out_dev;
    a.kchunks = kchunks;
    a.chunk = chunk;
    a.timeout_cycles = (long long)(2.0 * (clk_khz > 0 ? clk_khz : 2000000) * 1e3);  // about 2 s
    cudaError_t e = cudaMemsetAsync(base + 3 * mat, 0, 256, st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(apsp_mid_kernel), dim3(grid), dim3(kThreads), args, 0,
                                    st);
    note_launch();
    return e;
}

}  // namespace btas
