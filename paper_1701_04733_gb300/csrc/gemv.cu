// Level 2: tropical matrix-vector products, and single-source shortest paths
// by repeated vector-matrix products (Bellman-Ford in min-plus form).
//
//   trans == 0: y[i] = (+)_j A[i][j] (.) x[j]   one warp per row, 128-bit
//               loads along the row, warp-shuffle (+)-reduction
//   trans == 1: y[j] = (+)_i x[i] (.) A[i][j]   one thread per 4 columns,
//               row chunks spread over the grid, partial results combined
//               with atomic min/max (order-independent, so exact)
// Both stream A once: HBM-bound (4 bytes of A per term).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "grid_sync.cuh"
#include "kernels.h"

namespace btas {

namespace {

template <typename T, int SR>
__device__ __forceinline__ T op_plus(T a, T b) {
    return SR == kMin ? (b < a ? b : a) : (b > a ? b : a);
}
template <int SR>
__device__ __forceinline__ int op_times(int a, int b) {
    return clamp_i32<SR>(a + b);
}
template <int SR>
__device__ __forceinline__ float op_times(float a, float b) {
    return __fadd_rn(a, b);
}

// (+)-combine v into *addr atomically; returns true if *addr changed.
template <int SR>
__device__ __forceinline__ bool atomic_oplus(int *addr, int v) {
    const int old = SR == kMin ? atomicMin(addr, v) : atomicMax(addr, v);
    return SR == kMin ? v < old : v > old;
}
// Float min/max through integer atomics: non-negative floats order like
// their bit patterns as signed ints, negative floats in reverse as unsigned.
template <int SR>
__device__ __forceinline__ bool atomic_oplus(float *addr, float v) {
    if (SR == kMin) {
        if (__float_as_int(v) >= 0) return v < __int_as_float(atomicMin(reinterpret_cast<int *>(addr), __float_as_int(v)));
        return v < __uint_as_float(atomicMax(reinterpret_cast<unsigned *>(addr), __float_as_uint(v)));
    }
    if (__float_as_int(v) >= 0) return v > __int_as_float(atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v)));
    return v > __uint_as_float(atomicMin(reinterpret_cast<unsigned *>(addr), __float_as_uint(v)));
}

template <typename T, int SR>
__global__ void gemv_rows_kernel(int m, int n, const T *__restrict__ A, long long lda, const T *__restrict__ x,
                                 T *__restrict__ y, int accumulate, int vec) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= m) return;
    const T *row = A + (long long)warp * lda;
    T acc = Ident<T, SR>::v();
    if (vec) {
        int j = lane * 4;
        // four independent 128-bit loads in flight per lane
        for (; j + 384 + 4 <= n; j += 512) {
            uint4 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = __ldg(reinterpret_cast<const uint4 *>(row + j + 128 * u));
                b[u] = __ldg(reinterpret_cast<const uint4 *>(x + j + 128 * u));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t av[4] = {a[u].x, a[u].y, a[u].z, a[u].w}, bv[4] = {b[u].x, b[u].y, b[u].z, b[u].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    T ae, be;
                    memcpy(&ae, &av[q], 4);
                    memcpy(&be, &bv[q], 4);
                    acc = op_plus<T, SR>(acc, op_times<SR>(ae, be));
                }
            }
        }
        for (; j < n; j += 128) {
            if (j + 4 <= n) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(row + j));
                const uint4 b = __ldg(reinterpret_cast<const uint4 *>(x + j));
                const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    T ae, be;
                    memcpy(&ae, &av[q], 4);
                    memcpy(&be, &bv[q], 4);
                    acc = op_plus<T, SR>(acc, op_times<SR>(ae, be));
                }
            } else {
                for (int q = j; q < n; ++q) acc = op_plus<T, SR>(acc, op_times<SR>(row[q], x[q]));
            }
        }
    } else {
        for (int j = lane; j < n; j += 32) acc = op_plus<T, SR>(acc, op_times<SR>(row[j], x[j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = op_plus<T, SR>(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) y[warp] = accumulate ? op_plus<T, SR>(y[warp], acc) : acc;
}

constexpr int kColThreads = 256, kRowChunk = 64;

// y[j] (+)= (+)_{i in chunk} x[i] (.) A[i][j]; y must hold the (+)-identity
// or the accumulate start values.  *changed is set if some y entry changed.
template <typename T, int SR>
__global__ void gemv_cols_kernel(int m, int n, const T *__restrict__ A, long long lda, const T *__restrict__ x,
                                 T *y, int *changed, const int *skip, int vec) {
    if (skip != nullptr && __ldcg(skip) == 0) return;  // the previous relaxation changed nothing
    const int j0 = (blockIdx.x * kColThreads + threadIdx.x) * 4;
    const int i0 = blockIdx.y * kRowChunk, i1 = min(m, i0 + kRowChunk);
    if (j0 >= n) return;
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = Ident<T, SR>::v();
    const bool full = vec && j0 + 4 <= n;
#pragma unroll 8
    for (int i = i0; i < i1; ++i) {
        const T xi = __ldg(x + i);
        const T *row = A + (long long)i * lda;
        if (full) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(row + j0));
            const uint32_t av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                T ae;
                memcpy(&ae, &av[q], 4);
                acc[q] = op_plus<T, SR>(acc[q], op_times<SR>(xi, ae));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < n) acc[q] = op_plus<T, SR>(acc[q], op_times<SR>(xi, row[j0 + q]));
        }
    }
    bool ch = false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (j0 + q < n && acc[q] != Ident<T, SR>::v()) ch |= atomic_oplus<SR>(y + j0 + q, acc[q]);
    if (changed != nullptr && ch) atomicOr(changed, 1);
}

template <typename T>
__global__ void fill_kernel(T *y, int n, T v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = v;
}

template <typename T, int SR>
cudaError_t gemv_t(int trans, int m, int n, const void *A, long long lda, const void *x, void *y, int accumulate,
                   int *changed, const int *skip, cudaStream_t st) {
    const T *a = static_cast<const T *>(A);
    const T *xx = static_cast<const T *>(x);
    T *yy = static_cast<T *>(y);
    if (trans == 0) {
        const int vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(xx)) & 15) == 0 && (lda & 3) == 0;
        const int blocks = (m + 7) / 8;
        gemv_rows_kernel<T, SR><<<blocks, 256, 0, st>>>(m, n, a, lda, xx, yy, accumulate, vec);
        note_launch();
    } else {
        if (!accumulate) {
            int b = (n + 255) / 256;
            b = b > 1216 ? 1216 : (b < 1 ? 1 : b);
            fill_kernel<T><<<b, 256, 0, st>>>(yy, n, Ident<T, SR>::v());
            note_launch();
        }
        const int vec = (reinterpret_cast<uintptr_t>(a) & 15) == 0 && (lda & 3) == 0;
        dim3 grid((n + 4 * kColThreads - 1) / (4 * kColThreads), (m + kRowChunk - 1) / kRowChunk);
        gemv_cols_kernel<T, SR><<<grid, kColThreads, 0, st>>>(m, n, a, lda, xx, yy, changed, skip, vec);
        note_launch();
    }
    return cudaGetLastError();
}

// ---- Bellman-Ford SSSP (repeated vector-matrix products) in ONE
// cooperative launch.  d_0 = e_src; d_{t+1}[j] = min_i d_t[i] + W[i][j] until
// d stops changing (at most n - 1 products), with one grid barrier per
// product instead of a launch, a copy and a host read-back.
//
// A product is split into items of 64 rows x 1024 columns (256 threads, 4
// columns each); an item's partial minimum p over its rows is merged into
// d_{t+1} (reset to INF beforehand) with atomicMin.  W has a zero diagonal,
// so d_{t+1} <= d_t entrywise and the item holding row i = j has
// p <= d_t[j]: an item merges p only where p < d_t[j] (a change) or p equals
// it and it holds row j -- the same comparison is the change test.  Three
// rotating buffers: product t reads d_t, merges into d_{t+1} and resets
// d_{t+2}'s buffer.
constexpr int kSsspRows = 64, kSsspCols = 1024;

struct SsspArgs {
    const int *W;
    long long ldw;
    int n;
    int src;
    int vec;                  // W rows 16-byte aligned (int4 loads)
    int *buf0, *buf1, *buf2;  // n ints each
    int *dist;
    GridSync sync;            // status: info[1]
    int *info;                // [0] products that changed d, [1] status, [2] entries of W outside the domain, [3] any
};

__device__ __forceinline__ int *sssp_buf(const SsspArgs &a, int i) { return i == 0 ? a.buf0 : i == 1 ? a.buf1 : a.buf2; }

__global__ void __launch_bounds__(kColThreads) sssp_coop_kernel(const SsspArgs a) {
    const int n = a.n, tid = threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
    unsigned gen = 0;
    for (long long j = gtid; j < n; j += gthreads) {
        a.buf0[j] = j == a.src ? 0 : kInfI32;
        a.buf1[j] = kInfI32;
    }
    int v0 = 0, v1 = 0;
    if (!grid_barrier(a.sync, gen, false, nullptr, v0, v1)) return;
    const int cchunks = (n + kSsspCols - 1) / kSsspCols, rchunks = (n + kSsspRows - 1) / kSsspRows;
    const long long items = (long long)cchunks * rchunks;
    const long long it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
    int cur = 0, done = 0;
    const int *in = a.buf0;
    for (int t = 0; t + 1 < n; ++t) {
        int *out = sssp_buf(a, (cur + 1) % 3);
        int *nxt = sssp_buf(a, (cur + 2) % 3);
        for (long long j = gtid; j < n; j += gthreads) nxt[j] = kInfI32;
        bool ch = false;
        int bad = 0;
        __shared__ int s_x[kSsspRows];  // d_t over the item's rows
        for (long long it = it0; it < it1; ++it) {
            const int i0 = (int)(it / cchunks) * kSsspRows, i1 = min(n, i0 + kSsspRows);
            const int j0 = (int)(it % cchunks) * kSsspCols + tid * 4;
            __syncthreads();  // the previous item's reads of s_x are done
            if (tid < kSsspRows) s_x[tid] = i0 + tid < n ? __ldcg(in + i0 + tid) : kInfI32;
            __syncthreads();
            if (j0 >= n) continue;
            int4 acc = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
            if (t == 0) {
                // the first product reads every entry of W: check the domain
                // (zero diagonal, weights in [0, 2^28] or INF) on the way
                for (int i = i0; i < i1; ++i) {
                    const int xi = s_x[i - i0];
                    const int *row = a.W + (long long)i * a.ldw + j0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (j0 + c >= n) break;
                        const int v = row[c];
                        const bool fin = v >= 0 && v <= BTAS_I32_FINITE_MAX;
                        bad += ((!fin && v != kInfI32) || (i == j0 + c && v != 0)) ? 1 : 0;
                        if (c == 0) acc.x = __viaddmin_s32(xi, v, acc.x);
                        if (c == 1) acc.y = __viaddmin_s32(xi, v, acc.y);
                        if (c == 2) acc.z = __viaddmin_s32(xi, v, acc.z);
                        if (c == 3) acc.w = __viaddmin_s32(xi, v, acc.w);
                    }
                }
            } else if (a.vec && j0 + 4 <= n) {
#pragma unroll 8
                for (int i = i0; i < i1; ++i) {
                    const int xi = s_x[i - i0];
                    const int4 w = __ldg(reinterpret_cast<const int4 *>(a.W + (long long)i * a.ldw + j0));
                    acc.x = __viaddmin_s32(xi, w.x, acc.x);
                    acc.y = __viaddmin_s32(xi, w.y, acc.y);
                    acc.z = __viaddmin_s32(xi, w.z, acc.z);
                    acc.w = __viaddmin_s32(xi, w.w, acc.w);
                }
            } else {
                for (int i = i0; i < i1; ++i) {
                    const int xi = s_x[i - i0];
                    const int *row = a.W + (long long)i * a.ldw + j0;
                    // columns past n read as INF
                    acc.x = __viaddmin_s32(xi, row[0], acc.x);
                    acc.y = __viaddmin_s32(xi, j0 + 1 < n ? row[1] : kInfI32, acc.y);
                    acc.z = __viaddmin_s32(xi, j0 + 2 < n ? row[2] : kInfI32, acc.z);
                    acc.w = __viaddmin_s32(xi, j0 + 3 < n ? row[3] : kInfI32, acc.w);
                }
            }
            const int accv[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + c;
                if (j >= n) continue;
                const int p = clamp_i32<kMin>(accv[c]);
                const int o = __ldcg(in + j);
                if (p < kInfI32 && (p < o || (p == o && j >= i0 && j < i1))) {
                    atomicMin(out + j, p);
                    ch |= p < o;
                }
            }
        }
        int changed = 0;
        if (t == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
            if ((tid & 31) == 0 && bad) {
                atomicAdd(a.info + 2, bad);
                atomicExch(a.info + 3, 1);
            }
        }
        if (!grid_barrier(a.sync, gen, ch, t == 0 ? a.info + 3 : nullptr, changed, v1)) return;
        if (t == 0 && v1 != 0) return;  // W outside the domain: dist untouched
        in = out;
        cur = (cur + 1) % 3;
        if (!changed) break;
        ++done;
    }
    for (long long j = gtid; j < n; j += gthreads) a.dist[j] = __ldcg(in + j);
    if (blockIdx.x == 0 && tid == 0) a.info[0] = done;
}

}  // namespace

cudaError_t launch_gemv(int sr, int dtype, int trans, int m, int n, const void *A, long long lda, const void *x,
                        void *y, int accumulate, int *changed, cudaStream_t st, const int *skip) {
    if (dtype == BTAS_I32)
        return sr == kMin ? gemv_t<int, kMin>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st)
                          : gemv_t<int, kMax>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st);
    return sr == kMin ? gemv_t<float, kMin>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st)
                      : gemv_t<float, kMax>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st);
}

size_t sssp_coop_workspace(long long n) { return 3 * (((size_t)n * 4 + 255) & ~size_t(255)) + 512; }

cudaError_t launch_sssp_coop(const int *W, long long n, int src, int *dist, void *ws, int *info, cudaStream_t st) {
    DeviceInfo di{};
    int dev = 0;
    if (!current_device_info(&di, &dev)) return cudaErrorInvalidDevice;
    static std::mutex mu;
    static int cached[64];
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && cached[dev] > 0) {
            per_sm = cached[dev];
        } else {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sssp_coop_kernel, kColThreads, 0);
            if (e != cudaSuccess) return e;
            if (dev < 64) cached[dev] = per_sm;
        }
    }
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const size_t vb = ((size_t)n * 4 + 255) & ~size_t(255);
    char *base = static_cast<char *>(ws);
    SsspArgs a{};
    a.W = W;
    a.ldw = n;
    a.n = (int)n;
    a.src = src;
    a.vec = ((reinterpret_cast<uintptr_t>(W) & 15) == 0) && (n & 3) == 0;
    a.buf0 = reinterpret_cast<int *>(base);
    a.buf1 = reinterpret_cast<int *>(base + vb);
    a.buf2 = reinterpret_cast<int *>(base + 2 * vb);
    a.dist = dist;
    a.info = info;
    a.sync.bar = reinterpret_cast<unsigned *>(base + 3 * vb);
    a.sync.status = info + 1;
    a.sync.timeout_cycles = (long long)(2.0 * (di.clock_khz > 0 ? di.clock_khz : 2000000) * 1e3);  // about 2 s
    cudaError_t e = cudaMemsetAsync(base + 3 * vb, 0, 256, st);
    if (e != cudaSuccess) return e;
    const long long items = ((n + kSsspCols - 1) / kSsspCols) * ((n + kSsspRows - 1) / kSsspRows);
    const int grid = (int)std::max(1LL, std::min(items, (long long)per_sm * di.sms));
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(sssp_coop_kernel), dim3(grid), dim3(kColThreads),
                                    args, 0, st);
    note_launch();
    return e;
}

}  // namespace btas
