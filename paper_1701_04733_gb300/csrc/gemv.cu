// Level 2: tropical matrix-vector products, and single-source shortest paths
// by repeated vector-matrix products (Bellman-Ford in min-plus form).
//
//   trans == 0: y[i] = (+)_j A[i][j] (.) x[j]   one warp per row, 128-bit
//               loads along the row, warp-shuffle (+)-reduction
//   trans == 1: y[j] = (+)_i x[i] (.) A[i][j]   one thread per 4 columns,
//               row chunks spread over the grid, partial results combined
//               with atomic min/max (order-independent, so exact)
// Both stream A once: HBM-bound (4 bytes of A per term).
#include <cstdint>

#include "common.cuh"
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

}  // namespace

cudaError_t launch_gemv(int sr, int dtype, int trans, int m, int n, const void *A, long long lda, const void *x,
                        void *y, int accumulate, int *changed, cudaStream_t st, const int *skip) {
    if (dtype == BTAS_I32)
        return sr == kMin ? gemv_t<int, kMin>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st)
                          : gemv_t<int, kMax>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st);
    return sr == kMin ? gemv_t<float, kMin>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st)
                      : gemv_t<float, kMax>(trans, m, n, A, lda, x, y, accumulate, changed, skip, st);
}

}  // namespace btas
