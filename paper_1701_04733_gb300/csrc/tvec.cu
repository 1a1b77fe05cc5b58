// Level-1 tropical vector operations ("standard vector operations", abstract
// and Sec. III), built from Eq. 1-4:
//   dot  : r = (+)_i x_i (.) y_i        (grid-stride partial (+), then one block)
//   axpy : y_i <- y_i (+) (alpha (.) x_i)
//   add  : z_i = x_i (+) y_i
//   mul  : z_i = x_i (.) y_i
// All are HBM-bound streaming kernels.  (+) is associative, commutative and
// idempotent, so the reduction order does not change the result.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace btas {

template <typename T, int SR>
__device__ __forceinline__ T oplus(T a, T b) {
    return SR == kMin ? (b < a ? b : a) : (b > a ? b : a);
}
template <int SR>
__device__ __forceinline__ int otimes(int a, int b) {
    return clamp_i32<SR>(a + b);
}
template <int SR>
__device__ __forceinline__ float otimes(float a, float b) {
    return __fadd_rn(a, b);
}

template <typename T, int SR>
__global__ void dot_partial_kernel(long long n, const T *__restrict__ x, long long incx,
                                   const T *__restrict__ y, long long incy, T *partials) {
    T acc = Ident<T, SR>::v();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc = oplus<T, SR>(acc, otimes<SR>(x[i * incx], y[i * incy]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = oplus<T, SR>(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ T warp_acc[32];
    if ((threadIdx.x & 31) == 0) warp_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        T v = threadIdx.x < nw ? warp_acc[threadIdx.x] : Ident<T, SR>::v();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = oplus<T, SR>(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

template <typename T, int SR>
__global__ void dot_final_kernel(const T *partials, int count, T *result) {
    T acc = Ident<T, SR>::v();
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc = oplus<T, SR>(acc, partials[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = oplus<T, SR>(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ T warp_acc[32];
    if ((threadIdx.x & 31) == 0) warp_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T v = warp_acc[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = oplus<T, SR>(v, warp_acc[w]);
        *result = v;
    }
}

template <typename T, int SR>
__global__ void axpy_kernel(long long n, T alpha, const T *__restrict__ x, long long incx, T *y, long long incy) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i * incy] = oplus<T, SR>(y[i * incy], otimes<SR>(alpha, x[i * incx]));
}

template <typename T, int SR, int OP>
__global__ void ewise_kernel(long long n, const T *__restrict__ x, const T *__restrict__ y, T *__restrict__ z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        z[i] = OP == 0 ? oplus<T, SR>(x[i], y[i]) : otimes<SR>(x[i], y[i]);
}

static int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : static_cast<int>(b);
}

template <typename T, int SR>
static cudaError_t dot_t(long long n, const void *x, long long incx, const void *y, long long incy, void *result,
                         void *partials, int nblocks, cudaStream_t st) {
    dot_partial_kernel<T, SR><<<nblocks, 256, 0, st>>>(n, static_cast<const T *>(x), incx,
                                                       static_cast<const T *>(y), incy, static_cast<T *>(partials));
    note_launch();
    dot_final_kernel<T, SR><<<1, 256, 0, st>>>(static_cast<const T *>(partials), nblocks, static_cast<T *>(result));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_dot(int sr, int dtype, long long n, const void *x, long long incx, const void *y, long long incy,
                       void *result, void *partials, int nblocks, cudaStream_t st) {
    if (dtype == BTAS_I32)
        return sr == kMin ? dot_t<int, kMin>(n, x, incx, y, incy, result, partials, nblocks, st)
                          : dot_t<int, kMax>(n, x, incx, y, incy, result, partials, nblocks, st);
    return sr == kMin ? dot_t<float, kMin>(n, x, incx, y, incy, result, partials, nblocks, st)
                      : dot_t<float, kMax>(n, x, incx, y, incy, result, partials, nblocks, st);
}

cudaError_t launch_axpy(int sr, int dtype, long long n, uint32_t alpha_bits, const void *x, long long incx, void *y,
                        long long incy, cudaStream_t st) {
    const int b = blocks_for(n);
    if (dtype == BTAS_I32) {
        const int a = static_cast<int>(alpha_bits);
        if (sr == kMin) axpy_kernel<int, kMin><<<b, 256, 0, st>>>(n, a, (const int *)x, incx, (int *)y, incy);
        else axpy_kernel<int, kMax><<<b, 256, 0, st>>>(n, a, (const int *)x, incx, (int *)y, incy);
    } else {
        float a;
        memcpy(&a, &alpha_bits, 4);
        if (sr == kMin) axpy_kernel<float, kMin><<<b, 256, 0, st>>>(n, a, (const float *)x, incx, (float *)y, incy);
        else axpy_kernel<float, kMax><<<b, 256, 0, st>>>(n, a, (const float *)x, incx, (float *)y, incy);
    }
    note_launch();
    return cudaGetLastError();
}

template <typename T>
static void ewise_t(int op, int sr, long long n, const void *x, const void *y, void *z, cudaStream_t st) {
    const int b = blocks_for(n);
    const T *xx = static_cast<const T *>(x);
    const T *yy = static_cast<const T *>(y);
    T *zz = static_cast<T *>(z);
    if (op == 0) {
        if (sr == kMin) ewise_kernel<T, kMin, 0><<<b, 256, 0, st>>>(n, xx, yy, zz);
        else ewise_kernel<T, kMax, 0><<<b, 256, 0, st>>>(n, xx, yy, zz);
    } else {
        if (sr == kMin) ewise_kernel<T, kMin, 1><<<b, 256, 0, st>>>(n, xx, yy, zz);
        else ewise_kernel<T, kMax, 1><<<b, 256, 0, st>>>(n, xx, yy, zz);
    }
    note_launch();
}

cudaError_t launch_ewise(int op, int sr, int dtype, long long n, const void *x, const void *y, void *z,
                         cudaStream_t st) {
    if (dtype == BTAS_I32) ewise_t<int>(op, sr, n, x, y, z, st);
    else ewise_t<float>(op, sr, n, x, y, z, st);
    return cudaGetLastError();
}

}  // namespace btas
