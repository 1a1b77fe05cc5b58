// Memory-bound helper kernels of the CUDA path: transposition into the
// k-contiguous operand layout, the exact int32 <-> fp32 carrier conversion,
// fills, and the APSP domain scan.  All are HBM-bound: tiles of 32 x 32 move
// through padded shared memory so that both the read and the write are
// coalesced.
#include <cstdint>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace btas {

// Value map of the exact fp32 carrier for int32 data (used only when every
// finite magnitude is < 2^23, so every value and every pairwise sum is an
// exactly representable float):  INF <-> +inf, -INF <-> -inf.
__device__ __forceinline__ uint32_t carrier_map(uint32_t bits, int mode) {
    if (mode == 1) {
        const int v = static_cast<int>(bits);
        const float f = v == kInfI32 ? __int_as_float(0x7f800000)
                      : v == kNinfI32 ? __int_as_float(0xff800000)
                                      : static_cast<float>(v);
        return __float_as_uint(f);
    }
    if (mode == 2) {
        const float f = __uint_as_float(bits);
        // finite values are exact integers < 2^24; anything at or beyond the
        // int32 clamp threshold is INF (cannot occur for in-domain data)
        int v;
        if (f >= static_cast<float>(kClampI32)) v = kInfI32;
        else if (f <= -static_cast<float>(kClampI32)) v = kNinfI32;
        else v = static_cast<int>(f);
        return static_cast<uint32_t>(v);
    }
    return bits;
}

__global__ void transpose4_kernel(const uint32_t *__restrict__ src, long long lds, int rows, int cols,
                                  uint32_t *__restrict__ dst, long long ldd, int mode, const int *skip) {
    if (skip != nullptr && *skip == 0) return;
    __shared__ uint32_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int r = r0 + ty + i, c = c0 + tx;
        if (r < rows && c < cols) tile[ty + i][tx] = carrier_map(src[(long long)r * lds + c], mode);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int c = c0 + ty + i, r = r0 + tx;  // dst row c, dst col r
        if (r < rows && c < cols) dst[(long long)c * ldd + r] = tile[tx][ty + i];
    }
}

__global__ void convert4_kernel(const uint32_t *__restrict__ src, long long lds, int rows, int cols,
                                uint32_t *__restrict__ dst, long long ldd, int mode) {
    const long long total = (long long)rows * cols;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / cols, c = idx % cols;
        dst[r * ldd + c] = carrier_map(src[r * lds + c], mode);
    }
}

__global__ void fill4_kernel(uint32_t *dst, long long ldd, int rows, int cols, uint32_t bits) {
    const long long total = (long long)rows * cols;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / cols, c = idx % cols;
        dst[r * ldd + c] = bits;
    }
}

// out[0] = max finite weight, out[1] = count of out-of-domain entries
// (W: n x n, row pitch ldw).
__global__ void apsp_scan_kernel(const int *__restrict__ W, long long ldw, long long n, int *out) {
    const long long total = n * n;
    int mx = 0, bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / n, c = idx % n;
        const int v = W[r * ldw + c];
        if (r == c) {
            bad += v != 0;
        } else if (v != kInfI32) {
            if (v < 0 || v > BTAS_I32_FINITE_MAX) ++bad;
            else mx = max(mx, v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], mx);
        if (bad) atomicAdd(&out[1], bad);
    }
}

// dst = E (+) src: the tropical identity E (0 on the diagonal, the (+)-identity
// elsewhere) (+)-added to src, i.e. src with its diagonal replaced by
// min(src_ii, 0) (min-plus) or max(src_ii, 0) (max-plus).
__global__ void ident_oplus_kernel(const uint32_t *__restrict__ src, long long lds, int n,
                                   uint32_t *__restrict__ dst, long long ldd, int sr, int is_float) {
    const long long total = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / n, c = idx % n;
        uint32_t v = src[r * lds + c];
        if (r == c) {
            if (is_float) {
                const float f = __uint_as_float(v);
                v = __float_as_uint(sr == kMin ? fminf(f, 0.f) : fmaxf(f, 0.f));
            } else {
                const int x = static_cast<int>(v);
                v = static_cast<uint32_t>(sr == kMin ? min(x, 0) : max(x, 0));
            }
        }
        dst[r * ldd + c] = v;
    }
}

// BTAS_GEMM_CHECKED: the entries of a rows x cols operand outside the
// product's domain -- int32: neither |v| <= 2^28 nor the semiring's
// (+)-identity; fp32: NaN, or the infinity of the other semiring (-inf in a
// min-plus operand, +inf in a max-plus one) -- are added to *count (this
// call) and to status[0] (the device's running total).
__global__ void domain_check_kernel(const uint32_t *__restrict__ X, long long ld, int rows, int cols, int is_float,
                                    int sr, int *count, unsigned long long *status) {
    const long long total = (long long)rows * cols;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / cols, c = idx % cols;
        const uint32_t bits = X[r * ld + c];
        if (is_float) {
            const float f = __uint_as_float(bits);
            const bool wrong_inf = sr == kMin ? (f == -__int_as_float(0x7f800000)) : (f == __int_as_float(0x7f800000));
            bad += (f != f) || wrong_inf;
        } else {
            const int v = static_cast<int>(bits);
            const bool fin = v >= -BTAS_I32_FINITE_MAX && v <= BTAS_I32_FINITE_MAX;
            bad += !(fin || v == (sr == kMin ? kInfI32 : kNinfI32));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) {
        atomicAdd(count, bad);
        atomicAdd(status, (unsigned long long)bad);
    }
}

// After the domain checks of one call: *skip = 1 when the call found an
// entry outside the domain (the product kernels then return without
// writing C) or, on the packed path, when the packed kernels run instead
// (the packed decision already saw the count); a violation counts the call
// in status[1].
__global__ void checked_gate_kernel(const int *count, const int *pack_state, int *skip,
                                    unsigned long long *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool bad = *count != 0;
    if (bad) atomicAdd(status + 1, 1ULL);
    *skip = (bad || (pack_state != nullptr && pack_state[kPackStateUse] != 0)) ? 1 : 0;
}

static int grid_for(long long total, int threads) {
    long long b = (total + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : static_cast<int>(b);
}

cudaError_t launch_transpose4(const void *src, long long lds, int rows, int cols, void *dst, long long ldd,
                              int mode, const int *skip, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose4_kernel<<<grid, block, 0, st>>>(static_cast<const uint32_t *>(src), lds, rows, cols,
                                              static_cast<uint32_t *>(dst), ldd, mode, skip);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert4(const void *src, long long lds, int rows, int cols, void *dst, long long ldd,
                            int mode, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    convert4_kernel<<<grid_for((long long)rows * cols, 256), 256, 0, st>>>(
        static_cast<const uint32_t *>(src), lds, rows, cols, static_cast<uint32_t *>(dst), ldd, mode);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill4(void *dst, long long ldd, int rows, int cols, uint32_t bits, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    fill4_kernel<<<grid_for((long long)rows * cols, 256), 256, 0, st>>>(static_cast<uint32_t *>(dst), ldd,
                                                                         rows, cols, bits);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ident_oplus(const void *src, long long lds, int n, void *dst, long long ldd, int sr, int is_float,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ident_oplus_kernel<<<grid_for((long long)n * n, 256), 256, 0, st>>>(
        static_cast<const uint32_t *>(src), lds, n, static_cast<uint32_t *>(dst), ldd, sr, is_float);
    note_launch();
    return cudaGetLastError();
}

unsigned long long *device_status_words() {
    static std::mutex mu;
    static unsigned long long *words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (words[dev] == nullptr) {
        void *p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, 256) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        words[dev] = static_cast<unsigned long long *>(p);
    }
    return words[dev];
}

cudaError_t launch_domain_check(const void *X, long long ld, int rows, int cols, int is_float, int sr, int *count,
                                unsigned long long *status, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    domain_check_kernel<<<grid_for((long long)rows * cols, 256), 256, 0, st>>>(
        static_cast<const uint32_t *>(X), ld, rows, cols, is_float, sr, count, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_checked_gate(const int *count, const int *pack_state, int *skip, unsigned long long *status,
                                cudaStream_t st) {
    checked_gate_kernel<<<1, 32, 0, st>>>(count, pack_state, skip, status);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_apsp_scan(const int *W, long long n, int *out, cudaStream_t st, long long ldw) {
    if (n <= 0) return cudaSuccess;
    apsp_scan_kernel<<<grid_for(n * n, 256), 256, 0, st>>>(W, ldw > 0 ? ldw : n, n, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace btas
