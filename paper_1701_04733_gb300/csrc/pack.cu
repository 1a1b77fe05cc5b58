// Exact packed 16-bit path for int32 tropical products (BTAS_GEMM_PACKED).
//
// Both semirings (Eq. 1-4) commute with a shift of each operand: for
// min-plus, min_l (a_il + b_lj) = min_l ((a_il - lo_A) + (b_lj - lo_B)) +
// lo_A + lo_B, and for max-plus, max_l (a_il + b_lj) = hi_A + hi_B -
// min_l ((hi_A - a_il) + (hi_B - b_lj)).  After the shift every finite
// operand lies in [0, R] (R = hi - lo of its matrix), and when R_A + R_B <
// 0x7FFF every finite term fits below the 16-bit INF (0x7FFF), so the packed
// u16x2 min-plus kernel computes the product exactly; the (+)-identity maps
// to 0x7FFF, which absorbs in the saturating 16-bit add.  Whether the
// condition holds is decided on the device from a scan of both operands, so
// the call stays asynchronous: the packed kernels and the int32 kernels are
// both enqueued and the ones not chosen return at once.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace btas {
namespace {

__device__ unsigned long long g_packed_products = 0;

// state layout
constexpr int kUse = 0, kOffA = 1, kOffB = 2, kNotUse = 3, kLoA = 4, kHiA = 5, kLoB = 6, kHiB = 7, kBad = 8;

__device__ __forceinline__ bool finite_i32(int v) { return v >= -(1 << 28) && v <= (1 << 28); }

__global__ void pack_init_kernel(int *state) {
    if (threadIdx.x == 0) {
        state[kUse] = 0;
        state[kNotUse] = 1;
        state[kLoA] = INT_MAX;
        state[kHiA] = INT_MIN;
        state[kLoB] = INT_MAX;
        state[kHiB] = INT_MIN;
        state[kBad] = 0;
    }
}

// Finite range of a rows x cols int32 matrix, and the number of entries that
// are neither finite nor the semiring's (+)-identity.
__global__ void pack_range_kernel(const int *__restrict__ X, long long rows, long long cols, long long ld, int ident,
                                  int *lo_out, int *hi_out, int *bad_out) {
    int lo = INT_MAX, hi = INT_MIN, bad = 0;
    const long long total = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = X[(i / cols) * ld + i % cols];
        if (finite_i32(v)) {
            lo = min(lo, v);
            hi = max(hi, v);
        } else if (v != ident) {
            ++bad;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo != INT_MAX) atomicMin(lo_out, lo);
        if (hi != INT_MIN) atomicMax(hi_out, hi);
        if (bad) atomicAdd(bad_out, bad);
    }
}

// extra_bad (optional): entries outside the domain found by the caller's
// own check (BTAS_GEMM_CHECKED); any withdraws the packed path.
__global__ void pack_decide_kernel(int sr, int *state, const int *extra_bad) {
    if (threadIdx.x != 0) return;
    const bool any_a = state[kLoA] <= state[kHiA], any_b = state[kLoB] <= state[kHiB];
    const long long ra = any_a ? (long long)state[kHiA] - state[kLoA] : 0;
    const long long rb = any_b ? (long long)state[kHiB] - state[kLoB] : 0;
    const int use = state[kBad] == 0 && (extra_bad == nullptr || *extra_bad == 0) && ra + rb < BTAS_INF_U16;
    state[kUse] = use;
    state[kNotUse] = !use;
    state[kOffA] = any_a ? (sr == kMin ? state[kLoA] : state[kHiA]) : 0;
    state[kOffB] = any_b ? (sr == kMin ? state[kLoB] : state[kHiB]) : 0;
    if (use) atomicAdd(&g_packed_products, 1ULL);
}

__device__ __forceinline__ uint32_t shift16(int v, int sr, int off) {
    if (!finite_i32(v)) return BTAS_INF_U16;
    return (uint32_t)(sr == kMin ? v - off : off - v);
}

// A (m x k) -> duplicated 16-bit words of the shifted values (pitch ldad).
__global__ void pack_a_kernel(const int *__restrict__ A, long long lda, int m, int k, int sr, const int *state,
                              uint32_t *__restrict__ Ad, long long ldad) {
    if (__ldcg(state + kUse) == 0) return;
    const int off = __ldcg(state + kOffA);
    const long long total = (long long)m * k;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / k, c = i % k;
        Ad[r * ldad + c] = 0x10001u * shift16(A[r * lda + c], sr, off);
    }
}

// B (k x n) -> shifted uint16 values, row-major k x n (pitch ldbu).
__global__ void pack_b_kernel(const int *__restrict__ B, long long ldb, int k, int n, int sr, const int *state,
                              uint16_t *__restrict__ Bu, long long ldbu) {
    if (__ldcg(state + kUse) == 0) return;
    const int off = __ldcg(state + kOffB);
    const long long total = (long long)k * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n, c = i % n;
        Bu[r * ldbu + c] = (uint16_t)shift16(B[r * ldb + c], sr, off);
    }
}

// B given transposed (Bt: n x k) -> shifted uint16 B, row-major k x n,
// through 32 x 32 shared-memory tiles (coalesced on both sides).
__global__ void pack_bt_kernel(const int *__restrict__ Bt, long long ldb, int k, int n, int sr, const int *state,
                               uint16_t *__restrict__ Bu, long long ldbu) {
    if (__ldcg(state + kUse) == 0) return;
    __shared__ uint16_t tile[32][33];
    const int off = __ldcg(state + kOffB);
    const int j0 = blockIdx.y * 32, l0 = blockIdx.x * 32;  // Bt rows j (output cols), cols l (output rows)
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, l = l0 + threadIdx.x;
        if (j < n && l < k) tile[r][threadIdx.x] = (uint16_t)shift16(Bt[(long long)j * ldb + l], sr, off);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int l = l0 + r, j = j0 + threadIdx.x;
        if (l < k && j < n) Bu[(long long)l * ldbu + j] = tile[threadIdx.x][r];
    }
}

// Shifted 16-bit result -> int32 C (optionally (+)-accumulated into C).
__global__ void pack_finish_kernel(const uint16_t *__restrict__ Cu, long long ldcu, int m, int n, int sr,
                                   const int *state, int *__restrict__ C, long long ldc, int accumulate) {
    if (__ldcg(state + kUse) == 0) return;
    const int off = __ldcg(state + kOffA) + __ldcg(state + kOffB);
    const int ident = sr == kMin ? kInfI32 : kNinfI32;
    const long long total = (long long)m * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n, c = i % n;
        const int u = Cu[r * ldcu + c];
        int v = u >= BTAS_INF_U16 ? ident : (sr == kMin ? off + u : off - u);
        int *pc = C + r * ldc + c;
        if (accumulate) v = sr == kMin ? min(*pc, v) : max(*pc, v);
        *pc = v;
    }
}

unsigned grid_of(long long total) {
    return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
}

}  // namespace

cudaError_t launch_pack_prepare(int sr, int m, int n, int k, const int *A, long long lda, const int *B, long long ldb,
                                bool trans_b, int *state, uint32_t *adup, uint16_t *bu, long long ldbu,
                                cudaStream_t st, const int *extra_bad) {
    const int ident = sr == kMin ? kInfI32 : kNinfI32;
    pack_init_kernel<<<1, 32, 0, st>>>(state);
    pack_range_kernel<<<grid_of((long long)m * k), 256, 0, st>>>(A, m, k, lda, ident, state + kLoA, state + kHiA,
                                                                state + kBad);
    if (trans_b)
        pack_range_kernel<<<grid_of((long long)n * k), 256, 0, st>>>(B, n, k, ldb, ident, state + kLoB,
                                                                    state + kHiB, state + kBad);
    else
        pack_range_kernel<<<grid_of((long long)k * n), 256, 0, st>>>(B, k, n, ldb, ident, state + kLoB,
                                                                    state + kHiB, state + kBad);
    pack_decide_kernel<<<1, 32, 0, st>>>(sr, state, extra_bad);
    const long long ldad = (k + 3) & ~3LL;
    pack_a_kernel<<<grid_of((long long)m * k), 256, 0, st>>>(A, lda, m, k, sr, state, adup, ldad);
    if (trans_b) {
        const dim3 grid((unsigned)((k + 31) / 32), (unsigned)((n + 31) / 32));
        pack_bt_kernel<<<grid, dim3(32, 8), 0, st>>>(B, ldb, k, n, sr, state, bu, ldbu);
    } else {
        pack_b_kernel<<<grid_of((long long)k * n), 256, 0, st>>>(B, ldb, k, n, sr, state, bu, ldbu);
    }
    note_launch(7);
    return cudaGetLastError();
}

cudaError_t launch_pack_finish(int sr, int m, int n, const uint16_t *cu, long long ldcu, const int *state, int *C,
                               long long ldc, bool accumulate, cudaStream_t st) {
    pack_finish_kernel<<<grid_of((long long)m * n), 256, 0, st>>>(cu, ldcu, m, n, sr, state, C, ldc,
                                                                  accumulate ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

long long packed_products(int device) {
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return -1;
    if (device != prev && cudaSetDevice(device) != cudaSuccess) return -1;
    unsigned long long v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_packed_products, sizeof v);
    if (device != prev) cudaSetDevice(prev);
    return e == cudaSuccess ? (long long)v : -1;
}

}  // namespace btas
