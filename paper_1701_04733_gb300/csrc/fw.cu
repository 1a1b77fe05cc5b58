// Blocked Floyd-Warshall: the sequential algorithm of Algorithm 2 (pivot z
// outermost, relax D[x][y] through z) reorganised in B x B tiles.  For each
// pivot block kb:
//   phase 1: the diagonal tile relaxes through its own B pivots (one CTA,
//            pivots in order, tile held in shared memory);
//   phase 2: the tiles of row kb and column kb relax through the same pivots,
//            reading the finished diagonal tile;
//   phase 3: every other tile takes D[i][j] = min(D[i][j], min_k D[i][k] +
//            D[k][j]) over the B pivots of block kb -- a tropical product with
//            accumulate, run on the semiring GEMM kernel.
// For non-negative weights every relaxation order reaches the same distance
// matrix, so the result equals Algorithm 2 (and APSP by squaring) exactly,
// after n^3 terms instead of ceil(log2(n-1)) * n^3.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace btas {

namespace {

constexpr int FB = 128;  // tile edge
constexpr int FT = 256;  // threads

__device__ __forceinline__ int relax(int d, int a, int b) {
    const int s = a + b;  // operands in [0, INF]: no overflow
    return s < d ? s : d;
}

// Load tile (r0, c0) of D into shared memory (INF outside the matrix).
__device__ __forceinline__ void load_tile(int *sm, const int *D, long long n, int r0, int c0) {
    for (int idx = threadIdx.x; idx < FB * FB; idx += FT) {
        const int r = idx / FB, c = idx % FB;
        sm[idx] = (r0 + r < n && c0 + c < n) ? D[(long long)(r0 + r) * n + c0 + c] : kInfI32;
    }
}
__device__ __forceinline__ void store_tile(const int *sm, int *D, long long n, int r0, int c0) {
    for (int idx = threadIdx.x; idx < FB * FB; idx += FT) {
        const int r = idx / FB, c = idx % FB;
        if (r0 + r < n && c0 + c < n) D[(long long)(r0 + r) * n + c0 + c] = sm[idx];
    }
}

__global__ void __launch_bounds__(FT) fw_diag_kernel(int *D, long long n, int kb) {
    extern __shared__ int sm[];
    const int o = kb * FB;
    load_tile(sm, D, n, o, o);
    __syncthreads();
    for (int k = 0; k < FB; ++k) {
        for (int idx = threadIdx.x; idx < FB * FB; idx += FT) {
            const int r = idx / FB, c = idx % FB;
            sm[idx] = relax(sm[idx], sm[r * FB + k], sm[k * FB + c]);
        }
        __syncthreads();
    }
    store_tile(sm, D, n, o, o);
}

// blockIdx.x < nb: row panel tile (kb, b); else column panel tile (b, kb).
__global__ void __launch_bounds__(FT) fw_panel_kernel(int *D, long long n, int kb, int nb) {
    extern __shared__ int sm[];
    int *diag = sm, *blk = sm + FB * FB;
    const bool row = blockIdx.x < (unsigned)nb;
    const int b = row ? blockIdx.x : blockIdx.x - nb;
    if (b == kb) return;
    const int o = kb * FB;
    const int r0 = row ? o : b * FB, c0 = row ? b * FB : o;
    load_tile(diag, D, n, o, o);
    load_tile(blk, D, n, r0, c0);
    __syncthreads();
    for (int k = 0; k < FB; ++k) {
        for (int idx = threadIdx.x; idx < FB * FB; idx += FT) {
            const int r = idx / FB, c = idx % FB;
            blk[idx] = row ? relax(blk[idx], diag[r * FB + k], blk[k * FB + c])
                           : relax(blk[idx], blk[r * FB + k], diag[k * FB + c]);
        }
        __syncthreads();
    }
    store_tile(blk, D, n, r0, c0);
}

}  // namespace

cudaError_t launch_fw_phase12(int *D, long long n, int kb, cudaStream_t st) {
    const int nb = (int)((n + FB - 1) / FB);
    cudaError_t e = cudaFuncSetAttribute(fw_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FB * FB * 4);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fw_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * FB * FB * 4);
    if (e != cudaSuccess) return e;
    fw_diag_kernel<<<1, FT, FB * FB * 4, st>>>(D, n, kb);
    note_launch();
    if (nb > 1) {
        fw_panel_kernel<<<2 * nb, FT, 2 * FB * FB * 4, st>>>(D, n, kb, nb);
        note_launch();
    }
    return cudaGetLastError();
}

int fw_block() { return FB; }

}  // namespace btas
