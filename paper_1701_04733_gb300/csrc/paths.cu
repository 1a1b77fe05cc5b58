// APSP with path reconstruction: repeated min-plus squaring (Sec. III) that
// also carries a next-hop (successor) matrix.
//
// One squaring: D'[i][j] = min_k D[i][k] + D[k][j]; k* = the SMALLEST k that
// attains the minimum; N'[i][j] = -1 if D'[i][j] is INF, N[i][j] if k* == i
// (the first leg is empty), else N[i][k*] (the first hop of the walk
// i -> k* -> j).  N_0[i][j] = j for an edge, i on the diagonal, -1 otherwise.
// With positive weights, following N from i reaches j along a shortest path.
//
// Kernel: 64 x 64 output tile, 256 threads with 4 x 4 outputs each, k staged
// through a cp.async ring (A = D rows, B = D^T rows, both k-contiguous).  Per
// group of 4 consecutive k: the group minimum by DPX add-min (one per term);
// only if it is strictly smaller than the running minimum is the first k of
// the group attaining it recorded.  k increases monotonically per thread, so
// the smallest minimising k survives.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tgemm.cuh"

namespace btas {

namespace {

constexpr int PBM = 64, PBK = 32, PLD = PBK + 4, PST = 3, PNT = 256;
constexpr int PSTAGE = 2 * PBM * PLD;

constexpr int PSMEM = PST * PSTAGE * 4;  // 54 KiB: dynamic shared memory

__global__ void __launch_bounds__(PNT, 2)
paths_square_kernel(int n, const int *__restrict__ D, long long ldd, const int *__restrict__ Dt, long long ldt,
                    const int *__restrict__ N, int *__restrict__ D2, int *__restrict__ N2, int *changed, int vec_a) {
    extern __shared__ __align__(16) int smem[];
    const int tid = threadIdx.x;
    const int tiles = (n + PBM - 1) / PBM;
    const int bm = (blockIdx.x / tiles) * PBM, bn = (blockIdx.x % tiles) * PBM;
    const int tr = tid >> 4, tc = tid & 15;
    int val[4][4], idx[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            val[i][j] = 0x7FFFFFFF;
            idx[i][j] = -1;
        }
    const int KT = (n + PBK - 1) / PBK;
    auto load = [&](int s, int kt) {
        int *sa = smem + s * PSTAGE;
        int *sb = sa + PBM * PLD;
        stage_rows<int, PBM, PBK, PLD, PNT>(sa, D, ldd, bm, n, kt * PBK, n, vec_a != 0, kInfI32, tid, true);
        stage_rows<int, PBM, PBK, PLD, PNT>(sb, Dt, ldt, bn, n, kt * PBK, n, true, kInfI32, tid, true);
    };
#pragma unroll
    for (int s = 0; s < PST - 1; ++s) {
        if (s < KT) load(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<PST - 2>();
        __syncthreads();
        if (kt + PST - 1 < KT) load((kt + PST - 1) % PST, kt + PST - 1);
        cp_async_commit();
        const int *sa = smem + (kt % PST) * PSTAGE;
        const int *sb = sa + PBM * PLD;
#pragma unroll 2
        for (int kk = 0; kk < PBK; kk += 4) {
            int4 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const int4 *>(sa + (tr + 16 * i) * PLD + kk);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const int4 *>(sb + (tc + 16 * j) * PLD + kk);
            const int k0 = kt * PBK + kk;
            // Two levels: the minimum of the 4 sums of this k-group costs one
            // DPX add-min per term; only when it beats the running minimum
            // (rarely, once the minimum has settled) is the first k of the
            // group that attains it looked up.  An equal group minimum keeps
            // the earlier, smaller k.  Same result as a per-term argmin.
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int cm = __viaddmin_s32(a[i].x, b[j].x, 0x7FFFFFFF);
                    cm = __viaddmin_s32(a[i].y, b[j].y, cm);
                    cm = __viaddmin_s32(a[i].z, b[j].z, cm);
                    cm = __viaddmin_s32(a[i].w, b[j].w, cm);
                    if (cm < val[i][j]) {
                        val[i][j] = cm;
                        idx[i][j] = k0 + (a[i].x + b[j].x == cm   ? 0
                                          : a[i].y + b[j].y == cm ? 1
                                          : a[i].z + b[j].z == cm ? 2
                                                                  : 3);
                    }
                }
        }
    }
    cp_async_wait<0>();
    bool ch = false;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = bm + tr + 16 * i, c = bn + tc + 16 * j;
            if (r < n && c < n) {
                const int d = val[i][j] >= kClampI32 ? kInfI32 : val[i][j];
                const int k = idx[i][j];
                const int nx = d == kInfI32 ? -1 : (k == r ? N[(long long)r * n + c] : N[(long long)r * n + k]);
                if (d != D[(long long)r * ldd + c] || nx != N[(long long)r * n + c]) ch = true;
                D2[(long long)r * n + c] = d;
                N2[(long long)r * n + c] = nx;
            }
        }
    if (__any_sync(0xffffffffu, ch) && (tid & 31) == 0) atomicOr(changed, 1);
}

__global__ void next_init_kernel(const int *__restrict__ W, long long n, int *__restrict__ N) {
    const long long total = n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / n, c = idx % n;
        N[idx] = r == c ? (int)r : (W[idx] == kInfI32 ? -1 : (int)c);
    }
}

}  // namespace

cudaError_t launch_next_init(const int *W, long long n, int *N, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long b = (n * n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    next_init_kernel<<<(int)b, 256, 0, st>>>(W, n, N);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_paths_square(int n, const int *D, long long ldd, const int *Dt, long long ldt, const int *N,
                                int *D2, int *N2, int *changed, cudaStream_t st) {
    const int tiles = (n + PBM - 1) / PBM;
    const int vec_a = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && ((ldd & 3) == 0);
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(paths_square_kernel), PSMEM);
    if (e != cudaSuccess) return e;
    paths_square_kernel<<<tiles * tiles, PNT, PSMEM, st>>>(n, D, ldd, Dt, ldt, N, D2, N2, changed, vec_a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace btas
