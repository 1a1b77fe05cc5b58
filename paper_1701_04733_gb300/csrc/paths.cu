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

// Element type of the argmin squaring: int32 (one DPX add-min per term, INF
// absorbed by the clamp at INF - 2^28) or binary32 (one round-to-nearest add
// per term, +inf absorbing on its own).
template <typename T>
struct PathsElem;
template <>
struct PathsElem<int> {
    using V = int4;
    static __device__ __forceinline__ int start() { return 0x7FFFFFFF; }
    static __device__ __forceinline__ int inf() { return kInfI32; }
    // min(acc, a + b)
    static __device__ __forceinline__ int addmin(int a, int b, int acc) { return __viaddmin_s32(a, b, acc); }
    static __device__ __forceinline__ int sum(int a, int b) { return a + b; }
    static __device__ __forceinline__ int finish(int v) { return v >= kClampI32 ? kInfI32 : v; }
    static __device__ __forceinline__ bool is_inf(int v) { return v == kInfI32; }
};
template <>
struct PathsElem<float> {
    using V = float4;
    static __device__ __forceinline__ float start() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float addmin(float a, float b, float acc) { return fminf(__fadd_rn(a, b), acc); }
    static __device__ __forceinline__ float sum(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float finish(float v) { return v; }
    static __device__ __forceinline__ bool is_inf(float v) { return isinf(v); }
};

template <typename T>
__global__ void __launch_bounds__(PNT, 2)
paths_square_kernel(int n, const T *__restrict__ D, long long ldd, const T *__restrict__ Dt, long long ldt,
                    const int *__restrict__ N, T *__restrict__ D2, int *__restrict__ N2, int *changed, int vec_a) {
    using E = PathsElem<T>;
    using V = typename E::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    const int tiles = (n + PBM - 1) / PBM;
    const int bm = (blockIdx.x / tiles) * PBM, bn = (blockIdx.x % tiles) * PBM;
    const int tr = tid >> 4, tc = tid & 15;
    T val[4][4];
    int idx[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            val[i][j] = E::start();
            idx[i][j] = -1;
        }
    const int KT = (n + PBK - 1) / PBK;
    auto load = [&](int s, int kt) {
        T *sa = smem + s * PSTAGE;
        T *sb = sa + PBM * PLD;
        stage_rows<T, PBM, PBK, PLD, PNT>(sa, D, ldd, bm, n, kt * PBK, n, vec_a != 0, E::inf(), tid, true);
        stage_rows<T, PBM, PBK, PLD, PNT>(sb, Dt, ldt, bn, n, kt * PBK, n, true, E::inf(), tid, true);
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
        const T *sa = smem + (kt % PST) * PSTAGE;
        const T *sb = sa + PBM * PLD;
#pragma unroll 2
        for (int kk = 0; kk < PBK; kk += 4) {
            V a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const V *>(sa + (tr + 16 * i) * PLD + kk);
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const V *>(sb + (tc + 16 * j) * PLD + kk);
            const int k0 = kt * PBK + kk;
            // Two levels: the minimum of the 4 sums of this k-group costs one
            // add-then-min per term; only when it beats the running minimum
            // (rarely, once the minimum has settled) is the first k of the
            // group that attains it looked up (the sums are recomputed with
            // the same rounding, so equality is exact).  An equal group
            // minimum keeps the earlier, smaller k.  Same result as a
            // per-term argmin.
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    T cm = E::addmin(a[i].x, b[j].x, E::start());
                    cm = E::addmin(a[i].y, b[j].y, cm);
                    cm = E::addmin(a[i].z, b[j].z, cm);
                    cm = E::addmin(a[i].w, b[j].w, cm);
                    if (cm < val[i][j]) {
                        val[i][j] = cm;
                        idx[i][j] = k0 + (E::sum(a[i].x, b[j].x) == cm   ? 0
                                          : E::sum(a[i].y, b[j].y) == cm ? 1
                                          : E::sum(a[i].z, b[j].z) == cm ? 2
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
                const T d = E::finish(val[i][j]);
                const int k = idx[i][j];
                const int nx = E::is_inf(d) ? -1 : (k == r ? N[(long long)r * n + c] : N[(long long)r * n + k]);
                if (d != D[(long long)r * ldd + c] || nx != N[(long long)r * n + c]) ch = true;
                D2[(long long)r * n + c] = d;
                N2[(long long)r * n + c] = nx;
            }
        }
    if (__any_sync(0xffffffffu, ch) && (tid & 31) == 0) atomicOr(changed, 1);
}

// Keyed squaring.  While every finite entry of D is <= kKeyMax and n <=
// 2^13, the pair (value, k) of one term is encoded as the single int32 key
// (value << 13) | k, so that the minimum key holds the minimum value and,
// among equal values, the smallest k.  The key of term (i, k, j) is the sum
// A'[i][k] + B'[k][j] with A' = D << 13 and B' = (D << 13) | k (row index),
// so one plain min-plus product of A' and B' -- the tuned int32 kernels --
// computes distances and argmins at once.  Finite keys stay below the
// product kernel's INF clamp (2 * 49151 << 13 | 8191 < INF - 2^28); INF
// entries encode as INF, and every key with an INF term is clamped to INF.
constexpr int kKeyShift = 13;
constexpr int kKeyMaxN = 1 << kKeyShift;

__device__ __forceinline__ int key_a(int v) { return v >= kInfI32 ? kInfI32 : v << kKeyShift; }
__device__ __forceinline__ int key_b(int v, int k) { return v >= kInfI32 ? kInfI32 : (v << kKeyShift) | k; }

// A' (same layout as D) and B'^T (ldt pitch: B'^T[j][k] = key_b(D[k][j], k)),
// through 32 x 32 shared tiles so that both are written coalesced.
__global__ void paths_encode_kernel(const int *__restrict__ D, int n, int *__restrict__ Ak, int *__restrict__ BkT,
                                    long long ldt) {
    __shared__ int tile[32][33];
    const int k0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int k = k0 + r, j = j0 + threadIdx.x;
        if (k < n && j < n) {
            const int v = D[(long long)k * n + j];
            Ak[(long long)k * n + j] = key_a(v);
            tile[r][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = j0 + r, k = k0 + threadIdx.x;
        if (j < n && k < n) BkT[(long long)j * ldt + k] = key_b(tile[threadIdx.x][r], k);
    }
}

// Keys -> D' and N' (K may be D'), the change flag and the largest finite
// entry of D'.  N'[i][j] = -1 for INF, N[i][j] if the minimising k is i,
// else N[i][k] -- the rule of the unkeyed kernel.  One block per row: the
// gathers N[i][k] stay within one row, and the flag and maximum cost one
// atomic each per row.
__global__ void __launch_bounds__(256) paths_decode_kernel(const int *K, const int *__restrict__ D,
                                                           const int *__restrict__ N, int n, int *Dn,
                                                           int *__restrict__ Nn, int *changed, int *maxfin) {
    __shared__ int s_mx[8];
    const int i = blockIdx.x;
    const long long row = (long long)i * n;
    bool ch = false;
    int mx = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int key = K[row + j];
        int d = kInfI32, nx = -1;
        if (key < kInfI32) {
            const int k = key & (kKeyMaxN - 1);
            d = key >> kKeyShift;
            nx = N[row + (k == i ? j : k)];
            mx = max(mx, d);
        }
        ch |= d != D[row + j] || nx != N[row + j];
        Dn[row + j] = d;
        Nn[row + j] = nx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    const int any = __syncthreads_or(ch ? 1 : 0);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, s_mx[w]);
        mx = max(mx, s_mx[0]);
        if (any) atomicOr(changed, 1);
        atomicMax(maxfin, mx);
    }
}

template <typename T>
__global__ void next_init_kernel(const T *__restrict__ W, long long n, int *__restrict__ N) {
    const long long total = n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / n, c = idx % n;
        N[idx] = r == c ? (int)r : (PathsElem<T>::is_inf(W[idx]) ? -1 : (int)c);
    }
}

// Weight domain of the binary32 next-hop solve: zero diagonal, every other
// entry >= 0 or +inf (no NaN, no -inf).  out: number of entries outside it.
__global__ void paths_scan_f32_kernel(const float *__restrict__ W, long long n, int *out) {
    const long long total = n * n;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / n, c = idx % n;
        const float v = W[idx];
        bad += r == c ? (v != 0.f) : !(v >= 0.f);  // NaN and negative values (and -inf) fail v >= 0
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(out, bad);
}

}  // namespace

static int paths_grid(long long n) {
    long long b = (n * n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_next_init(const int *W, long long n, int *N, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    next_init_kernel<int><<<paths_grid(n), 256, 0, st>>>(W, n, N);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_next_init_f32(const float *W, long long n, int *N, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    next_init_kernel<float><<<paths_grid(n), 256, 0, st>>>(W, n, N);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_paths_scan_f32(const float *W, long long n, int *bad, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    paths_scan_f32_kernel<<<paths_grid(n), 256, 0, st>>>(W, n, bad);
    note_launch();
    return cudaGetLastError();
}

int paths_key_max() { return 49151; }
int paths_key_max_n() { return kKeyMaxN; }

cudaError_t launch_paths_encode(const int *D, int n, int *Ak, int *BkT, long long ldt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid((n + 31) / 32, (n + 31) / 32);
    paths_encode_kernel<<<grid, dim3(32, 8), 0, st>>>(D, n, Ak, BkT, ldt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_paths_decode(const int *K, const int *D, const int *N, long long n, int *Dn, int *Nn, int *changed,
                                int *maxfin, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    paths_decode_kernel<<<(int)n, 256, 0, st>>>(K, D, N, (int)n, Dn, Nn, changed, maxfin);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_paths_square_t(int n, const T *D, long long ldd, const T *Dt, long long ldt, const int *N,
                                         T *D2, int *N2, int *changed, cudaStream_t st) {
    const int tiles = (n + PBM - 1) / PBM;
    const int vec_a = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && ((ldd & 3) == 0);
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(paths_square_kernel<T>), PSMEM);
    if (e != cudaSuccess) return e;
    paths_square_kernel<T><<<tiles * tiles, PNT, PSMEM, st>>>(n, D, ldd, Dt, ldt, N, D2, N2, changed, vec_a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_paths_square(int n, const int *D, long long ldd, const int *Dt, long long ldt, const int *N,
                                int *D2, int *N2, int *changed, cudaStream_t st) {
    return launch_paths_square_t<int>(n, D, ldd, Dt, ldt, N, D2, N2, changed, st);
}

cudaError_t launch_paths_square_f32(int n, const float *D, long long ldd, const float *Dt, long long ldt,
                                    const int *N, float *D2, int *N2, int *changed, cudaStream_t st) {
    return launch_paths_square_t<float>(n, D, ldd, Dt, ldt, N, D2, N2, changed, st);
}

}  // namespace btas
