// APSP with path reconstruction: repeated min-plus squaring (Sec. III) that
// also carries a next-hop (successor) matrix.
//
// One squaring: D'[i][j] = min_k D[i][k] + D[k][j]; k* = the SMALLEST k that
// attains the minimum; N'[i][j] = -1 if D'[i][j] is INF, N[i][j] if k* == i
// (the first leg is empty), else N[i][k*] (the first hop of the walk
// i -> k* -> j).  N_0[i][j] = j for an edge, i on the diagonal, -1 otherwise.
// With positive weights, following N from i reaches j along a shortest path.
//
// Argmin kernel: BM x BN output tile, TM x TN outputs per thread (warps of
// 4 x 8 threads, as in the product kernels), k staged through a cp.async
// ring (A = D rows, B = D^T rows, both k-contiguous).  k is taken in groups
// of 8: the running minimum absorbs the group's 8 terms (int32: DPX add-min,
// or, on NS of the TN columns, multiply-adds by a runtime one and 3-input
// mins, which moves the adds to the FMA pipe; binary32: two-lane
// round-to-nearest adds and 3-input mins), and
// when that lowers it the thread records the GROUP, one compare and one
// select per 8 terms.  Groups arrive in increasing k and only a strict
// decrease moves the record, so the recorded group is the first one that
// attains the final minimum.  The epilogue re-forms that group's 8 sums from
// D and D^T with the same rounding (so equality is exact) and takes the
// smallest k among them: the smallest minimising k overall.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tgemm.cuh"

namespace btas {

namespace {

constexpr int kGroup = 8;  // k per recorded group

// BK: k per shared-memory stage, ST: stages, MINB: CTAs per SM the registers
// are sized for, UNR: groups per unrolled step, NS: int32 columns on the FMA
// pipe.
template <int BM_, int BN_, int TM_, int TN_, int BK_, int ST_, int MINB_, int UNR_ = 1, int NS_ = 0>
struct ArgCfg {
    static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, BK = BK_, ST = ST_, MINB = MINB_, UNR = UNR_;
    static constexpr int NS = NS_;
    static constexpr int WARPS_M = BM / (4 * TM), WARPS_N = BN / (8 * TN);
    static constexpr int NT = WARPS_M * WARPS_N * 32;
    static constexpr int LD = BK + 4;  // padded row: conflict-free 128-bit fragment loads
    static constexpr int STAGE = (BM + BN) * LD;
    static constexpr int SMEM = ST * STAGE * 4;
    static_assert(BM % (4 * TM) == 0 && BN % (8 * TN) == 0 && BK % kGroup == 0, "tile shape");
};
// 64 x 64 tiles, 4 x 4 outputs per thread, two CTAs per SM, two groups per
// unrolled step; on 2 of the 4 columns the int32 form adds on the FMA pipe.
// Measured on GB300 against 128 x 128 (8 x 8 per thread, one CTA per SM),
// 128 x 64, 32 x 64 (four CTAs per SM), k depth 64 and 4 stages: those were
// 3-25 % slower, the DPX-only int32 form 3-9 % slower.
using ArgTile = ArgCfg<64, 64, 4, 4, 32, 3, 2, 2, 2>;

// Element type of the argmin squaring: int32 (one DPX add-min per term, INF
// absorbed by the clamp at INF - 2^28) or binary32 (one round-to-nearest add
// per term, +inf absorbing on its own).
template <typename T>
struct PathsElem;
template <>
struct PathsElem<int> {
    static __device__ __forceinline__ int start() { return 0x7FFFFFFF; }
    static __device__ __forceinline__ int inf() { return kInfI32; }
    static __device__ __forceinline__ int sum(int a, int b) { return a + b; }
    static __device__ __forceinline__ int finish(int v) { return v >= kClampI32 ? kInfI32 : v; }
    static __device__ __forceinline__ bool is_inf(int v) { return v == kInfI32; }
    // min(v, the 8 sums a[q] + b[q])
    static __device__ __forceinline__ int fold8(int v, const uint4 &a0, const uint4 &a1, const uint4 &b0,
                                                const uint4 &b1) {
        v = __viaddmin_s32((int)a0.x, (int)b0.x, v);
        v = __viaddmin_s32((int)a0.y, (int)b0.y, v);
        v = __viaddmin_s32((int)a0.z, (int)b0.z, v);
        v = __viaddmin_s32((int)a0.w, (int)b0.w, v);
        v = __viaddmin_s32((int)a1.x, (int)b1.x, v);
        v = __viaddmin_s32((int)a1.y, (int)b1.y, v);
        v = __viaddmin_s32((int)a1.z, (int)b1.z, v);
        v = __viaddmin_s32((int)a1.w, (int)b1.w, v);
        return v;
    }
    // The same minimum with the 8 adds as multiply-adds by a runtime one (FMA
    // pipe) and four 3-input mins (ALU pipe).
    static __device__ __forceinline__ int fold8_fma(int v, const uint4 &a0, const uint4 &a1, const uint4 &b0,
                                                    const uint4 &b1, int one) {
        v = __vimin3_s32(v, imad_add((int)a0.x, one, (int)b0.x), imad_add((int)a0.y, one, (int)b0.y));
        v = __vimin3_s32(v, imad_add((int)a0.z, one, (int)b0.z), imad_add((int)a0.w, one, (int)b0.w));
        v = __vimin3_s32(v, imad_add((int)a1.x, one, (int)b1.x), imad_add((int)a1.y, one, (int)b1.y));
        v = __vimin3_s32(v, imad_add((int)a1.z, one, (int)b1.z), imad_add((int)a1.w, one, (int)b1.w));
        return v;
    }
};
template <>
struct PathsElem<float> {
    static __device__ __forceinline__ float start() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float sum(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float finish(float v) { return v; }
    static __device__ __forceinline__ bool is_inf(float v) { return isinf(v); }
    static __device__ __forceinline__ float fold8(float v, const uint4 &a0, const uint4 &a1, const uint4 &b0,
                                                  const uint4 &b1) {
        float l, h;
        unpack2(fadd2(pack64(a0.x, a0.y), pack64(b0.x, b0.y)), l, h);
        v = fsel3<kMin>(v, l, h);
        unpack2(fadd2(pack64(a0.z, a0.w), pack64(b0.z, b0.w)), l, h);
        v = fsel3<kMin>(v, l, h);
        unpack2(fadd2(pack64(a1.x, a1.y), pack64(b1.x, b1.y)), l, h);
        v = fsel3<kMin>(v, l, h);
        unpack2(fadd2(pack64(a1.z, a1.w), pack64(b1.z, b1.w)), l, h);
        v = fsel3<kMin>(v, l, h);
        return v;
    }
    static __device__ __forceinline__ float fold8_fma(float v, const uint4 &a0, const uint4 &a1, const uint4 &b0,
                                                      const uint4 &b1, int) {
        return fold8(v, a0, a1, b0, b1);
    }
};

template <typename T>
__device__ __forceinline__ T as_elem(uint32_t u) {
    if constexpr (std::is_same<T, int>::value) return (int)u;
    else return __uint_as_float(u);
}

// The 8 values v[k0 .. k0+7] of one row (k >= n: never read, left at fill).
template <typename T>
__device__ __forceinline__ void load_group(const T *row, int k0, int n, bool vec, uint32_t (&v)[kGroup]) {
    if (vec && k0 + kGroup <= n) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(row + k0));
        const uint4 y = __ldg(reinterpret_cast<const uint4 *>(row + k0 + 4));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
        const uint32_t *r = reinterpret_cast<const uint32_t *>(row);
#pragma unroll
        for (int q = 0; q < kGroup; ++q) v[q] = k0 + q < n ? __ldg(r + k0 + q) : 0u;
    }
}

template <class Cfg, typename T>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
paths_square_kernel(int n, const T *__restrict__ D, long long ldd, const T *__restrict__ Dt, long long ldt,
                    const int *__restrict__ N, T *__restrict__ D2, int *__restrict__ N2, int *changed, int vec_a,
                    int one) {
    using E = PathsElem<T>;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, TM = Cfg::TM, TN = Cfg::TN, BK = Cfg::BK, LD = Cfg::LD;
    constexpr int ST = Cfg::ST, NT = Cfg::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x;
    int tm, tn;
    raster(blockIdx.x, (n + BM - 1) / BM, (n + BN - 1) / BN, 8, tm, tn);
    const int bm = tm * BM, bn = tn * BN;
    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp / Cfg::WARPS_N, wn = warp % Cfg::WARPS_N;
    const int row_base = wm * (4 * TM) + (lane >> 3);  // + 4*i
    const int col_base = wn * (8 * TN) + (lane & 7);   // + 8*j
    T val[TM][TN];
    int grp[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            val[i][j] = E::start();
            grp[i][j] = -1;
        }
    const int KT = (n + BK - 1) / BK;
    auto load = [&](int s, int kt) {
        T *sa = smem + s * Cfg::STAGE;
        T *sb = sa + BM * LD;
        stage_rows<T, BM, BK, LD, NT>(sa, D, ldd, bm, n, kt * BK, n, vec_a != 0, E::inf(), tid, true);
        stage_rows<T, BN, BK, LD, NT>(sb, Dt, ldt, bn, n, kt * BK, n, true, E::inf(), tid, true);
    };
#pragma unroll
    for (int s = 0; s < ST - 1; ++s) {
        if (s < KT) load(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        if (kt + ST - 1 < KT) load((kt + ST - 1) % ST, kt + ST - 1);
        cp_async_commit();
        const T *sa = smem + (kt % ST) * Cfg::STAGE;
        const T *sb = sa + BM * LD;
#pragma unroll Cfg::UNR
        for (int kk = 0; kk < BK; kk += kGroup) {
            const int g = (kt * BK + kk) / kGroup;
            uint4 b0[TN], b1[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const T *p = sb + (col_base + 8 * j) * LD + kk;
                b0[j] = *reinterpret_cast<const uint4 *>(p);
                b1[j] = *reinterpret_cast<const uint4 *>(p + 4);
            }
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const T *p = sa + (row_base + 4 * i) * LD + kk;
                const uint4 a0 = *reinterpret_cast<const uint4 *>(p);
                const uint4 a1 = *reinterpret_cast<const uint4 *>(p + 4);
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const T v = j < Cfg::NS ? E::fold8_fma(val[i][j], a0, a1, b0[j], b1[j], one)
                                            : E::fold8(val[i][j], a0, a1, b0[j], b1[j]);
                    grp[i][j] = v < val[i][j] ? g : grp[i][j];
                    val[i][j] = v;
                }
            }
        }
    }
    cp_async_wait<0>();

    // Epilogue: the smallest k of the recorded group whose sum equals the
    // minimum, then N'[r][c] = -1 (INF), N[r][c] (k == r) or N[r][k].
    const bool vec_d = vec_a != 0;
    bool ch = false;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = bm + row_base + 4 * i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = bn + col_base + 8 * j;
            if (c >= n) continue;
            const T raw = val[i][j];
            const T d = E::finish(raw);
            int nx = -1;
            if (!E::is_inf(d)) {
                const int k0 = max(grp[i][j], 0) * kGroup;
                uint32_t x[kGroup], y[kGroup];
                load_group<T>(D + (long long)r * ldd, k0, n, vec_d, x);
                load_group<T>(Dt + (long long)c * ldt, k0, n, true, y);
                int k = k0;
#pragma unroll
                for (int q = kGroup - 1; q >= 0; --q)
                    if (k0 + q < n && E::sum(as_elem<T>(x[q]), as_elem<T>(y[q])) == raw) k = k0 + q;
                nx = N[(long long)r * n + (k == r ? c : k)];
            }
            if (d != D[(long long)r * ldd + c] || nx != N[(long long)r * n + c]) ch = true;
            D2[(long long)r * n + c] = d;
            N2[(long long)r * n + c] = nx;
        }
    }
    if (__any_sync(0xffffffffu, ch) && lane == 0) atomicOr(changed, 1);
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
    using Cfg = ArgTile;
    if (n <= 0) return cudaSuccess;
    const int vec_a = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && ((ldd & 3) == 0);
    const int tiles = ((n + Cfg::BM - 1) / Cfg::BM) * ((n + Cfg::BN - 1) / Cfg::BN);
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(paths_square_kernel<Cfg, T>), Cfg::SMEM);
    if (e != cudaSuccess) return e;
    paths_square_kernel<Cfg, T><<<tiles, Cfg::NT, Cfg::SMEM, st>>>(n, D, ldd, Dt, ldt, N, D2, N2, changed,
                                                                          vec_a, 1);
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
