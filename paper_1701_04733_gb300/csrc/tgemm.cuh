// Tropical matrix product C = A (x) B on sm_103a CUDA cores.
//
// Semiring product of the matrix-product listing in Sec. IV ("replace + by
// min and x by +"), for min-plus (Eq. 3-4) and max-plus (Eq. 1-2).  This is
// not a multiply-add contraction, so it runs on the integer/FP32 ALUs, not on
// the tensor cores.
//
// Layout ("NT"): A is m x k row-major, B is supplied TRANSPOSED as Bt (n x k
// row-major), so both operands are k-contiguous.  That lets one 128-bit
// shared-memory load bring four consecutive k values of a row into four
// consecutive registers, which the paired instructions below consume without
// register moves.
//
// CTA tile BM x BN x BK, 8 x 8 outputs per thread, warps of 4 x 8 threads
// covering 32 x 64 outputs.  Thread (ty, tx) of warp (wm, wn) owns rows
// wm*32 + 4*i + ty and columns wn*64 + 8*j + tx: for every fragment load the
// warp reads 4 (A) or 8 (B) consecutive smem rows, and rows are padded to
// BK + 4 words, so every 128-bit load is a single conflict-free wavefront.
// Tiles stream through a STAGES-deep cp.async ring (16-byte copies; edge
// chunks are filled element-wise with the semiring's absorbing value).
//
// Inner-loop variants (measured on GB300: the fused DPX add-min issues at 64
// lanes/SM/clock, as do FMNMX and IMAD; 3-input min/max does two
// reductions per issue):
//   kI32Dpx    one __viaddmin/__viaddmax_s32 per term (ALU pipe only)
//   kI32Mix    per k-pair and output: on NS of the 8 columns, two IMAD adds
//              (FMA pipe) + one 3-input min; DPX on the others, balancing the
//              ALU and FMA pipes
//   kF32X2     add.f32x2 (two RN adds, FMA pipe) + one 3-input min.f32
//   kF32Scalar FADD + FMNMX per term (reference variant)
// All variants compute the same exact result: each term is one exact
// integer add or one round-to-nearest fp32 add, and min/max is independent
// of order.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "tgemm_args.h"

namespace btas {

template <int BM_, int BN_, int BK_, int STAGES_>
struct TileCfg {
    static constexpr int BM = BM_, BN = BN_, BK = BK_, STAGES = STAGES_;
    static constexpr int WARPS_M = BM / 32, WARPS_N = BN / 64;
    static constexpr int kThreads = WARPS_M * WARPS_N * 32;
    static constexpr int kLd = BK + 4;
    static constexpr int kStageElems = (BM + BN) * kLd;
    static constexpr int kSmemBytes = STAGES * kStageElems * 4;
    static_assert(BM % 32 == 0 && BN % 64 == 0 && BK % 8 == 0, "tile shape");
};

template <typename T, int ROWS, int BK, int LD, int NT>
__device__ __forceinline__ void stage_rows(T *sm, const T *g, long long ldg, int row0, int rows_total,
                                           int k0, int K, bool vec, T fill, int tid) {
    constexpr int CPR = BK / 4;
    constexpr int CHUNKS = ROWS * CPR;
    static_assert(CHUNKS % NT == 0, "chunks per thread");
#pragma unroll
    for (int t = 0; t < CHUNKS / NT; ++t) {
        const int c = tid + t * NT;
        const int r = c / CPR, kc = (c % CPR) * 4;
        const int gr = row0 + r, gk = k0 + kc;
        T *dst = sm + r * LD + kc;
        if (vec && gr < rows_total && gk + 4 <= K) {
            cp_async16(dst, g + (long long)gr * ldg + gk);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T v = fill;
                if (gr < rows_total && gk + e < K) v = g[(long long)gr * ldg + gk + e];
                dst[e] = v;
            }
        }
    }
}

// One 4-deep k slice of the 8x8 register tile.
template <int VAR, int SR, int NS>
struct Step;

template <int SR, int NS>
struct Step<kI32Dpx, SR, NS> {
    static __device__ __forceinline__ void run(int (&acc)[8][8], const int4 (&a)[8], const int4 (&b)[8], int) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int av = q == 0 ? a[i].x : q == 1 ? a[i].y : q == 2 ? a[i].z : a[i].w;
                    const int bv = q == 0 ? b[j].x : q == 1 ? b[j].y : q == 2 ? b[j].z : b[j].w;
                    acc[i][j] = iaddsel<SR>(av, bv, acc[i][j]);
                }
    }
};

template <int SR, int NS>
struct Step<kI32Mix, SR, NS> {
    static __device__ __forceinline__ void run(int (&acc)[8][8], const int4 (&a)[8], const int4 (&b)[8], int one) {
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int a0 = p == 0 ? a[i].x : a[i].z, a1 = p == 0 ? a[i].y : a[i].w;
                    const int b0 = p == 0 ? b[j].x : b[j].z, b1 = p == 0 ? b[j].y : b[j].w;
                    if (j < NS) {
                        const int s0 = imad_add(a0, one, b0);
                        const int s1 = imad_add(a1, one, b1);
                        acc[i][j] = isel3<SR>(acc[i][j], s0, s1);
                    } else {
                        acc[i][j] = iaddsel<SR>(a1, b1, iaddsel<SR>(a0, b0, acc[i][j]));
                    }
                }
    }
};

template <int SR, int NS>
struct Step<kF32X2, SR, NS> {
    static __device__ __forceinline__ void run(float (&acc)[8][8], const ulonglong2 (&a)[8],
                                               const ulonglong2 (&b)[8], int) {
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint64_t s = fadd2(p == 0 ? a[i].x : a[i].y, p == 0 ? b[j].x : b[j].y);
                    float lo, hi;
                    unpack2(s, lo, hi);
                    acc[i][j] = fsel3<SR>(acc[i][j], lo, hi);
                }
    }
};

template <int SR, int NS>
struct Step<kF32Scalar, SR, NS> {
    static __device__ __forceinline__ void run(float (&acc)[8][8], const float4 (&a)[8], const float4 (&b)[8], int) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float av = q == 0 ? a[i].x : q == 1 ? a[i].y : q == 2 ? a[i].z : a[i].w;
                    const float bv = q == 0 ? b[j].x : q == 1 ? b[j].y : q == 2 ? b[j].z : b[j].w;
                    acc[i][j] = fsel2<SR>(acc[i][j], __fadd_rn(av, bv));
                }
    }
};

template <int VAR>
struct VarTypes;
template <>
struct VarTypes<kI32Dpx> { using T = int; using Frag = int4; };
template <>
struct VarTypes<kI32Mix> { using T = int; using Frag = int4; };
template <>
struct VarTypes<kF32X2> { using T = float; using Frag = ulonglong2; };
template <>
struct VarTypes<kF32Scalar> { using T = float; using Frag = float4; };

template <typename T, int SR>
__device__ __forceinline__ T finish(T v) {
    if constexpr (std::is_same<T, int>::value) return clamp_i32<SR>(v);
    else return v;
}

template <class Cfg, int VAR, int SR, int NS>
__global__ void __launch_bounds__(Cfg::kThreads, 1) tgemm_nt_kernel(const GemmArgs args) {
    using T = typename VarTypes<VAR>::T;
    using Frag = typename VarTypes<VAR>::Frag;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, LD = Cfg::kLd, ST = Cfg::STAGES;
    constexpr int NT = Cfg::kThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);

    const int M = args.m, N = args.n, K = args.k;
    const int tid = threadIdx.x;
    // grouped rasterisation: consecutive CTAs share A row panels and walk
    // group_m tile rows before moving to the next column of tiles
    const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
    const int gm = args.group_m;
    const int pid = blockIdx.x;
    const int per_group = gm * tiles_n;
    const int g = pid / per_group;
    const int first_m = g * gm;
    const int gsz = min(tiles_m - first_m, gm);
    const int tm = first_m + (pid % per_group) % gsz;
    const int tn = (pid % per_group) / gsz;
    const int bm = tm * BM, bn = tn * BN;

    const T *A = static_cast<const T *>(args.A);
    const T *Bt = static_cast<const T *>(args.Bt);
    T *C = static_cast<T *>(args.C);
    const T *P = static_cast<const T *>(args.prev);

    if (args.skip != nullptr && *args.skip == 0) {
        // converged squaring: D_{s+1} = D_s, copy the tile through
        for (int idx = tid; idx < BM * BN; idx += NT) {
            const int r = bm + idx / BN, c = bn + idx % BN;
            if (r < M && c < N) C[(long long)r * args.ldc + c] = P[(long long)r * args.ldp + c];
        }
        return;
    }

    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp / Cfg::WARPS_N, wn = warp % Cfg::WARPS_N;
    const int ty = lane >> 3, tx = lane & 7;
    const int row_base = wm * 32 + ty;  // + 4*i
    const int col_base = wn * 64 + tx;  // + 8*j

    const T ident = Ident<T, SR>::v();
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            T v = ident;
            if (args.accumulate) {
                const int r = bm + row_base + 4 * i, c = bn + col_base + 8 * j;
                if (r < M && c < N) v = C[(long long)r * args.ldc + c];
            }
            acc[i][j] = v;
        }

    const int KT = (K + BK - 1) / BK;
    const bool va = args.vec_a != 0, vb = args.vec_b != 0;
    auto load_stage = [&](int s, int kt) {
        T *sa = smem + s * Cfg::kStageElems;
        T *sb = sa + BM * LD;
        stage_rows<T, BM, BK, LD, NT>(sa, A, args.lda, bm, M, kt * BK, K, va, ident, tid);
        stage_rows<T, BN, BK, LD, NT>(sb, Bt, args.ldb, bn, N, kt * BK, K, vb, ident, tid);
    };

#pragma unroll
    for (int s = 0; s < ST - 1; ++s) {
        if (s < KT) load_stage(s, s);
        cp_async_commit();
    }

    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        {
            const int nk = kt + ST - 1;
            if (nk < KT) load_stage(nk % ST, nk);
            cp_async_commit();
        }
        const T *sa = smem + (kt % ST) * Cfg::kStageElems;
        const T *sb = sa + BM * LD;
#pragma unroll 2
        for (int kk = 0; kk < BK; kk += 4) {
            Frag a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a[i] = *reinterpret_cast<const Frag *>(sa + (row_base + 4 * i) * LD + kk);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                b[j] = *reinterpret_cast<const Frag *>(sb + (col_base + 8 * j) * LD + kk);
            Step<VAR, SR, NS>::run(acc, a, b, args.one);
        }
    }
    cp_async_wait<0>();

    bool ch = false;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = bm + row_base + 4 * i, c = bn + col_base + 8 * j;
            if (r < M && c < N) {
                const T v = finish<T, SR>(acc[i][j]);
                if (P != nullptr && v != P[(long long)r * args.ldp + c]) ch = true;
                C[(long long)r * args.ldc + c] = v;
            }
        }
    if (args.changed != nullptr) {
        if (__any_sync(0xffffffffu, ch) && lane == 0) atomicOr(args.changed, 1);
    }
}

}  // namespace btas
