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
// CTA tile BM x BN x BK, TM x TN outputs per thread (8 x 8 for the product
// kernels, 4 x 4 for the small task tile of the persistent kernel), warps
// of 4 x 8 threads covering 4TM x 8TN outputs.  Thread (ty, tx) of warp
// (wm, wn) owns rows wm*4TM + 4*i + ty and columns wn*8TN + 8*j + tx: for
// every fragment load the warp reads 4 (A) or 8 (B) consecutive smem rows,
// and rows are padded to BK + 4 words, so every 128-bit load is a single
// conflict-free wavefront.
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
//   kF32Add2   two scalar RN adds + one 3-input min.f32 per k pair
//   kF32Scalar FADD + FMNMX per term (reference variant)
// All variants compute the same exact result: each term is one exact
// integer add or one round-to-nearest fp32 add, and min/max is independent
// of order.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "tgemm_args.h"

namespace btas {

// MINB: CTAs per SM the register budget is sized for (1: <= 255 registers,
// 2: <= 128).  FK: k depth of one register fragment (4 = 128-bit smem loads,
// 2 = 64-bit loads and half the fragment registers).
// UNR: unroll factor of the k-slice loop inside one smem stage.  TM x TN:
// outputs per thread.
template <int BM_, int BN_, int BK_, int STAGES_, int MINB_ = 1, int FK_ = 4, int UNR_ = 2, int TM_ = 8, int TN_ = 8>
struct TileCfg {
    static constexpr int BM = BM_, BN = BN_, BK = BK_, STAGES = STAGES_, MINB = MINB_, FK = FK_, UNR = UNR_;
    static constexpr int TM = TM_, TN = TN_;
    static constexpr int WARPS_M = BM / (4 * TM), WARPS_N = BN / (8 * TN);
    static constexpr int kThreads = WARPS_M * WARPS_N * 32;
    static constexpr int kLd = BK + 4;
    static constexpr int kStageElems = (BM + BN) * kLd;
    static constexpr int kSmemBytes = STAGES * kStageElems * 4;
    static_assert(BM % (4 * TM) == 0 && BN % (8 * TN) == 0 && BK % 8 == 0, "tile shape");
    static_assert(FK == 2 || FK == 4, "fragment depth");
};

template <typename T, int ROWS, int BK, int LD, int NT>
__device__ __forceinline__ void stage_rows(T *sm, const T *g, long long ldg, int row0, int rows_total,
                                           int k0, int K, bool vec, T fill, int tid, bool ro = false) {
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
        } else if (ro) {
            // asynchronous element copies: unaligned rows do not stall the pipeline
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (gr < rows_total && gk + e < K) cp_async4(dst + e, g + (long long)gr * ldg + gk + e);
                else dst[e] = fill;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T v = fill;
                if (gr < rows_total && gk + e < K) v = __ldcg(g + (long long)gr * ldg + gk + e);
                dst[e] = v;
            }
        }
    }
}

// Register fragments: for each of the TM rows (A) or TN columns (B) of a
// thread, FK consecutive k values.  Integer and scalar-fp32 variants view
// them as 32-bit words; the f32x2 variant as FK/2 64-bit pairs.
template <int FK>
struct Frag32 { uint32_t v[FK]; };
template <>
struct __align__(16) Frag32<4> { uint32_t v[4]; };
template <>
struct __align__(8) Frag32<2> { uint32_t v[2]; };

template <int FK>
__device__ __forceinline__ Frag32<FK> lds_frag(const void *p) {
    Frag32<FK> f;
    if constexpr (FK == 4) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        f.v[0] = t.x; f.v[1] = t.y; f.v[2] = t.z; f.v[3] = t.w;
    } else {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        f.v[0] = t.x; f.v[1] = t.y;
    }
    return f;
}

__device__ __forceinline__ uint64_t pack64(uint32_t lo, uint32_t hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
    return d;
}

// One FK-deep k slice of the TM x TN register tile.
template <int VAR, int SR, int NS, int FK, int TM, int TN>
struct Step;

template <int SR, int NS, int FK, int TM, int TN>
struct Step<kI32Dpx, SR, NS, FK, TM, TN> {
    static __device__ __forceinline__ void run(int (&acc)[TM][TN], const Frag32<FK> (&a)[TM],
                                               const Frag32<FK> (&b)[TN], int) {
#pragma unroll
        for (int q = 0; q < FK; ++q)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = iaddsel<SR>((int)a[i].v[q], (int)b[j].v[q], acc[i][j]);
    }
};

template <int SR, int NS, int FK, int TM, int TN>
struct Step<kI32Mix, SR, NS, FK, TM, TN> {
    static __device__ __forceinline__ void run(int (&acc)[TM][TN], const Frag32<FK> (&a)[TM],
                                               const Frag32<FK> (&b)[TN], int one) {
#pragma unroll
        for (int p = 0; p < FK / 2; ++p)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const int a0 = (int)a[i].v[2 * p], a1 = (int)a[i].v[2 * p + 1];
                    const int b0 = (int)b[j].v[2 * p], b1 = (int)b[j].v[2 * p + 1];
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

template <int SR, int NS, int FK, int TM, int TN>
struct Step<kF32X2, SR, NS, FK, TM, TN> {
    static __device__ __forceinline__ void run(float (&acc)[TM][TN], const Frag32<FK> (&a)[TM],
                                               const Frag32<FK> (&b)[TN], int) {
#pragma unroll
        for (int p = 0; p < FK / 2; ++p)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const uint64_t s = fadd2(pack64(a[i].v[2 * p], a[i].v[2 * p + 1]),
                                             pack64(b[j].v[2 * p], b[j].v[2 * p + 1]));
                    float lo, hi;
                    unpack2(s, lo, hi);
                    acc[i][j] = fsel3<SR>(acc[i][j], lo, hi);
                }
    }
};

// Two scalar RN adds + one 3-input min/max per k pair.
template <int SR, int NS, int FK, int TM, int TN>
struct Step<kF32Add2, SR, NS, FK, TM, TN> {
    static __device__ __forceinline__ void run(float (&acc)[TM][TN], const Frag32<FK> (&a)[TM],
                                               const Frag32<FK> (&b)[TN], int) {
#pragma unroll
        for (int p = 0; p < FK / 2; ++p)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const float s0 = __fadd_rn(__uint_as_float(a[i].v[2 * p]), __uint_as_float(b[j].v[2 * p]));
                    const float s1 = __fadd_rn(__uint_as_float(a[i].v[2 * p + 1]), __uint_as_float(b[j].v[2 * p + 1]));
                    acc[i][j] = fsel3<SR>(acc[i][j], s0, s1);
                }
    }
};

template <int SR, int NS, int FK, int TM, int TN>
struct Step<kF32Scalar, SR, NS, FK, TM, TN> {
    static __device__ __forceinline__ void run(float (&acc)[TM][TN], const Frag32<FK> (&a)[TM],
                                               const Frag32<FK> (&b)[TN], int) {
#pragma unroll
        for (int q = 0; q < FK; ++q)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    acc[i][j] = fsel2<SR>(acc[i][j], __fadd_rn(__uint_as_float(a[i].v[q]), __uint_as_float(b[j].v[q])));
    }
};

template <int VAR>
struct VarTypes { using T = float; };
template <>
struct VarTypes<kI32Dpx> { using T = int; };
template <>
struct VarTypes<kI32Mix> { using T = int; };

// Largest finite value of a min-plus output as an int (-1 for INF).  FP32
// outputs here are carriers of exact integers (APSP), so the cast is exact.
template <typename T>
__device__ __forceinline__ int finite_int(T v) {
    if constexpr (std::is_same<T, int>::value) return v < kInfI32 ? v : -1;
    else return v < __int_as_float(0x7f800000) ? static_cast<int>(v) : -1;
}

template <typename T, int SR>
__device__ __forceinline__ T finish(T v) {
    if constexpr (std::is_same<T, int>::value) return clamp_i32<SR>(v);
    else return v;
}

// Converged squaring (D_{s+1} = D_s): copy one BM x BN tile of P into C.
template <class Cfg, typename T>
__device__ __forceinline__ void copy_tile(const GemmArgs &args, int bm, int bn, int tid) {
    // Bit copy of the 4-byte tile prev -> C.  Each thread issues its loads in
    // batches of 8 (16-byte vectors where the pointers and pitches allow)
    // before storing, so several loads are in flight per thread.
    static_assert(sizeof(T) == 4, "4-byte elements");
    constexpr int BM = Cfg::BM, BN = Cfg::BN, NT = Cfg::kThreads;
    constexpr int Q = BN / 4;  // 4-element chunks per tile row
    static_assert((BM * Q) % NT == 0, "chunks divide evenly among the threads");
    constexpr int PER = BM * Q / NT;
    constexpr int BATCH = PER < 8 ? PER : 8;
    static_assert(PER % BATCH == 0, "whole batches");
    const uint32_t *P = static_cast<const uint32_t *>(args.prev);
    uint32_t *C = static_cast<uint32_t *>(args.C);
    const bool vec = ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(C)) & 15) == 0 &&
                     ((args.ldp | args.ldc) & 3) == 0;
#pragma unroll 1
    for (int b0 = 0; b0 < PER; b0 += BATCH) {
        uint4 v[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int q = tid + (b0 + u) * NT;
            const int r = bm + q / Q, c = bn + (q % Q) * 4;
            const uint32_t *src = P + (long long)r * args.ldp + c;
            if (vec && r < args.m && c + 4 <= args.n) {
                v[u] = __ldcg(reinterpret_cast<const uint4 *>(src));
            } else {
                const bool rr = r < args.m;
                v[u].x = rr && c < args.n ? __ldcg(src) : 0u;
                v[u].y = rr && c + 1 < args.n ? __ldcg(src + 1) : 0u;
                v[u].z = rr && c + 2 < args.n ? __ldcg(src + 2) : 0u;
                v[u].w = rr && c + 3 < args.n ? __ldcg(src + 3) : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int q = tid + (b0 + u) * NT;
            const int r = bm + q / Q, c = bn + (q % Q) * 4;
            if (r >= args.m) continue;
            uint32_t *dst = C + (long long)r * args.ldc + c;
            if (vec && c + 4 <= args.n) {
                *reinterpret_cast<uint4 *>(dst) = v[u];
            } else {
                if (c < args.n) dst[0] = v[u].x;
                if (c + 1 < args.n) dst[1] = v[u].y;
                if (c + 2 < args.n) dst[2] = v[u].z;
                if (c + 3 < args.n) dst[3] = v[u].w;
            }
        }
    }
}

// One BM x BN output tile at (bm, bn).  Returns this thread's "some output
// differs from prev" bit.  With Ct != nullptr the tile is also stored
// transposed (Ct[c][r], leading dimension ldct) through shared memory, so a
// following squaring finds its k-contiguous B operand ready.  With Cd / Cu
// (int32 only) it also stores the packed 16-bit operand forms: Cd = the value
// clamped to INF16 and duplicated into both halfwords, Cu = the clamped
// value (values are non-negative APSP distances here).  Loads of data
// that other CTAs of the same launch may have written go through L2
// (cp.async.cg, __ldcg), never through the non-coherent L1.
template <class Cfg, int VAR, int SR, int NS>
__device__ __forceinline__ bool nt_tile(const GemmArgs &args, int bm, int bn, unsigned char *smem_raw, int tid,
                                        void *Ct = nullptr, long long ldct = 0, uint32_t *Cd = nullptr,
                                        long long ldcd = 0, uint16_t *Cu = nullptr, long long ldcu = 0,
                                        bool k_backward = false) {
    using T = typename VarTypes<VAR>::T;
    constexpr int FK = Cfg::FK, TM = Cfg::TM, TN = Cfg::TN;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, LD = Cfg::kLd, ST = Cfg::STAGES;
    constexpr int NT = Cfg::kThreads;
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int M = args.m, N = args.n, K = args.k;
    const T *A = static_cast<const T *>(args.A);
    const T *Bt = static_cast<const T *>(args.Bt);
    T *C = static_cast<T *>(args.C);
    const T *P = static_cast<const T *>(args.prev);

    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp / Cfg::WARPS_N, wn = warp % Cfg::WARPS_N;
    const int ty = lane >> 3, tx = lane & 7;
    const int row_base = wm * (4 * TM) + ty;  // + 4*i
    const int col_base = wn * (8 * TN) + tx;  // + 8*j

    const T ident = Ident<T, SR>::v();
    const int KT = (K + BK - 1) / BK;
    const bool va = args.vec_a != 0, vb = args.vec_b != 0;
    auto load_stage = [&](int s, int kt) {
        T *sa = smem + s * Cfg::kStageElems;
        T *sb = sa + BM * LD;
        if (k_backward) kt = KT - 1 - kt;  // (+) is order-free: same result in either k order
        stage_rows<T, BM, BK, LD, NT>(sa, A, args.lda, bm, M, kt * BK, K, va, ident, tid, args.ro_a != 0);
        stage_rows<T, BN, BK, LD, NT>(sb, Bt, args.ldb, bn, N, kt * BK, K, vb, ident, tid, args.ro_b != 0);
    };

#pragma unroll
    for (int s = 0; s < ST - 1; ++s) {
        if (s < KT) load_stage(s, s);
        cp_async_commit();
    }

    // The accumulator (C with accumulate) is read after the first stages'
    // copies are issued, so the two latencies overlap (short-k accumulate
    // products, e.g. Floyd-Warshall's phase 3 at k = 128, pay them per tile).
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            T v = ident;
            if (args.accumulate) {
                const int r = bm + row_base + 4 * i, c = bn + col_base + 8 * j;
                if (r < M && c < N) v = __ldcg(C + (long long)r * args.ldc + c);
            }
            acc[i][j] = v;
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
#pragma unroll Cfg::UNR
        for (int kk = 0; kk < BK; kk += FK) {
            Frag32<FK> a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = lds_frag<FK>(sa + (row_base + 4 * i) * LD + kk);
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = lds_frag<FK>(sb + (col_base + 8 * j) * LD + kk);
            Step<VAR, SR, NS, FK, TM, TN>::run(acc, a, b, args.one);
        }
    }
    cp_async_wait<0>();

    bool ch = false;
    int mx = -1;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int r = bm + row_base + 4 * i, c = bn + col_base + 8 * j;
            acc[i][j] = finish<T, SR>(acc[i][j]);
            if (r < M && c < N) {
                const T v = acc[i][j];
                if (P != nullptr && v != __ldcg(P + (long long)r * args.ldp + c)) ch = true;
                if (SR == kMin && args.maxfin != nullptr) mx = max(mx, finite_int(v));
                C[(long long)r * args.ldc + c] = v;
                if constexpr (std::is_same<T, int>::value) {
                    if (Cd != nullptr) {
                        // 16-bit forms for a following packed squaring (used only
                        // when every finite entry is < 0x7FFF / 2, so exact)
                        const uint32_t u = v >= BTAS_INF_U16 ? BTAS_INF_U16 : (uint32_t)v;
                        Cd[(long long)r * ldcd + c] = u * 0x10001u;
                        Cu[(long long)r * ldcu + c] = (uint16_t)u;
                    }
                }
            }
        }
    if (SR == kMin && args.maxfin != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0 && mx >= 0) atomicMax(args.maxfin, mx);
    }
    if (Ct != nullptr) {
        // stage the tile transposed: tile[c][r], row pitch BM + 1 words
        static_assert(BN * (BM + 1) <= Cfg::STAGES * Cfg::kStageElems, "transpose staging fits");
        __syncthreads();  // every warp is done reading the last k stage
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) smem[(col_base + 8 * j) * (BM + 1) + row_base + 4 * i] = acc[i][j];
        __syncthreads();
        T *CT = static_cast<T *>(Ct);
        for (int idx = tid; idx < BM * BN; idx += NT) {
            const int c = idx / BM, r = idx % BM;
            if (bn + c < N && bm + r < M) CT[(long long)(bn + c) * ldct + bm + r] = smem[c * (BM + 1) + r];
        }
        __syncthreads();  // smem is reused by the caller's next tile
    }
    return ch;
}

// Grouped rasterisation: consecutive CTAs share A row panels and walk
// group_m tile rows before moving to the next column of tiles.
__device__ __forceinline__ void raster(int pid, int tiles_m, int tiles_n, int gm, int &tm, int &tn) {
    const int per_group = gm * tiles_n;
    const int g = pid / per_group;
    const int first_m = g * gm;
    const int gsz = min(tiles_m - first_m, gm);
    tm = first_m + (pid % per_group) % gsz;
    tn = (pid % per_group) / gsz;
}

template <class Cfg, int VAR, int SR, int NS>
__global__ void __launch_bounds__(Cfg::kThreads, Cfg::MINB) tgemm_nt_kernel(const GemmArgs args) {
    using T = typename VarTypes<VAR>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int tiles_m = (args.m + Cfg::BM - 1) / Cfg::BM, tiles_n = (args.n + Cfg::BN - 1) / Cfg::BN;
    int tm, tn;
    if (args.kwave > 0) raster(blockIdx.x, tiles_n, tiles_m, args.group_m, tn, tm);
    else raster(blockIdx.x, tiles_m, tiles_n, args.group_m, tm, tn);
    const int bm = tm * Cfg::BM, bn = tn * Cfg::BN;
    if (args.bypass != nullptr && __ldcg(args.bypass) != 0) return;
    if (args.skip != nullptr && __ldcg(args.skip) == 0) {
        copy_tile<Cfg, T>(args, bm, bn, tid);
        return;
    }
    const bool back = args.kwave > 0 && ((blockIdx.x / args.kwave) & 1) != 0;
    const bool ch = nt_tile<Cfg, VAR, SR, NS>(args, bm, bn, smem_raw, tid, nullptr, 0, nullptr, 0, nullptr, 0, back);
    if (args.changed != nullptr) {
        if (__any_sync(0xffffffffu, ch) && (tid & 31) == 0) atomicOr(args.changed, 1);
    }
}

}  // namespace btas
