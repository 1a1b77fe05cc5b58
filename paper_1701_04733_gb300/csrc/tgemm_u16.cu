// Exact packed 16-bit min-plus product: two outputs per 32-bit lane.
//
// Values live in [0, 0x7FFF] with INF16 = 0x7FFF.  Output pair
// (C[i][j], C[i][j+1]) sits in one 32-bit register; the A value A[i][l] is
// duplicated into both halfwords (a pre-pass writes A as 32-bit words
// A[i][l] * 0x10001), and (B[l][j], B[l][j+1]) is already adjacent in
// row-major B.  Because every operand is <= 0x7FFF, a halfword sum is at most
// 0xFFFE: a plain 32-bit add of two packed words never carries between the
// halves, and the unsigned per-halfword min never sees a wrapped value.  The
// accumulator starts at INF16 in both halves, so every result is
// min(INF16, exact minimum) -- the saturating semantics of the 16-bit
// encoding.  For APSP with (n-1) * max w < 0x7FFF every distance is below
// INF16, so the result equals the int32 computation (Sec. III squaring).
//
// Tile: BM = 128 rows x 128 column pairs (256 columns) x BK = 32, 256
// threads, 8 rows x 8 pairs per thread.  A (duplicated) is staged k-contiguous
// with padded rows like the int32 kernel; B is staged as 32 rows of 128 packed
// words.  A thread owns pairs tx*4 + {0..3} + 32*h (h = 0..3 over the two
// warp columns), so each B fragment load is a conflict-free 128-bit load.
// Inner loop: on NS of the 8 pairs, two 32-bit IMAD adds (FMA pipe) + one
// 3-input per-halfword min; DPX __viaddmin_u16x2 on the others.
#include <cstdint>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"

namespace btas {

namespace u16 {
constexpr int BM = 128, BNP = 128, BK = 32, ST = 3, NT = 256;
constexpr int LDA = BK + 4;          // words per A smem row
constexpr int LDB = BNP;             // words per B smem row (reads are row-contiguous)
constexpr int A_ELEMS = BM * LDA;
constexpr int B_ELEMS = BK * LDB;
constexpr int STAGE = A_ELEMS + B_ELEMS;
constexpr int SMEM = ST * STAGE * 4;
}  // namespace u16

struct U16KArgs {
    int m, n, k;
    const uint32_t *Ad;  // m x k duplicated words
    long long ldad;
    const uint16_t *B;
    long long ldb;
    uint16_t *C;
    long long ldc;
    const uint16_t *prev;
    long long ldp;
    int *changed;
    const int *skip;
    int one;
    int vec_a, vec_b;
    int *maxfin;
    const int *gate;  // optional: *gate == 0 => do nothing
    int *Ci;          // optional: accumulate into int32 Ci = min(Ci, widened result) instead of writing C
    long long ldci;
    int xr0, xr1, xc0, xc1;  // rows / columns of Ci not to write (another stream owns them)
    // > 0: rasterise by groups of kgroup tile COLUMNS (rows fastest, so consecutive
    // waves share their B panels) and run k backwards in every other wave of kwave
    // CTAs: a wave then starts on the k-slices the previous one left in L2
    int kwave;
    int kgroup;
};

__global__ void dup_u16_kernel(const uint16_t *__restrict__ A, long long lda, int m, int k, uint32_t *__restrict__ Ad,
                               long long ldad, const int *skip) {
    if (skip != nullptr && *skip == 0) return;
    const long long total = (long long)m * k;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long r = idx / k, c = idx % k;
        Ad[r * ldad + c] = 0x10001u * A[r * lda + c];
    }
}

__global__ void narrow_u16_kernel(const int *__restrict__ src, long long total, uint16_t *__restrict__ dst) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int v = src[idx];
        dst[idx] = (uint16_t)(v >= BTAS_INF_U16 ? BTAS_INF_U16 : v);
    }
}

__global__ void widen_u16_i32_kernel(const uint16_t *__restrict__ src, long long total, int *__restrict__ dst) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int v = src[idx];
        dst[idx] = v >= BTAS_INF_U16 ? kInfI32 : v;
    }
}

template <int NS>
__global__ void __launch_bounds__(u16::NT, 1) tgemm_u16_kernel(const U16KArgs args) {
    using namespace u16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *smem = reinterpret_cast<uint32_t *>(smem_raw);
    const int M = args.m, N = args.n, K = args.k;
    const int NP = (N + 1) / 2;  // column pairs
    const int tid = threadIdx.x;
    const int tiles_m = (M + BM - 1) / BM, tiles_n = (NP + BNP - 1) / BNP;
    const int pid = blockIdx.x;
    int tm, tn;
    if (args.kwave > 0) {
        // groups of kgroup tile columns, rows fastest: consecutive waves share B panels
        const int GN = args.kgroup;
        const int per_group = GN * tiles_m;
        const int g = pid / per_group;
        const int first_n = g * GN;
        const int gsz = min(tiles_n - first_n, GN);
        tn = first_n + (pid % per_group) % gsz;
        tm = (pid % per_group) / gsz;
    } else {
        constexpr int GM = 8;
        const int per_group = GM * tiles_n;
        const int g = pid / per_group;
        const int first_m = g * GM;
        const int gsz = min(tiles_m - first_m, GM);
        tm = first_m + (pid % per_group) % gsz;
        tn = (pid % per_group) / gsz;
    }
    const int bm = tm * BM, bnp = tn * BNP;  // bnp in pairs; column = 2*pair
    const bool k_back = args.kwave > 0 && ((pid / args.kwave) & 1) != 0;

    if (args.gate != nullptr && __ldcg(args.gate) == 0) return;
    if (args.Ci != nullptr) {
        // Pull this CTA's tile of Ci into L2 while its products run: the
        // min-accumulate epilogue then reads it from L2.  With a short k (128
        // in blocked Floyd-Warshall) that read is a third of the kernel time
        // otherwise, since one CTA per SM leaves nothing to overlap it with.
        for (int l = tid; l < BM * 8; l += NT) {  // 8 lines of 32 words per tile row
            const int r = bm + (l >> 3), c = 2 * bnp + (l & 7) * 32;
            if (r < M && c < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(args.Ci + (long long)r * args.ldci + c));
        }
    }
    if (args.skip != nullptr && *args.skip == 0) {
        for (int idx = tid; idx < BM * BNP * 2; idx += NT) {
            const int r = bm + idx / (BNP * 2), c = 2 * bnp + idx % (BNP * 2);
            if (r < M && c < N) args.C[(long long)r * args.ldc + c] = args.prev[(long long)r * args.ldp + c];
        }
        return;
    }

    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int ty = lane >> 3, tx = lane & 7;
    const int row_base = wm * 32 + ty;       // + 4*i
    const int pair_base = wn * 64 + tx * 4;  // + 32*h + q, h in {0,1}, q in 0..3

    uint32_t acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = kInfU16x2;

    const int KT = (K + BK - 1) / BK;
    auto load_stage = [&](int s, int kt) {
        uint32_t *sa = smem + s * STAGE;
        uint32_t *sb = sa + A_ELEMS;
        const int k0 = (k_back ? KT - 1 - kt : kt) * BK;  // min is order-free
        // A: BM rows x BK words, 8 chunks per row
#pragma unroll
        for (int t = 0; t < (BM * BK / 4) / NT; ++t) {
            const int c = tid + t * NT;
            const int r = c >> 3, kc = (c & 7) * 4;
            const int gr = bm + r, gk = k0 + kc;
            uint32_t *dst = sa + r * LDA + kc;
            if (args.vec_a && gr < M && gk + 4 <= K) {
                cp_async16(dst, args.Ad + (long long)gr * args.ldad + gk);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    dst[e] = (gr < M && gk + e < K) ? args.Ad[(long long)gr * args.ldad + gk + e] : kInfU16x2;
            }
        }
        // B: BK rows x BNP words (2*BNP u16), 32 chunks of 8 u16 per row
#pragma unroll
        for (int t = 0; t < (BK * BNP / 4) / NT; ++t) {
            const int c = tid + t * NT;
            const int r = c >> 5, wc = (c & 31) * 4;  // word column within tile
            const int gk = k0 + r, gcol = 2 * (bnp + wc);
            uint32_t *dst = sb + r * LDB + wc;
            if (args.vec_b && gk < K && gcol + 8 <= N) {
                cp_async16(dst, args.B + (long long)gk * args.ldb + gcol);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c0 = gcol + 2 * e;
                    uint32_t lo = BTAS_INF_U16, hi = BTAS_INF_U16;
                    if (gk < K) {
                        if (c0 < N) lo = args.B[(long long)gk * args.ldb + c0];
                        if (c0 + 1 < N) hi = args.B[(long long)gk * args.ldb + c0 + 1];
                    }
                    dst[e] = lo | (hi << 16);
                }
            }
        }
    };

#pragma unroll
    for (int s = 0; s < ST - 1; ++s) {
        if (s < KT) load_stage(s, s);
        cp_async_commit();
    }
    const int one = args.one;
    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        {
            const int nk = kt + ST - 1;
            if (nk < KT) load_stage(nk % ST, nk);
            cp_async_commit();
        }
        const uint32_t *sa = smem + (kt % ST) * STAGE;
        const uint32_t *sb = sa + A_ELEMS;
#pragma unroll 2
        for (int kk = 0; kk < BK; kk += 4) {
            uint4 a[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = *reinterpret_cast<const uint4 *>(sa + (row_base + 4 * i) * LDA + kk);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                uint4 b0[2], b1[2];  // k = kk+2p and kk+2p+1, pairs h*32 + 0..3
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    b0[h] = *reinterpret_cast<const uint4 *>(sb + (kk + 2 * p) * LDB + pair_base + 32 * h);
                    b1[h] = *reinterpret_cast<const uint4 *>(sb + (kk + 2 * p + 1) * LDB + pair_base + 32 * h);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t a0 = p == 0 ? a[i].x : a[i].z, a1 = p == 0 ? a[i].y : a[i].w;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int h = j >> 2, q = j & 3;
                        const uint32_t bb0 = q == 0 ? b0[h].x : q == 1 ? b0[h].y : q == 2 ? b0[h].z : b0[h].w;
                        const uint32_t bb1 = q == 0 ? b1[h].x : q == 1 ? b1[h].y : q == 2 ? b1[h].z : b1[h].w;
                        if (j < NS) {
                            const uint32_t s0 = (uint32_t)imad_add((int)a0, one, (int)bb0);
                            const uint32_t s1 = (uint32_t)imad_add((int)a1, one, (int)bb1);
                            acc[i][j] = u16x2_min3(acc[i][j], s0, s1);
                        } else {
                            acc[i][j] = u16x2_addmin(a1, bb1, u16x2_addmin(a0, bb0, acc[i][j]));
                        }
                    }
                }
            }
        }
    }
    cp_async_wait<0>();

    bool ch = false;
    int mx = -1;
    if (args.Ci != nullptr) {
        // int32 accumulate: Ci = min(Ci, result), INF16 read as INF.  Each
        // thread's 8 columns per half (h) are consecutive, so rows are read
        // and written as 16-byte vectors, two rows' loads in flight at once.
        const bool vec = ((reinterpret_cast<uintptr_t>(args.Ci) & 15) == 0) && ((args.ldci & 3) == 0);
#pragma unroll
        for (int i0 = 0; i0 < 8; i0 += 2) {
            int4 old[2][2][2];  // [row][h][vector]
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const int r = bm + row_base + 4 * (i0 + ii);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = 2 * (bnp + pair_base + 32 * h);
                    const int *pc = args.Ci + (long long)r * args.ldci + c0;
                    if (vec && r < M && c0 + 8 <= N) {
                        old[ii][h][0] = *reinterpret_cast<const int4 *>(pc);
                        old[ii][h][1] = *reinterpret_cast<const int4 *>(pc + 4);
                    } else {
                        int t[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) t[e] = (r < M && c0 + e < N) ? pc[e] : kInfI32;
                        old[ii][h][0] = make_int4(t[0], t[1], t[2], t[3]);
                        old[ii][h][1] = make_int4(t[4], t[5], t[6], t[7]);
                    }
                }
            }
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const int i = i0 + ii;
                const int r = bm + row_base + 4 * i;
                if (r >= M || (r >= args.xr0 && r < args.xr1)) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = 2 * (bnp + pair_base + 32 * h);
                    int v[8] = {old[ii][h][0].x, old[ii][h][0].y, old[ii][h][0].z, old[ii][h][0].w,
                                old[ii][h][1].x, old[ii][h][1].y, old[ii][h][1].z, old[ii][h][1].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t w = acc[i][4 * h + q];
                        const uint32_t lo = w & 0xFFFFu, hi = w >> 16;
                        if (lo < BTAS_INF_U16) v[2 * q] = min(v[2 * q], (int)lo);
                        if (hi < BTAS_INF_U16) v[2 * q + 1] = min(v[2 * q + 1], (int)hi);
                    }
                    int *pc = args.Ci + (long long)r * args.ldci + c0;
                    const bool clear = c0 + 8 <= args.xc0 || c0 >= args.xc1;  // none of the 8 excluded
                    if (vec && c0 + 8 <= N && clear) {
                        *reinterpret_cast<int4 *>(pc) = make_int4(v[0], v[1], v[2], v[3]);
                        *reinterpret_cast<int4 *>(pc + 4) = make_int4(v[4], v[5], v[6], v[7]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (c0 + e < N && (c0 + e < args.xc0 || c0 + e >= args.xc1)) pc[e] = v[e];
                    }
                }
            }
        }
        return;
    }
    // Each thread's 8 columns per half (h) are consecutive: 16 bytes of C and
    // of prev.  Where aligned and inside the matrix, prev is read and C
    // written as 16-byte vectors, with both halves of two rows read before
    // any store; elsewhere element by element.
    const bool vec_c = ((reinterpret_cast<uintptr_t>(args.C) & 15) == 0) && ((args.ldc & 7) == 0) &&
                       (args.prev == nullptr ||
                        (((reinterpret_cast<uintptr_t>(args.prev) & 15) == 0) && ((args.ldp & 7) == 0)));
#pragma unroll
    for (int i0 = 0; i0 < 8; i0 += 2) {
        uint4 pv[2][2];
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {
            const int r = bm + row_base + 4 * (i0 + ii);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c0 = 2 * (bnp + pair_base + 32 * h);
                pv[ii][h] = make_uint4(0, 0, 0, 0);
                if (args.prev && vec_c && r < M && c0 + 8 <= N)
                    pv[ii][h] = *reinterpret_cast<const uint4 *>(args.prev + (long long)r * args.ldp + c0);
            }
        }
#pragma unroll
        for (int ii = 0; ii < 2; ++ii) {
            const int i = i0 + ii;
            const int r = bm + row_base + 4 * i;
            if (r >= M) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c0 = 2 * (bnp + pair_base + 32 * h);
                if (vec_c && c0 + 8 <= N) {
                    const uint4 w = make_uint4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
                    if (args.prev)
                        ch |= (w.x != pv[ii][h].x) | (w.y != pv[ii][h].y) | (w.z != pv[ii][h].z) | (w.w != pv[ii][h].w);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t lo = acc[i][4 * h + q] & 0xFFFFu, hi = acc[i][4 * h + q] >> 16;
                        if (lo < BTAS_INF_U16) mx = max(mx, (int)lo);
                        if (hi < BTAS_INF_U16) mx = max(mx, (int)hi);
                    }
                    *reinterpret_cast<uint4 *>(args.C + (long long)r * args.ldc + c0) = w;
                    continue;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + 2 * q;
                    const uint32_t v = acc[i][4 * h + q];
                    const uint16_t lo = (uint16_t)(v & 0xFFFF), hi = (uint16_t)(v >> 16);
                    if (c < N) {
                        if (args.prev && lo != args.prev[(long long)r * args.ldp + c]) ch = true;
                        if (lo < BTAS_INF_U16) mx = max(mx, (int)lo);
                        args.C[(long long)r * args.ldc + c] = lo;
                    }
                    if (c + 1 < N) {
                        if (args.prev && hi != args.prev[(long long)r * args.ldp + c + 1]) ch = true;
                        if (hi < BTAS_INF_U16) mx = max(mx, (int)hi);
                        args.C[(long long)r * args.ldc + c + 1] = hi;
                    }
                }
            }
        }
    }
    if (args.maxfin != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx >= 0) atomicMax(args.maxfin, mx);
    }
    if (args.changed != nullptr) {
        if (__any_sync(0xffffffffu, ch) && lane == 0) atomicOr(args.changed, 1);
    }
}


// Floyd-Warshall's packed phase 3 (Ci accumulate at k = 128) at 2 CTAs per
// SM: 128 x 128 tiles (64 column pairs), 8 rows x 4 pairs per thread, DPX
// add-min on every term.  With k / BK = 4 slices per tile, the prologue and
// the accumulate epilogue of one CTA overlap the other CTA's products, which
// the 1-CTA/SM kernel above cannot do.
namespace u16c2 {
constexpr int BM = 128, BNP = 64, BK = 32, ST = 3, NT = 256, RI = 8, PQ = 4;
constexpr int LDA = BK + 4, LDB = BNP;
constexpr int STAGE = BM * LDA + BK * LDB;
constexpr int SMEM = ST * STAGE * 4;  // 79872 bytes
}  // namespace u16c2

__global__ void __launch_bounds__(u16c2::NT, 2) tgemm_u16_ci2_kernel(const U16KArgs args) {
    using namespace u16c2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *smem = reinterpret_cast<uint32_t *>(smem_raw);
    const int M = args.m, N = args.n, K = args.k;
    const int NP = (N + 1) / 2;
    const int tid = threadIdx.x;
    const int tiles_m = (M + BM - 1) / BM, tiles_n = (NP + BNP - 1) / BNP;
    const int pid = blockIdx.x;
    constexpr int GM = 8;
    const int per_group = GM * tiles_n;
    const int g = pid / per_group;
    const int first_m = g * GM;
    const int gsz = min(tiles_m - first_m, GM);
    const int bm = (first_m + (pid % per_group) % gsz) * BM;
    const int bnp = ((pid % per_group) / gsz) * BNP;  // first column pair
    if (args.gate != nullptr && __ldcg(args.gate) == 0) return;
    // this tile of Ci into L2 while its products run (the epilogue reads it)
    for (int l = tid; l < BM * 4; l += NT) {  // 4 lines of 32 words per tile row
        const int r = bm + (l >> 2), c = 2 * bnp + (l & 3) * 32;
        if (r < M && c < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(args.Ci + (long long)r * args.ldci + c));
    }
    const int warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;
    const int ty = lane >> 3, tx = lane & 7;
    const int row_base = wm * (4 * RI) + ty;        // + 4*i
    const int pair_base = wn * (8 * PQ) + tx * PQ;  // + q
    uint32_t acc[RI][PQ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < PQ; ++j) acc[i][j] = kInfU16x2;
    const int KT = (K + BK - 1) / BK;
    auto load = [&](int s, int kt) {
        uint32_t *sa = smem + s * STAGE;
        uint32_t *sb = sa + BM * LDA;
        const int k0 = kt * BK;
#pragma unroll
        for (int t = 0; t < (BM * BK / 4) / NT; ++t) {
            const int c = tid + t * NT;
            const int r = c >> 3, kc = (c & 7) * 4;
            const int gr = bm + r, gk = k0 + kc;
            uint32_t *dst = sa + r * LDA + kc;
            if (args.vec_a && gr < M && gk + 4 <= K) {
                cp_async16(dst, args.Ad + (long long)gr * args.ldad + gk);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    dst[e] = (gr < M && gk + e < K) ? args.Ad[(long long)gr * args.ldad + gk + e] : kInfU16x2;
            }
        }
        constexpr int CPR = BNP / 4;  // chunks of 4 words per B row
#pragma unroll
        for (int t = 0; t < (BK * BNP / 4) / NT; ++t) {
            const int c = tid + t * NT;
            const int r = c / CPR, wc = (c % CPR) * 4;
            const int gk = k0 + r, gcol = 2 * (bnp + wc);
            uint32_t *dst = sb + r * LDB + wc;
            if (args.vec_b && gk < K && gcol + 8 <= N) {
                cp_async16(dst, args.B + (long long)gk * args.ldb + gcol);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c0 = gcol + 2 * e;
                    uint32_t lo = BTAS_INF_U16, hi = BTAS_INF_U16;
                    if (gk < K) {
                        if (c0 < N) lo = args.B[(long long)gk * args.ldb + c0];
                        if (c0 + 1 < N) hi = args.B[(long long)gk * args.ldb + c0 + 1];
                    }
                    dst[e] = lo | (hi << 16);
                }
            }
        }
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
        const uint32_t *sa = smem + (kt % ST) * STAGE;
        const uint32_t *sb = sa + BM * LDA;
#pragma unroll 2
        for (int kk = 0; kk < BK; kk += 4) {
            uint4 av[RI];
#pragma unroll
            for (int i = 0; i < RI; ++i) av[i] = *reinterpret_cast<const uint4 *>(sa + (row_base + 4 * i) * LDA + kk);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 t = *reinterpret_cast<const uint4 *>(sb + (kk + q) * LDB + pair_base);
                const uint32_t b[PQ] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const uint32_t ai = q == 0 ? av[i].x : q == 1 ? av[i].y : q == 2 ? av[i].z : av[i].w;
#pragma unroll
                    for (int j = 0; j < PQ; ++j) acc[i][j] = u16x2_addmin(ai, b[j], acc[i][j]);
                }
            }
        }
    }
    cp_async_wait<0>();
    // Ci = min(Ci, result), INF16 read as INF; rows [xr0, xr1) and columns
    // [xc0, xc1) left alone.  This thread's 8 columns are consecutive: rows
    // are read and written as 16-byte vectors, four rows' loads in flight
    // before any store.
    const int c0 = 2 * (bnp + pair_base);
    const bool vec = ((reinterpret_cast<uintptr_t>(args.Ci) & 15) == 0) && ((args.ldci & 3) == 0);
#pragma unroll
    for (int i0 = 0; i0 < RI; i0 += 4) {
        int4 old[4][2];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int r = bm + row_base + 4 * (i0 + ii);
            const int *pc = args.Ci + (long long)r * args.ldci + c0;
            if (vec && r < M && c0 + 8 <= N) {
                old[ii][0] = *reinterpret_cast<const int4 *>(pc);
                old[ii][1] = *reinterpret_cast<const int4 *>(pc + 4);
            } else {
                int t[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) t[e] = (r < M && c0 + e < N) ? pc[e] : kInfI32;
                old[ii][0] = make_int4(t[0], t[1], t[2], t[3]);
                old[ii][1] = make_int4(t[4], t[5], t[6], t[7]);
            }
        }
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int i = i0 + ii;
            const int r = bm + row_base + 4 * i;
            if (r >= M || (r >= args.xr0 && r < args.xr1)) continue;
            int v[8] = {old[ii][0].x, old[ii][0].y, old[ii][0].z, old[ii][0].w,
                        old[ii][1].x, old[ii][1].y, old[ii][1].z, old[ii][1].w};
#pragma unroll
            for (int q = 0; q < PQ; ++q) {
                const uint32_t w = acc[i][q];
                const uint32_t lo = w & 0xFFFFu, hi = w >> 16;
                if (lo < BTAS_INF_U16) v[2 * q] = min(v[2 * q], (int)lo);
                if (hi < BTAS_INF_U16) v[2 * q + 1] = min(v[2 * q + 1], (int)hi);
            }
            int *pc = args.Ci + (long long)r * args.ldci + c0;
            const bool clear = c0 + 8 <= args.xc0 || c0 >= args.xc1;  // none of the 8 excluded
            if (vec && c0 + 8 <= N && clear) {
                *reinterpret_cast<int4 *>(pc) = make_int4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<int4 *>(pc + 4) = make_int4(v[4], v[5], v[6], v[7]);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (c0 + e < N && (c0 + e < args.xc0 || c0 + e >= args.xc1)) pc[e] = v[e];
            }
        }
    }
}

static int grid_for(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

cudaError_t launch_narrow_u16(const int *src, long long total, uint16_t *dst, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    narrow_u16_kernel<<<grid_for(total), 256, 0, st>>>(src, total, dst);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_widen_u16_i32(const uint16_t *src, long long total, int *dst, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    widen_u16_i32_kernel<<<grid_for(total), 256, 0, st>>>(src, total, dst);
    note_launch();
    return cudaGetLastError();
}

template <int NS>
static cudaError_t launch_ns(const U16KArgs &ka, cudaStream_t st) {
    const char *one = getenv("BTAS_U16_CI_1CTA");
    if (ka.Ci != nullptr && ka.skip == nullptr && ka.prev == nullptr && ka.maxfin == nullptr && ka.changed == nullptr &&
        !(one && *one == '1')) {
        cudaError_t e = set_smem_once(reinterpret_cast<const void *>(tgemm_u16_ci2_kernel), u16c2::SMEM);
        if (e != cudaSuccess) return e;
        const long long tiles =
            (long long)((ka.m + u16c2::BM - 1) / u16c2::BM) * (((ka.n + 1) / 2 + u16c2::BNP - 1) / u16c2::BNP);
        tgemm_u16_ci2_kernel<<<(unsigned)tiles, u16c2::NT, u16c2::SMEM, st>>>(ka);
        note_launch();
        return cudaGetLastError();
    }
    auto kern = tgemm_u16_kernel<NS>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(kern), u16::SMEM);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((ka.m + u16::BM - 1) / u16::BM) * (((ka.n + 1) / 2 + u16::BNP - 1) / u16::BNP);
    kern<<<(unsigned)tiles, u16::NT, u16::SMEM, st>>>(ka);
    note_launch();
    return cudaGetLastError();
}

// Runs the duplication pre-pass into `adup` (m x round4(k) words, caller
// workspace) and the packed product.  ns selects the IMAD/DPX split.
cudaError_t launch_tgemm_u16_ws(const U16Args &a, uint32_t *adup, int ns, cudaStream_t st) {
    const long long ldad = (a.k + 3) & ~3LL;
    if (!a.adup_ready) {
        dup_u16_kernel<<<grid_for((long long)a.m * a.k), 256, 0, st>>>(a.A, a.lda, a.m, a.k, adup, ldad, a.skip);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    U16KArgs ka{};
    ka.m = a.m; ka.n = a.n; ka.k = a.k;
    ka.Ad = adup; ka.ldad = ldad;
    ka.B = a.B; ka.ldb = a.ldb;
    ka.C = a.C; ka.ldc = a.ldc;
    ka.prev = a.prev; ka.ldp = a.ldp;
    ka.changed = a.changed;
    ka.skip = a.skip;
    ka.one = 1;
    ka.maxfin = a.maxfin;
    ka.gate = a.gate;
    ka.Ci = a.Ci;
    ka.ldci = a.ldci;
    ka.xr0 = a.xr0;
    ka.xr1 = a.xr1;
    ka.xc0 = a.xc0;
    ka.xc1 = a.xc1;
    {
        // Grids of two or more waves: groups of 12 tile columns, k backwards in
        // every other wave (see U16KArgs::kwave); BTAS_KWAVE=0 turns it off.
        DeviceInfo di{};
        const int sms = current_device_info(&di, nullptr) ? di.sms : 152;
        const long long tiles = (long long)((a.m + u16::BM - 1) / u16::BM) * (((a.n + 1) / 2 + u16::BNP - 1) / u16::BNP);
        const char *kw = getenv("BTAS_KWAVE");
        if (tiles >= 2LL * sms && !(kw && atoi(kw) == 0)) {
            ka.kwave = sms;
            ka.kgroup = 12;
        }
    }
    ka.vec_a = (reinterpret_cast<uintptr_t>(adup) & 15) == 0;
    ka.vec_b = (reinterpret_cast<uintptr_t>(a.B) & 15) == 0 && (a.ldb & 7) == 0;
    switch (ns) {
        case 0: return launch_ns<0>(ka, st);
        case 4: return launch_ns<4>(ka, st);
        case 6: return launch_ns<6>(ka, st);
        case 8: return launch_ns<8>(ka, st);
        default: return launch_ns<5>(ka, st);
    }
}

}  // namespace btas
