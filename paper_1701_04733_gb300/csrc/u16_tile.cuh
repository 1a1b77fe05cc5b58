// One output tile (128 x 128, or 64 x 64 for small instances) of an exact
// packed 16-bit min-plus squaring, for the persistent tile-task kernel.  Same
// arithmetic as tgemm_u16.cu (two outputs per 32-bit lane, A duplicated into
// both halfwords, B pairs adjacent in row-major storage, per-halfword DPX
// add-min; exact when every operand is <= 0x7FFF), sized for 256 threads at
// 2 CTAs/SM: 8 rows x 4 column pairs per thread (4 x 2 for the 64 tile).  Inputs come from the 16-bit forms of D_{s-1} (Ad: duplicated
// words, U: uint16 values); the epilogue writes D_s as int32 (INF16 widened to
// INF), transposed int32, and again in both 16-bit forms, so the next
// squaring can run in either precision.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace btas {

struct U16Tile {
    int n;
    const uint32_t *Ad;  // n x n duplicated words, pitch ldad (multiple of 4)
    long long ldad;
    const uint16_t *U;   // n x n values, pitch ldu (multiple of 8)
    long long ldu;
    const int *prev;     // int32 D_{s-1} (unused: change detection reads U)
    long long ldp;
    int *C;              // int32 D_s
    long long ldc;
    int *Ct;             // optional: int32 D_s transposed
    long long ldct;
    uint32_t *Cd;        // optional: duplicated words of D_s
    long long ldcd;
    uint16_t *Cu;        // optional: uint16 D_s
    long long ldcu;
    int *maxfin;         // optional: atomicMax of the largest finite output
};

namespace u16t {
constexpr int BK = 32, ST = 3, NT = 256;
constexpr int LDA = BK + 4;  // words per A row
// BM rows x BNP column pairs (2 BNP columns) per tile; RI rows and PQ
// column pairs per thread
template <int BM_, int BNP_>
struct Shape {
    static constexpr int BM = BM_, BNP = BNP_;
    static constexpr int LDB = BNP;  // words per B row
    static constexpr int STAGE = BM * LDA + BK * LDB;
    static constexpr int SMEM = ST * STAGE * 4;
    static constexpr int RI = BM / 16, PQ = BNP / 16;
    static_assert(PQ == 2 || PQ == 4, "column pairs per thread");
};
using Big = Shape<128, 64>;   // 79872 bytes of shared memory
using Small = Shape<64, 32>;
constexpr int SMEM = Big::SMEM;
}  // namespace u16t

// Returns this thread's "some output differs from prev" bit.  smem must hold
// max(Shape::SMEM, BM * (2 BNP + 1) * 4) bytes.
template <class Sh>
__device__ __forceinline__ bool u16_tile_t(const U16Tile &a, int bm, int bn, unsigned char *smem_raw, int tid) {
    using namespace u16t;
    constexpr int BM = Sh::BM, BNP = Sh::BNP, LDB = Sh::LDB, STAGE = Sh::STAGE, RI = Sh::RI, PQ = Sh::PQ;
    constexpr int BN = 2 * BNP;  // output columns of the tile
    uint32_t *smem = reinterpret_cast<uint32_t *>(smem_raw);
    const int n = a.n;
    const int bnp = bn / 2;  // first column pair of the tile
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
    const bool va = ((reinterpret_cast<uintptr_t>(a.Ad) & 15) == 0) && ((a.ldad & 3) == 0);
    const bool vb = ((reinterpret_cast<uintptr_t>(a.U) & 15) == 0) && ((a.ldu & 7) == 0);
    const int KT = (n + BK - 1) / BK;
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
            if (va && gr < n && gk + 4 <= n) {
                cp_async16(dst, a.Ad + (long long)gr * a.ldad + gk);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    dst[e] = (gr < n && gk + e < n) ? __ldcg(a.Ad + (long long)gr * a.ldad + gk + e) : kInfU16x2;
            }
        }
        constexpr int CPR = BNP / 4;  // chunks of 4 words per B row
#pragma unroll
        for (int t = 0; t < (BK * BNP / 4) / NT; ++t) {
            const int c = tid + t * NT;
            const int r = c / CPR, wc = (c % CPR) * 4;
            const int gk = k0 + r, gcol = 2 * (bnp + wc);
            uint32_t *dst = sb + r * LDB + wc;
            if (vb && gk < n && gcol + 8 <= n) {
                cp_async16(dst, a.U + (long long)gk * a.ldu + gcol);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c0 = gcol + 2 * e;
                    uint32_t lo = BTAS_INF_U16, hi = BTAS_INF_U16;
                    if (gk < n) {
                        if (c0 < n) lo = __ldcg(a.U + (long long)gk * a.ldu + c0);
                        if (c0 + 1 < n) hi = __ldcg(a.U + (long long)gk * a.ldu + c0 + 1);
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
                uint32_t b[PQ];
                if constexpr (PQ == 4) {
                    const uint4 t = *reinterpret_cast<const uint4 *>(sb + (kk + q) * LDB + pair_base);
                    b[0] = t.x; b[1] = t.y; b[2] = t.z; b[3] = t.w;
                } else {
                    const uint2 t = *reinterpret_cast<const uint2 *>(sb + (kk + q) * LDB + pair_base);
                    b[0] = t.x; b[1] = t.y;
                }
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
    // Epilogue.  Change detection compares against U, the 16-bit form of
    // D_{s-1}: on the domain where this squaring is exact (finite entries
    // below 0x7FFF, INF stored as 0x7FFF) the 16-bit and int32 forms are in
    // one-to-one correspondence.  All loads of U are issued before any store;
    // rows whose 2 PQ columns lie inside the matrix use 16-byte stores.
    bool ch = false;
    int mx = -1;
    if (a.Ct != nullptr) __syncthreads();  // smem is reused for the transposed tile
    int *tr = reinterpret_cast<int *>(smem_raw);
    const int c0 = bn + 2 * pair_base;  // this thread's 2 PQ consecutive columns
    const bool vec_c = ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0) && ((a.ldc & 3) == 0) &&
                       (a.Cd == nullptr || (((reinterpret_cast<uintptr_t>(a.Cd) & 15) == 0) && ((a.ldcd & 3) == 0) &&
                                            ((reinterpret_cast<uintptr_t>(a.Cu) & 15) == 0) && ((a.ldcu & 7) == 0)));
    uint32_t pv[RI][PQ];
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        const int r = bm + row_base + 4 * i;
        const uint16_t *pu = a.U + (long long)r * a.ldu + c0;
        if (r < n && vb && c0 + 2 * PQ <= n) {
            if constexpr (PQ == 4) {
                const uint4 t = __ldcg(reinterpret_cast<const uint4 *>(pu));
                pv[i][0] = t.x; pv[i][1] = t.y; pv[i][2] = t.z; pv[i][3] = t.w;
            } else {
                const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(pu));
                pv[i][0] = t.x; pv[i][1] = t.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < PQ; ++q) {
                const uint32_t lo = (r < n && c0 + 2 * q < n) ? __ldcg(pu + 2 * q) : BTAS_INF_U16;
                const uint32_t hi = (r < n && c0 + 2 * q + 1 < n) ? __ldcg(pu + 2 * q + 1) : BTAS_INF_U16;
                pv[i][q] = lo | (hi << 16);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        const int rl = row_base + 4 * i, r = bm + rl;
#pragma unroll
        for (int j = 0; j < PQ; ++j) ch |= acc[i][j] != pv[i][j];
        int v[2 * PQ];
#pragma unroll
        for (int j = 0; j < PQ; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t u = h ? (acc[i][j] >> 16) : (acc[i][j] & 0xFFFFu);
                v[2 * j + h] = u >= BTAS_INF_U16 ? kInfI32 : (int)u;
                if (a.Ct != nullptr) tr[(2 * (pair_base + j) + h) * (BM + 1) + rl] = v[2 * j + h];
            }
        }
        if (r >= n) continue;
        if (vec_c && c0 + 2 * PQ <= n) {
#pragma unroll
            for (int e = 0; e < 2 * PQ; ++e)
                if (v[e] < kInfI32) mx = max(mx, v[e]);
            int *pc = a.C + (long long)r * a.ldc + c0;
#pragma unroll
            for (int e = 0; e < 2 * PQ; e += 4)
                *reinterpret_cast<int4 *>(pc + e) = make_int4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            if (a.Cd != nullptr) {
                uint32_t *pd = a.Cd + (long long)r * a.ldcd + c0;
                uint32_t d[2 * PQ];
#pragma unroll
                for (int e = 0; e < 2 * PQ; ++e) d[e] = (v[e] >= kInfI32 ? BTAS_INF_U16 : (uint32_t)v[e]) * 0x10001u;
#pragma unroll
                for (int e = 0; e < 2 * PQ; e += 4)
                    *reinterpret_cast<uint4 *>(pd + e) = make_uint4(d[e], d[e + 1], d[e + 2], d[e + 3]);
                uint16_t *pu = a.Cu + (long long)r * a.ldcu + c0;
                if constexpr (PQ == 4)
                    *reinterpret_cast<uint4 *>(pu) = make_uint4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                else
                    *reinterpret_cast<uint2 *>(pu) = make_uint2(acc[i][0], acc[i][1]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 2 * PQ; ++e) {
                const int c = c0 + e;
                if (c >= n) continue;
                if (v[e] < kInfI32) mx = max(mx, v[e]);
                a.C[(long long)r * a.ldc + c] = v[e];
                if (a.Cd != nullptr) {
                    const uint32_t u = v[e] >= kInfI32 ? BTAS_INF_U16 : (uint32_t)v[e];
                    a.Cd[(long long)r * a.ldcd + c] = u * 0x10001u;
                    a.Cu[(long long)r * a.ldcu + c] = (uint16_t)u;
                }
            }
        }
    }
    if (a.maxfin != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx >= 0) atomicMax(a.maxfin, mx);
    }
    if (a.Ct != nullptr) {
        __syncthreads();
        for (int idx = tid; idx < BM * BN; idx += NT) {
            const int c = idx / BM, r = idx % BM;
            if (bn + c < n && bm + r < n) a.Ct[(long long)(bn + c) * a.ldct + bm + r] = tr[c * (BM + 1) + r];
        }
        __syncthreads();
    }
    return ch;
}

__device__ __forceinline__ bool u16_tile(const U16Tile &a, int bm, int bn, unsigned char *smem_raw, int tid) {
    return u16_tile_t<u16t::Big>(a, bm, bn, smem_raw, tid);
}

}  // namespace btas
