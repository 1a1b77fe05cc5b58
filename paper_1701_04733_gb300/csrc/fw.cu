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
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tgemm.cuh"

namespace btas {

namespace {

constexpr int FB = 128;  // tile edge
constexpr int FT = 256;  // threads: 16 x 16, each owning 8 rows x 8 columns of the tile

// A thread's tile coordinates: rows ty*8 .. ty*8+7 (contiguous) and columns
// tx*4 + {0..3} and 64 + tx*4 + {0..3} (two groups, so that a warp's row
// loads are contiguous 16-byte chunks: no bank conflicts).
__device__ __forceinline__ int fw_col(int tx, int c) { return (c < 4 ? 0 : 64 - 4) + tx * 4 + c; }

// Load tile (r0, c0) of D into shared memory (INF outside the matrix), in
// 16-byte vectors where the rows allow (n a multiple of 4).
__device__ __forceinline__ void load_tile(int *sm, const int *D, long long n, int r0, int c0) {
    const bool vec = (n & 3) == 0;
    for (int idx = threadIdx.x; idx < FB * FB / 4; idx += blockDim.x) {
        const int r = idx / (FB / 4), c = (idx % (FB / 4)) * 4;
        const long long gr = r0 + r, gc = c0 + c;
        int4 v;
        if (vec && gr < n && gc + 4 <= n) {
            v = *reinterpret_cast<const int4 *>(D + gr * n + gc);
        } else {
            int t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) t[e] = (gr < n && gc + e < n) ? D[gr * n + gc + e] : kInfI32;
            v = make_int4(t[0], t[1], t[2], t[3]);
        }
        *reinterpret_cast<int4 *>(sm + r * FB + c) = v;
    }
}
// Store the tile; with pmax, also atomicMax the largest finite value stored.
__device__ __forceinline__ void store_tile(const int *sm, int *D, long long n, int r0, int c0, int *pmax) {
    const bool vec = (n & 3) == 0;
    int mx = -1;
    for (int idx = threadIdx.x; idx < FB * FB / 4; idx += blockDim.x) {
        const int r = idx / (FB / 4), c = (idx % (FB / 4)) * 4;
        const long long gr = r0 + r, gc = c0 + c;
        if (gr >= n) continue;
        const int4 v = *reinterpret_cast<const int4 *>(sm + r * FB + c);
        const int t[4] = {v.x, v.y, v.z, v.w};
        if (vec && gc + 4 <= n) {
            *reinterpret_cast<int4 *>(D + gr * n + gc) = v;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (t[e] < kInfI32) mx = max(mx, t[e]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (gc + e < n) {
                    D[gr * n + gc + e] = t[e];
                    if (t[e] < kInfI32) mx = max(mx, t[e]);
                }
        }
    }
    if (pmax != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx >= 0) atomicMax(pmax, mx);
    }
}

// d[r][c] = min(d[r][c], colsrc[row r][k] + rowsrc[k][column c]) for the
// thread's 8 x 8 outputs: 8 broadcast loads of the column, two 16-byte loads
// of the row, 64 DPX add-min.
__device__ __forceinline__ void relax8(int (&d)[8][8], const int *colsrc, const int *rowsrc, int i0, int tx, int k) {
    int a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = colsrc[(i0 + r) * FB + k];
    const int4 b0 = *reinterpret_cast<const int4 *>(rowsrc + k * FB + tx * 4);
    const int4 b1 = *reinterpret_cast<const int4 *>(rowsrc + k * FB + 64 + tx * 4);
    const int b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) d[r][c] = __viaddmin_s32(a[r], b[c], d[r][c]);
}

// The pivots of one block: blk[i][j] = min(blk[i][j], colsrc[i][k] +
// rowsrc[k][j]) for k = 0 .. kmax-1 in order (kmax < FB only in the last
// block, whose padding pivots are INF rows and columns and change nothing).
// Each thread keeps its 8 x 8 outputs in registers.  Pivot k reads row k of
// rowsrc and column k of colsrc; during pivot k neither changes (zero
// diagonal, non-negative weights), so after relaxing, only the owners of
// row k+1 (when rowsrc is blk: PUB_ROW) and of column k+1 (when colsrc is
// blk: PUB_COL) publish those values to shared memory, and one barrier per
// pivot orders them before the next pivot's reads.  Pivots go in groups of
// 8, unrolled, so the published row and column of each are known at compile
// time (registers are not indexed at run time).  Operands lie in [0, INF]:
// a + b cannot overflow, and one DPX add-min is one relaxation.
template <bool PUB_ROW, bool PUB_COL>
__device__ __forceinline__ void pivots(int *blk, const int *colsrc, const int *rowsrc, int kmax) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = ty * 8;
    int d[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) d[r][c] = blk[(i0 + r) * FB + fw_col(tx, c)];
    for (int kg = 0; kg < kmax; kg += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kg + q;
            if (k < kmax) {  // pivots past the matrix edge are INF rows/columns: no-ops
                relax8(d, colsrc, rowsrc, i0, tx, k);
                const int kn = k + 1;
                const int qr = (q + 1) & 7;  // row of kn within its owner (compile time)
                if (PUB_ROW && (kn >> 3) == ty) {
                    *reinterpret_cast<int4 *>(blk + (i0 + qr) * FB + tx * 4) =
                        make_int4(d[qr][0], d[qr][1], d[qr][2], d[qr][3]);
                    *reinterpret_cast<int4 *>(blk + (i0 + qr) * FB + 64 + tx * 4) =
                        make_int4(d[qr][4], d[qr][5], d[qr][6], d[qr][7]);
                }
                // column kn: group h = kn >= 64, owner tx = (kn & 63) >> 2, slot (kn & 3) = (q + 1) & 3
                const int qc = (q + 1) & 3;
                if (PUB_COL && ((kn & 63) >> 2) == tx && kn < FB) {
                    const bool hi = kn >= 64;
#pragma unroll
                    for (int r = 0; r < 8; ++r) blk[(i0 + r) * FB + kn] = hi ? d[r][4 + qc] : d[r][qc];
                }
                __syncthreads();
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        *reinterpret_cast<int4 *>(blk + (i0 + r) * FB + tx * 4) = make_int4(d[r][0], d[r][1], d[r][2], d[r][3]);
        *reinterpret_cast<int4 *>(blk + (i0 + r) * FB + 64 + tx * 4) = make_int4(d[r][4], d[r][5], d[r][6], d[r][7]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(FT, 1) fw_diag_kernel(int *D, long long n, int kb, int *pmax) {
    extern __shared__ __align__(16) int sm[];
    const int o = kb * FB;
    load_tile(sm, D, n, o, o);
    __syncthreads();
    pivots<true, true>(sm, sm, sm, (int)min((long long)FB, n - o));
    store_tile(sm, D, n, o, o, pmax);
}

// blockIdx.x < nb: row panel tile (kb, b) relaxes through diag[i][k] +
// blk[k][j]; else column panel tile (b, kb) through blk[i][k] + diag[k][j].
__global__ void __launch_bounds__(FT, 1) fw_panel_kernel(int *D, long long n, int kb, int nb, int *pmax) {
    extern __shared__ __align__(16) int sm[];
    int *diag = sm, *blk = sm + FB * FB;
    const bool row = blockIdx.x < (unsigned)nb;
    const int b = row ? blockIdx.x : blockIdx.x - nb;
    if (b == kb) return;
    const int o = kb * FB;
    const int r0 = row ? o : b * FB, c0 = row ? b * FB : o;
    load_tile(diag, D, n, o, o);
    load_tile(blk, D, n, r0, c0);
    __syncthreads();
    const int kmax = (int)min((long long)FB, n - o);
    if (row) pivots<true, false>(blk, diag, blk, kmax);
    else pivots<false, true>(blk, blk, diag, kmax);
    store_tile(blk, D, n, r0, c0, pmax);
}

// Lookahead: the phase-3 update of pivot block kb applied to block row and
// block column kb + 1 only -- the tiles that pivot block kb + 1's phases 1-2
// read and write -- so that those phases can run while the rest of phase 3
// (which leaves block row and column kb + 1 alone) is still going on.
// blockIdx.x < nb: tile (kb + 1, b), b != kb (b = kb + 1 is the diagonal
// tile); else tile (b, kb + 1), b != kb, kb + 1.  Each CTA takes
// T = min(T, D[rows of T, pivots of kb] (x) D[pivots of kb, columns of T]),
// the same terms phase 3 would, with the pivot tiles final after phases 1-2
// of kb.
constexpr int FXT = 1024;  // lookahead update: 32 x 32 threads, 4 x 4 outputs each (no barriers, many warps)

__global__ void __launch_bounds__(FXT, 1) fw_cross_kernel(int *D, long long n, int kb, int nb) {
    extern __shared__ __align__(16) int sm[];
    int *colsrc = sm, *rowsrc = sm + FB * FB, *blk = sm + 2 * FB * FB;
    const bool row = blockIdx.x < (unsigned)nb;
    const int b = row ? blockIdx.x : blockIdx.x - nb;
    const int kn = kb + 1;
    if (b == kb || (!row && b == kn)) return;
    const int o = kb * FB;
    const int r0 = row ? kn * FB : b * FB, c0 = row ? b * FB : kn * FB;
    load_tile(colsrc, D, n, r0, o);
    load_tile(rowsrc, D, n, o, c0);
    load_tile(blk, D, n, r0, c0);
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = ty * 4, j0 = tx * 4;
    int d[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int4 v = *reinterpret_cast<const int4 *>(blk + (i0 + r) * FB + j0);
        d[r][0] = v.x; d[r][1] = v.y; d[r][2] = v.z; d[r][3] = v.w;
    }
    const int kmax = (int)min((long long)FB, n - o);
#pragma unroll 4
    for (int k = 0; k < kmax; ++k) {
        int a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = colsrc[(i0 + r) * FB + k];
        const int4 bv = *reinterpret_cast<const int4 *>(rowsrc + k * FB + j0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            d[r][0] = __viaddmin_s32(a[r], bv.x, d[r][0]);
            d[r][1] = __viaddmin_s32(a[r], bv.y, d[r][1]);
            d[r][2] = __viaddmin_s32(a[r], bv.z, d[r][2]);
            d[r][3] = __viaddmin_s32(a[r], bv.w, d[r][3]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r)
        *reinterpret_cast<int4 *>(blk + (i0 + r) * FB + j0) = make_int4(d[r][0], d[r][1], d[r][2], d[r][3]);
    __syncthreads();
    store_tile(blk, D, n, r0, c0, nullptr);
}

// Packed phase 3: state[0] = 1 when every finite entry of the pivot row and
// column panels (after phase 2) is < 0x7FFF / 2, so that every finite term of
// the phase-3 product is < 0x7FFF and the packed u16x2 product is exact;
// state[1] = !state[0].
__global__ void fw_pack_decide_kernel(const int *pmax, int *state) {
    if (threadIdx.x != 0) return;
    const int use = 2LL * __ldcg(pmax) < BTAS_INF_U16;
    state[0] = use;
    state[1] = !use;
}

// Column panel D[:, o:o+bw] -> duplicated 16-bit words (n x ldad); row panel
// D[o:o+bw, :] -> uint16 (bw x ldbu).  INF (or anything >= 0x7FFF, which the
// decision rules out for finite entries) becomes 0x7FFF.
__global__ void fw_pack_panels_kernel(const int *D, long long n, long long o, int bw, const int *state,
                                      uint32_t *Ad, long long ldad, uint16_t *Bu, long long ldbu) {
    if (__ldcg(state) == 0) return;
    const long long colp = n * bw, total = colp + (long long)bw * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < colp) {
            const long long i = idx / bw, k = idx % bw;
            const int v = D[i * n + o + k];
            const uint32_t u = v >= BTAS_INF_U16 ? BTAS_INF_U16 : (uint32_t)v;
            Ad[i * ldad + k] = u * 0x10001u;
        } else {
            const long long q = idx - colp, k = q / n, j = q % n;
            const int v = D[(o + k) * n + j];
            Bu[k * ldbu + j] = (uint16_t)(v >= BTAS_INF_U16 ? BTAS_INF_U16 : v);
        }
    }
}

}  // namespace

cudaError_t launch_fw_pack(int *D, long long n, int kb, const int *pmax, int *state, uint32_t *Ad, long long ldad,
                           uint16_t *Bu, long long ldbu, cudaStream_t st) {
    const long long o = (long long)kb * FB;
    const int bw = (int)std::min<long long>(FB, n - o);
    fw_pack_decide_kernel<<<1, 32, 0, st>>>(pmax, state);
    const long long total = 2 * n * bw;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
    fw_pack_panels_kernel<<<grid, 256, 0, st>>>(D, n, o, bw, state, Ad, ldad, Bu, ldbu);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_fw_phase12(int *D, long long n, int kb, int *pmax, cudaStream_t st) {
    const int nb = (int)((n + FB - 1) / FB);
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(fw_diag_kernel), FB * FB * 4);
    if (e != cudaSuccess) return e;
    e = set_smem_once(reinterpret_cast<const void *>(fw_panel_kernel), 2 * FB * FB * 4);
    if (e != cudaSuccess) return e;
    fw_diag_kernel<<<1, FT, FB * FB * 4, st>>>(D, n, kb, pmax);
    note_launch();
    if (nb > 1) {
        fw_panel_kernel<<<2 * nb, FT, 2 * FB * FB * 4, st>>>(D, n, kb, nb, pmax);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_fw_cross(int *D, long long n, int kb, cudaStream_t st) {
    const int nb = (int)((n + FB - 1) / FB);
    if (kb + 1 >= nb) return cudaSuccess;
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(fw_cross_kernel), 3 * FB * FB * 4);
    if (e != cudaSuccess) return e;
    fw_cross_kernel<<<2 * nb, FXT, 3 * FB * FB * 4, st>>>(D, n, kb, nb);
    note_launch();
    return cudaGetLastError();
}

int fw_block() { return FB; }

namespace {

// Phase 3 of one pivot block in ONE launch on the int32 product tile: every
// 128 x 128 tile of D outside tile rows and columns [x0, x1) (the pivot
// block, and block kb + 1 while its phases run ahead on the other stream)
// takes D[i][j] = min(D[i][j], min_k D[i][o+k] + RPT[j][k]) over the bw
// pivots of the block (RPT: the pivot row panel, transposed).  One launch
// instead of one product per rectangle around the excluded rows and
// columns: a single tail wave per pivot block.  The excluded range is whole
// tiles (pivot blocks are FB = 128 wide), so the compressed tile grid maps
// back by shifting the indices at or above x0 past the range.
//
// The 2-CTA/SM product tile.  Measured on GB300 at n = 8192 against k = 128
// staged whole (four 32-deep stages in flight, one CTA per SM, 64- or
// 128-bit fragments): 38.3 ms for the int32 solve against 43.3 and 44.8 ms.
using FwCfg = TileCfg<128, 128, 32, 3, 2, 2, 1>;
static_assert(FwCfg::BM == FB && FwCfg::BN == FB, "tiles are pivot blocks");

__global__ void __launch_bounds__(FwCfg::kThreads, FwCfg::MINB)
fw_phase3_kernel(const GemmArgs a, int x0, int x1, int resident) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.bypass != nullptr && __ldcg(a.bypass) != 0) return;  // the packed phase 3 ran instead
    const int tiles = (a.m + FB - 1) / FB, skip = x1 - x0, t = tiles - skip;
    auto tile_of = [&](int pid, int &tm, int &tn) {
        raster(pid, t, t, a.group_m, tm, tn);
        if (tm >= x0) tm += skip;
        if (tn >= x0) tn += skip;
    };
    int tm, tn;
    tile_of(blockIdx.x, tm, tn);
    // Pull the C tile of the CTA that takes this one's place on the SM
    // (blockIdx + the CTAs resident at once) into L2, so that its
    // accumulator read at k = 128 comes from L2 rather than HBM.
    const int succ = blockIdx.x + resident;
    if (succ < t * t) {
        int sm, sn;
        tile_of(succ, sm, sn);
        const int *C = static_cast<const int *>(a.C);
        for (int l = threadIdx.x; l < FB * (FB / 32); l += blockDim.x) {  // 128-byte lines
            const long long r = (long long)sm * FB + l / (FB / 32), c = (long long)sn * FB + (l % (FB / 32)) * 32;
            if (r < a.m && c < a.n) asm volatile("prefetch.global.L2 [%0];" ::"l"(C + r * a.ldc + c));
        }
    }
    nt_tile<FwCfg, kI32Mix, kMin, 4>(a, tm * FB, tn * FB, smem_raw, threadIdx.x);
}

}  // namespace

cudaError_t launch_fw_phase3_i32(int *D, long long n, long long o, int bw, const int *RPT, int x0, int x1,
                                 const int *bypass, cudaStream_t st) {
    const int tiles = (int)((n + FB - 1) / FB), t = tiles - (x1 - x0);
    if (t <= 0 || bw <= 0) return cudaSuccess;
    GemmArgs a{};
    a.m = a.n = (int)n;
    a.k = bw;
    a.A = D + o; a.lda = n;      // the pivot column panel D[:, o:o+bw]
    a.Bt = RPT; a.ldb = FB;      // the pivot row panel, transposed
    a.C = D; a.ldc = n;
    a.accumulate = 1;
    a.one = 1;
    a.vec_a = (reinterpret_cast<uintptr_t>(D + o) & 15) == 0 && (n & 3) == 0;
    a.vec_b = (reinterpret_cast<uintptr_t>(RPT) & 15) == 0;
    a.ro_a = a.ro_b = 1;  // columns [o, o+bw) and RPT are not written by this launch
    a.group_m = 8;
    a.bypass = bypass;
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(fw_phase3_kernel), FwCfg::kSmemBytes);
    if (e != cudaSuccess) return e;
    DeviceInfo di{};
    const int sms = current_device_info(&di, nullptr) ? di.sms : 148;
    fw_phase3_kernel<<<(unsigned)t * (unsigned)t, FwCfg::kThreads, FwCfg::kSmemBytes, st>>>(a, x0, x1,
                                                                                          FwCfg::MINB * sms);
    note_launch();
    return cudaGetLastError();
}

}  // namespace btas
