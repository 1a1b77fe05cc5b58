// APSP by repeated squaring (Sec. III) for mid-size graphs in ONE
// cooperative launch.
//
// Between the one-block kernel (n <= 64) and the tiled product kernels (n >
// 1792) a solve is bound by launches and host round trips: a few dozen
// tiles per squaring cannot fill the GPU, and every squaring waits for the
// previous one's change flag.  Here one cooperative grid runs the domain check and all
// squarings, with ONE grid barrier per squaring.
//
// Work split.  Squaring s is a space of units (64 x 64 output tile, 32-wide
// k-step), cut into equal contiguous shares, one per block ("stream-K"): a
// block's share covers the end of one tile's k-range, whole tiles, and the
// start of another, so the blocks finish together whatever n is.  The
// consecutive units of one tile in a share form a piece (a tile and a
// k-range) whose partial minimum p the block merges into X_s.
//
// Merging without a second pass.  With a zero diagonal and non-negative
// weights X_s <= X_{s-1} entrywise: the terms k = i and k = j of the product
// are X_{s-1}[i][j] itself.  So the piece holding k = j has
// p <= X_{s-1}[i][j], and X_s[i][j] < X_{s-1}[i][j] exactly when some piece
// finds p < X_{s-1}[i][j].  A piece merges p into X_s (reset to INF
// beforehand) with atomicMin where p < X_{s-1}[i][j], or where p equals it
// and the piece holds k = j; any other p cannot be the minimum.  The same
// comparison is the change test, so a squaring needs no checking pass, and
// (+) = min being associative, commutative and idempotent makes the merge
// exact in any order.
//
// Precision per squaring.  Every finite entry of X_s is one of the values
// merged during squaring s, so their maximum bounds max(X_s).  When the
// bound is <= 16383 the next squaring runs on packed 16-bit pairs (two terms
// per DPX add-min, INF as 0x7FFF; sums of operands stay <= 32766, so 0x7FFF
// still means "no path"), else on int32 (DPX add-min, INF absorbed by the
// clamp at INF - 2^28).  Both are exact: results are bit-identical to the
// other paths.
//
// Buffers.  X_s lives in buf[(s - 1) % 3] and X_0, a pitch-ldx copy of W, in
// buf2.  Squaring s reads X_{s-1}, merges into X_s and resets X_{s+1}'s
// buffer, which held X_{s-2}.  The grid barrier after a squaring also
// carries its change flag and merged maximum to every block.  Every barrier
// wait is bounded (clock64); on expiry the kernel records BTAS_ERR_TIMEOUT
// and all blocks return.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "grid_sync.cuh"
#include "kernels.h"

namespace btas {
namespace {

constexpr int kT = 64, kThreads = 256, kKc = 32;  // tile edge, threads, k step
constexpr int kLdA = kT + 4;                      // k-major A stage row (words)
constexpr int kU16Max = 16383;                    // operand bound of the packed squaring

struct MidArgs {
    const int *W;
    long long ldw;
    int n;
    int S;
    int early;
    int u16_ok;  // 0: int32 squarings only
    int withhold;  // test hook: the last block skips the first barrier, so the others' waits expire
    int *D;
    long long ldd;
    int *buf0, *buf1, *buf2;  // n x ldx each; columns n .. ldx-1 always hold INF
    long long ldx;            // round4(n): 16-byte rows for vector staging
    unsigned *bar;  // [0, 16) barrier counters, [32, 33] release word (grid_sync.cuh), [64 + s] largest merged value
    int *info;      // [0] bad entries, [1] max weight, [2] squarings that changed, [3] status,
                    // [4] representations used (1 int32, 4 packed 16-bit)
    int *mailbox;   // optional, host-mapped: info[0 .. 4] copied there by block 0 as it exits
    long long timeout_cycles;
};

struct MidSmem {
    int a[2][kKc][kLdA];  // A stage, k-major: a[k][row]; packed mode: duplicated 16-bit words
    int b[2][kKc][kT];    // B stage: b[k][col]; packed mode: b[k][pair] in the first kT / 2 words
};

__device__ __forceinline__ bool grid_barrier(const MidArgs &a, unsigned &gen, bool flag, const int *pval, int &v0,
                                             int &v1) {
    return btas::grid_barrier(GridSync{a.bar, a.info + 3, a.timeout_cycles}, gen, flag, pval, v0, v1);
}

__device__ __forceinline__ int *bufp(const MidArgs &a, int i) { return i == 0 ? a.buf0 : i == 1 ? a.buf1 : a.buf2; }

// 16-bit form of an entry of a packed squaring's operand: <= 16383, or 0x7FFF for INF
__device__ __forceinline__ unsigned u16_of(int v) { return (unsigned)min(v, BTAS_INF_U16); }

// One k-step of operands from global memory (L2: X is written by other
// blocks), into registers.  A = X[bm.., kb..] (64 x 32) as 16-byte vectors
// along k, B = X[kb.., bn..] (32 x 64) along columns.  Lane pairs of a warp
// read 32 contiguous bytes of one of 16 rows, which also makes the
// transposing shared-memory stores below conflict-free.  A vector that
// starts inside the matrix ends inside the row (ldx is a multiple of 4) and
// reads INF padding past column n-1; k-chunks end on multiples of 32, so no
// vector crosses one.
__device__ __forceinline__ void fetch(const int *in, long long ldx, int n, int bm, int bn, int kb, int k1, int tid,
                                      int4 (&va)[2], int4 (&vb)[2]) {
    const int4 inf4 = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = tid + q * kThreads;
        const int kg = (e & 1) + 2 * ((e >> 5) & 3), r = ((e >> 1) & 15) + 16 * (e >> 7);
        const int gi = bm + r, gk = kb + 4 * kg;
        va[q] = (gi < n && gk < k1) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gi * ldx + gk)) : inf4;
        const int rk = e >> 4, cb = (e & 15) * 4;
        const int gkb = kb + rk, gj = bn + cb;
        vb[q] = (gkb < k1 && gj < n) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gkb * ldx + gj)) : inf4;
    }
}

// Registers -> one shared stage: A transposed to k-major, B as is; the
// packed form stores A as duplicated 16-bit words and B as column pairs.
template <bool U16>
__device__ __forceinline__ void stash(MidSmem &sm, int buf, int tid, const int4 (&va)[2], const int4 (&vb)[2]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = tid + q * kThreads;
        const int kg = (e & 1) + 2 * ((e >> 5) & 3), r = ((e >> 1) & 15) + 16 * (e >> 7);
        int *col = &sm.a[buf][4 * kg][r];
        if (U16) {
            col[0] = (int)(u16_of(va[q].x) * 0x10001u);
            col[kLdA] = (int)(u16_of(va[q].y) * 0x10001u);
            col[2 * kLdA] = (int)(u16_of(va[q].z) * 0x10001u);
            col[3 * kLdA] = (int)(u16_of(va[q].w) * 0x10001u);
        } else {
            col[0] = va[q].x;
            col[kLdA] = va[q].y;
            col[2 * kLdA] = va[q].z;
            col[3 * kLdA] = va[q].w;
        }
        const int rk = e >> 4, cb = (e & 15) * 4;
        if (U16) {
            const uint2 w = make_uint2(u16_of(vb[q].x) | (u16_of(vb[q].y) << 16),
                                       u16_of(vb[q].z) | (u16_of(vb[q].w) << 16));
            *reinterpret_cast<uint2 *>(&sm.b[buf][rk][cb / 2]) = w;
        } else {
            *reinterpret_cast<int4 *>(&sm.b[buf][rk][cb]) = vb[q];
        }
    }
}

// One piece: the 64 x 64 tile (bm, bn) of X_{s-1} (x) X_{s-1} over k in
// [k0, k1), merged into out.  256 threads, 4 x 4 outputs each; the next
// k-step's operands are in flight while this one is computed.
template <bool U16>
__device__ __forceinline__ void run_item(const MidArgs &a, const int *in, int *out, int bm, int bn, int k0, int k1,
                                         MidSmem &sm, int tid, bool &ch, int &mx) {
    const int n = a.n;
    const long long ldx = a.ldx;
    const int ty = tid >> 4, tx = tid & 15;
    const int r0 = bm + ty * 4, c0 = bn + tx * 4;
    // X_{s-1} over this thread's outputs (the merge bound), fetched first
    int4 old[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        old[r] = (r0 + r < n && c0 < n) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)(r0 + r) * ldx + c0))
                                        : make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
    int acc[4][4];         // int32 mode
    unsigned acc16[4][2];  // packed mode: columns (c0 + 2p, c0 + 2p + 1) in (low, high)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = kInfI32;
        acc16[r][0] = acc16[r][1] = kInfU16x2;
    }
    int4 va[2], vb[2];
    fetch(in, ldx, n, bm, bn, k0, k1, tid, va, vb);
    stash<U16>(sm, 0, tid, va, vb);
    __syncthreads();
    int buf = 0;
    for (int kb = k0; kb < k1; kb += kKc) {
        const bool more = kb + kKc < k1;
        if (more) fetch(in, ldx, n, bm, bn, kb + kKc, k1, tid, va, vb);
#pragma unroll 8
        for (int k = 0; k < kKc; ++k) {
            const int4 av = *reinterpret_cast<const int4 *>(&sm.a[buf][k][ty * 4]);
            const int ar[4] = {av.x, av.y, av.z, av.w};
            if (U16) {
                const uint2 bv = *reinterpret_cast<const uint2 *>(&sm.b[buf][k][tx * 2]);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc16[r][0] = u16x2_addmin((unsigned)ar[r], bv.x, acc16[r][0]);
                    acc16[r][1] = u16x2_addmin((unsigned)ar[r], bv.y, acc16[r][1]);
                }
            } else {
                const int4 bv = *reinterpret_cast<const int4 *>(&sm.b[buf][k][tx * 4]);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[r][0] = __viaddmin_s32(ar[r], bv.x, acc[r][0]);
                    acc[r][1] = __viaddmin_s32(ar[r], bv.y, acc[r][1]);
                    acc[r][2] = __viaddmin_s32(ar[r], bv.z, acc[r][2]);
                    acc[r][3] = __viaddmin_s32(ar[r], bv.w, acc[r][3]);
                }
            }
        }
        if (more) stash<U16>(sm, buf ^ 1, tid, va, vb);
        __syncthreads();
        buf ^= 1;
    }
    // merge: p < old (a change), or p == old from the piece holding k = j
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = r0 + r;
        const int o[4] = {old[r].x, old[r].y, old[r].z, old[r].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = c0 + c;
            int p;
            if (U16) {
                const unsigned h = (acc16[r][c >> 1] >> (16 * (c & 1))) & 0xFFFFu;
                p = h >= (unsigned)BTAS_INF_U16 ? kInfI32 : (int)h;
            } else {
                p = clamp_i32<kMin>(acc[r][c]);
            }
            if (i < n && j < n && p < kInfI32 && (p < o[c] || (p == o[c] && j >= k0 && j < k1))) {
                atomicMin(out + (long long)i * ldx + j, p);
                mx = max(mx, p);
                ch |= p < o[c];
            }
        }
    }
}

// A block's share [u0, u1) of squaring s, unit u = k-step u % KS of tile
// u / KS, as pieces of consecutive units of one tile.
template <bool U16>
__device__ __forceinline__ void squaring(const MidArgs &a, const int *in, int *out, int tiles, int KS, long long u0,
                                         long long u1, MidSmem &sm, int tid, bool &ch, int &mx) {
    const int n = a.n;
    long long u = u0;
    while (u < u1) {
        const int tile = (int)(u / KS), ks = (int)(u % KS);
        const long long pe = min(u1, (long long)(tile + 1) * KS);
        const int k0 = ks * kKc, k1 = min(n, (int)(pe - (long long)tile * KS) * kKc);
        run_item<U16>(a, in, out, (tile / tiles) * kT, (tile % tiles) * kT, k0, k1, sm, tid, ch, mx);
        u = pe;
    }
}

// Phase 0 of both forms of the kernel: the domain check, W -> X_0 (buf2) and
// X_1's buffer (buf0) to INF; the entries outside the domain and the largest
// finite weight go to info[0] and info[1].  Returns whether this block found
// an entry outside the domain.
__device__ __forceinline__ bool mid_phase0(const MidArgs &a, long long gtid, long long gthreads) {
    const int n = a.n;
    const long long ldx = a.ldx, nx = (long long)n * ldx;
    int bad = 0, mx = 0;
    for (long long idx = gtid; idx < nx; idx += gthreads) {
        const int i = (int)(idx / ldx), j = (int)(idx % ldx);
        int v = kInfI32;
        if (j < n) {
            v = a.W[(long long)i * a.ldw + j];
            const bool fin = v >= 0 && v <= BTAS_I32_FINITE_MAX;
            if ((!fin && v != kInfI32) || (i == j && v != 0)) ++bad;
            if (fin) mx = max(mx, v);
        }
        a.buf2[idx] = v;
        a.buf0[idx] = kInfI32;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(a.info + 0, bad);
        atomicMax(a.info + 1, mx);
    }
    return __syncthreads_or(bad != 0) != 0;
}

// The result X_last -> D (W was read only in phase 0, so D may be W), and the
// squarings that changed D and the representations used to info[2], info[4].
__device__ __forceinline__ void mid_finish(const MidArgs &a, const int *in, long long gtid, long long gthreads,
                                           int done, int path) {
    const int n = a.n;
    const long long ldx = a.ldx;
    for (long long idx = gtid; idx < (long long)n * n; idx += gthreads)
        a.D[(idx / n) * a.ldd + idx % n] = __ldcg(in + (idx / n) * ldx + idx % n);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[2] = done;
        a.info[4] = path;
    }
}

__device__ __forceinline__ void mid_body(const MidArgs &a) {
    __shared__ __align__(16) MidSmem sm;
    const int n = a.n, tid = threadIdx.x;
    const long long ldx = a.ldx;
    const long long nx = (long long)n * ldx;
    const long long gthreads = (long long)gridDim.x * kThreads;
    const long long gtid = (long long)blockIdx.x * kThreads + tid;
    unsigned gen = 0;

    // phase 0: domain check, W -> X_0 (buf2), X_1's buffer to INF
    const bool bad_block = mid_phase0(a, gtid, gthreads);
    int nbad = 0, bound = 0;  // bound: >= every finite entry of X_{s-1}
    if (a.withhold && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier(a, gen, bad_block, a.info + 1, nbad, bound)) return;
    if (nbad != 0) return;  // D untouched

    // stream-K split of the (tile, k-step) units: equal shares, +-1 unit
    const int tiles = (n + kT - 1) / kT, KS = (n + kKc - 1) / kKc;
    const long long U = (long long)tiles * tiles * KS;
    const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
    const int4 inf4 = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
    const int *in = a.buf2;           // X_0
    int cur = 0, done = 0, path = 0;  // X_s (s >= 1) lives in buf[(s - 1) % 3]
    for (int s = 1; s <= a.S; ++s) {
        int *out = bufp(a, cur);
        if (s < a.S) {
            int4 *nxt = reinterpret_cast<int4 *>(bufp(a, (cur + 1) % 3));
            for (long long idx = gtid; idx < nx / 4; idx += gthreads) nxt[idx] = inf4;
        }
        const bool u16 = a.u16_ok && bound <= kU16Max;
        path |= u16 ? 4 : 1;
        bool ch = false;
        int mx = 0;
        if (u16)
            squaring<true>(a, in, out, tiles, KS, u0, u1, sm, tid, ch, mx);
        else
            squaring<false>(a, in, out, tiles, KS, u0, u1, sm, tid, ch, mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0 && mx > 0) atomicMax(reinterpret_cast<int *>(a.bar + 64 + s), mx);
        int changed = 0;
        if (!grid_barrier(a, gen, ch, reinterpret_cast<const int *>(a.bar + 64 + s), changed, bound)) return;
        done += changed != 0;
        in = out;
        cur = (cur + 1) % 3;
        if (!changed && a.early) break;
    }
    mid_finish(a, in, gtid, gthreads, done, path);
}


// ---- Wide warp-specialised form for the larger mid sizes: 128 x 128
// tiles, one block per SM, two producer warps that stage each unit (128 x 32
// of A transposed to k-major, 32 x 128 of B; the packed forms converted)
// into a kWStages-deep shared ring, and eight consumer warps with 8 x 8
// outputs per thread (a third of the shared-memory loads per term of the
// 64 x 64 form).  Full/empty mbarriers order the ring.  Every mbarrier wait
// is bounded: on expiry the waiting thread records BTAS_ERR_TIMEOUT and
// leaves the squaring, and the grid barrier that follows returns false in
// every block.
constexpr int kWConsumers = 256, kWProducers = 64, kWThreads = kWConsumers + kWProducers;
constexpr int kWT = 128;        // tile edge
constexpr int kWLdA = kWT + 4;  // k-major A row (words)
constexpr int kWStages = 4;

struct WwStage {
    int a[kKc][kWLdA];  // A[k][row]; packed: duplicated 16-bit words
    int b[kKc][kWT];    // B[k][col]; packed: column pairs in the first kWT / 2 words
};
struct WwSmem {
    WwStage st[kWStages];
    unsigned long long full[kWStages], empty[kWStages];
};
constexpr int kWwSmem = (int)sizeof(WwSmem);

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    unsigned long long state;  // the arrival's phase token, not needed here
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(b)) : "memory");
    asm volatile("" ::"l"(state));
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the phase with this parity; false (and
// the status word set) on expiry or once another block has given up.
__device__ __forceinline__ bool mbar_wait(const MidArgs &a, unsigned long long *b, unsigned parity) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        if (mbar_test(b, parity)) return true;
        if ((it & 255) == 0 && gsync::ld_relaxed_i32(a.info + 3) != 0) return false;
        if (clock64() - t0 > a.timeout_cycles) {
            atomicCAS(a.info + 3, 0, BTAS_ERR_TIMEOUT);
            return false;
        }
    }
}

// Producers: every unit of the share [u0, u1) into ring slot q % kWStages, q =
// qbase + (u - u0).  Returns false on a timeout.
template <bool U16>
__device__ __forceinline__ bool ww_produce(const MidArgs &a, const int *in, int tiles, int KS, long long u0,
                                           long long u1, long long qbase, WwSmem &sm, int ptid) {
    const int n = a.n;
    const long long ldx = a.ldx;
    const int lane = ptid & 31;
    const int4 inf4 = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
    for (long long u = u0; u < u1; ++u) {
        const long long q = qbase + (u - u0);
        const int slot = (int)(q % kWStages);
        const long long round = q / kWStages;
        if (round > 0 && !mbar_wait(a, &sm.empty[slot], (unsigned)((round - 1) & 1))) return false;
        const int tile = (int)(u / KS), ks = (int)(u % KS);
        const int bm = (tile / tiles) * kWT, bn = (tile % tiles) * kWT;
        const int kb = ks * kKc, k1 = min(n, kb + kKc);
        WwStage &st = sm.st[slot];
        // A: 128 rows x 8 k-groups of 4 (1024 vectors, 16 per thread, all in
        // flight before any store); element e: k-group (e & 1) + 2 * ((e >> 5)
        // & 3), row ((e >> 1) & 15) + 16 * (e >> 7), so that a warp's
        // transposing stores hit 32 distinct banks.  A vector that starts
        // inside the matrix ends inside the padded row (ldx is a multiple of
        // 4) and reads INF padding past column n - 1.
        {
            int4 v[16];
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
                const int e = ptid + q4 * kWProducers;
                const int kg = (e & 1) + 2 * ((e >> 5) & 3), r = ((e >> 1) & 15) + 16 * (e >> 7);
                const int gi = bm + r, gk = kb + 4 * kg;
                v[q4] = (gi < n && gk < k1) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gi * ldx + gk))
                                            : inf4;
            }
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
                const int e = ptid + q4 * kWProducers;
                const int kg = (e & 1) + 2 * ((e >> 5) & 3), r = ((e >> 1) & 15) + 16 * (e >> 7);
                int *col = &st.a[4 * kg][r];
                if (U16) {
                    col[0] = (int)(u16_of(v[q4].x) * 0x10001u);
                    col[kWLdA] = (int)(u16_of(v[q4].y) * 0x10001u);
                    col[2 * kWLdA] = (int)(u16_of(v[q4].z) * 0x10001u);
                    col[3 * kWLdA] = (int)(u16_of(v[q4].w) * 0x10001u);
                } else {
                    col[0] = v[q4].x;
                    col[kWLdA] = v[q4].y;
                    col[2 * kWLdA] = v[q4].z;
                    col[3 * kWLdA] = v[q4].w;
                }
            }
        }
        // B: 32 k-rows x 32 column groups of 4 (1024 vectors), rows contiguous
        {
            int4 v[16];
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
                const int e = ptid + q4 * kWProducers;
                const int rk = e >> 5, cb = (e & 31) * 4;
                const int gkb = kb + rk, gj = bn + cb;
                v[q4] = (gkb < k1 && gj < n) ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)gkb * ldx + gj))
                                             : inf4;
            }
#pragma unroll
            for (int q4 = 0; q4 < 16; ++q4) {
                const int e = ptid + q4 * kWProducers;
                const int rk = e >> 5, cb = (e & 31) * 4;
                if (U16) {
                    const uint2 w = make_uint2(u16_of(v[q4].x) | (u16_of(v[q4].y) << 16),
                                               u16_of(v[q4].z) | (u16_of(v[q4].w) << 16));
                    *reinterpret_cast<uint2 *>(&st.b[rk][cb / 2]) = w;
                } else {
                    *reinterpret_cast<int4 *>(&st.b[rk][cb]) = v[q4];
                }
            }
        }
        __threadfence_block();
        __syncwarp();  // every lane's stores, ordered before the warp's arrival
        if (lane == 0) mbar_arrive(&sm.full[slot]);
    }
    return true;
}

// Consumers: the pieces of the share (a tile and its consecutive units),
// computed from the ring and merged as in run_item.  Thread (ty, tx) =
// (tid / 16, tid % 16) owns rows bm + 8 ty .. + 7 and columns bn + 8 tx .. + 7
// (packed: pairs 4 tx .. 4 tx + 3).  Returns false on a timeout.
template <bool U16>
__device__ __forceinline__ bool ww_consume(const MidArgs &a, const int *in, int *out, int tiles, int KS, long long u0,
                                           long long u1, long long qbase, WwSmem &sm, int tid, bool &ch, int &mx) {
    const int n = a.n;
    const long long ldx = a.ldx;
    const int ty = tid >> 4, tx = tid & 15, lane = tid & 31;
    long long u = u0;
    while (u < u1) {
        const int tile = (int)(u / KS), ks = (int)(u % KS);
        const long long pe = min(u1, (long long)(tile + 1) * KS);
        const int k0 = ks * kKc, k1 = min(n, (int)(pe - (long long)tile * KS) * kKc);
        const int bm = (tile / tiles) * kWT, bn = (tile % tiles) * kWT;
        const int r0 = bm + ty * 8, c0 = bn + tx * 8;
        int acc[8][8];         // int32 mode
        unsigned acc16[8][4];  // packed mode: columns (c0 + 2p, c0 + 2p + 1)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (U16) {
#pragma unroll
                for (int p = 0; p < 4; ++p) acc16[r][p] = kInfU16x2;
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = kInfI32;
            }
        }
        for (long long v = u; v < pe; ++v) {
            const long long q = qbase + (v - u0);
            const int slot = (int)(q % kWStages);
            if (!mbar_wait(a, &sm.full[slot], (unsigned)((q / kWStages) & 1))) return false;
            const WwStage &st = sm.st[slot];
#pragma unroll 4
            for (int k = 0; k < kKc; ++k) {
                const int4 a0 = *reinterpret_cast<const int4 *>(&st.a[k][ty * 8]);
                const int4 a1 = *reinterpret_cast<const int4 *>(&st.a[k][ty * 8 + 4]);
                const int ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                if (U16) {
                    const uint4 bv = *reinterpret_cast<const uint4 *>(&st.b[k][tx * 4]);
                    const unsigned br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int p = 0; p < 4; ++p) acc16[r][p] = u16x2_addmin((unsigned)ar[r], br[p], acc16[r][p]);
                } else {
                    const int4 b0 = *reinterpret_cast<const int4 *>(&st.b[k][tx * 8]);
                    const int4 b1 = *reinterpret_cast<const int4 *>(&st.b[k][tx * 8 + 4]);
                    const int br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[r][c] = __viaddmin_s32(ar[r], br[c], acc[r][c]);
                }
            }
            __syncwarp();  // the warp is done reading the slot
            if (lane == 0) mbar_arrive(&sm.empty[slot]);
        }
        // merge, with X_{s-1} read row by row now: p < old, or p == old from
        // the piece holding k = j
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = r0 + r;
            int o[8];
            if (i < n && c0 < n) {
                // a vector that starts inside the row ends inside the padded row
                const int4 inf4 = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
                const int4 x0 = __ldcg(reinterpret_cast<const int4 *>(in + (long long)i * ldx + c0));
                const int4 x1 =
                    c0 + 4 < n ? __ldcg(reinterpret_cast<const int4 *>(in + (long long)i * ldx + c0 + 4)) : inf4;
                o[0] = x0.x; o[1] = x0.y; o[2] = x0.z; o[3] = x0.w;
                o[4] = x1.x; o[5] = x1.y; o[6] = x1.z; o[7] = x1.w;
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) o[c] = kInfI32;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = c0 + c;
                int p;
                if (U16) {
                    const unsigned hh = (acc16[r][c >> 1] >> (16 * (c & 1))) & 0xFFFFu;
                    p = hh >= (unsigned)BTAS_INF_U16 ? kInfI32 : (int)hh;
                } else {
                    p = clamp_i32<kMin>(acc[r][c]);
                }
                if (i < n && j < n && p < kInfI32 && (p < o[c] || (p == o[c] && j >= k0 && j < k1))) {
                    atomicMin(out + (long long)i * ldx + j, p);
                    mx = max(mx, p);
                    ch |= p < o[c];
                }
            }
        }
        u = pe;
    }
    return true;
}

__device__ __forceinline__ void mid_wide_body(const MidArgs &a) {
    extern __shared__ __align__(16) unsigned char ww_raw[];
    WwSmem &sm = *reinterpret_cast<WwSmem *>(ww_raw);
    const int n = a.n, tid = threadIdx.x;
    const bool producer = tid >= kWConsumers;
    const long long ldx = a.ldx;
    const long long nx = (long long)n * ldx;
    const long long gthreads = (long long)gridDim.x * kWThreads;
    const long long gtid = (long long)blockIdx.x * kWThreads + tid;
    unsigned gen = 0;
    if (tid == 0) {
        for (int s = 0; s < kWStages; ++s) {
            mbar_init(&sm.full[s], kWProducers / 32);
            mbar_init(&sm.empty[s], kWConsumers / 32);
        }
    }
    __syncthreads();
    // phase 0: domain check, W -> X_0 (buf2), X_1's buffer to INF
    const bool bad_block = mid_phase0(a, gtid, gthreads);
    int nbad = 0, bound = 0;
    if (a.withhold && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier(a, gen, bad_block, a.info + 1, nbad, bound)) return;
    if (nbad != 0) return;  // D untouched

    const int tiles = (n + kWT - 1) / kWT, KS = (n + kKc - 1) / kKc;
    const long long U = (long long)tiles * tiles * KS;
    const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
    const int4 inf4 = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
    const int *in = a.buf2;
    int cur = 0, done = 0, path = 0;
    long long qbase = 0;  // units through this block's ring so far
    for (int s = 1; s <= a.S; ++s) {
        int *out = bufp(a, cur);
        if (s < a.S) {
            int4 *nxt = reinterpret_cast<int4 *>(bufp(a, (cur + 1) % 3));
            for (long long idx = gtid; idx < nx / 4; idx += gthreads) nxt[idx] = inf4;
        }
        const bool u16 = a.u16_ok && bound <= kU16Max;
        path |= u16 ? 4 : 1;
        bool ch = false;
        int mx = 0;
        if (producer) {
            if (u16) ww_produce<true>(a, in, tiles, KS, u0, u1, qbase, sm, tid - kWConsumers);
            else ww_produce<false>(a, in, tiles, KS, u0, u1, qbase, sm, tid - kWConsumers);
        } else {
            if (u16) ww_consume<true>(a, in, out, tiles, KS, u0, u1, qbase, sm, tid, ch, mx);
            else ww_consume<false>(a, in, out, tiles, KS, u0, u1, qbase, sm, tid, ch, mx);
        }
        qbase += u1 - u0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0 && mx > 0) atomicMax(reinterpret_cast<int *>(a.bar + 64 + s), mx);
        int changed = 0;
        if (!grid_barrier(a, gen, ch, reinterpret_cast<const int *>(a.bar + 64 + s), changed, bound)) return;
        done += changed != 0;
        in = out;
        cur = (cur + 1) % 3;
        if (!changed && a.early) break;
    }
    mid_finish(a, in, gtid, gthreads, done, path);
}

// Block 0 leaves the status words in the caller's host-mapped mailbox as it
// exits, on every path (the words are final by then: the domain count
// before the first grid barrier, the timeout status before any block gives
// up, the squarings and representations from block 0 itself), so the
// caller reads them after the stream without a copy.
__device__ __forceinline__ void mid_post(const MidArgs &a) {
    if (a.mailbox == nullptr || blockIdx.x != 0 || threadIdx.x != 0) return;
#pragma unroll
    for (int i = 0; i < 5; ++i) a.mailbox[i] = __ldcg(a.info + i);
    __threadfence_system();
}

__global__ void __launch_bounds__(kThreads, 2) apsp_mid_kernel(const MidArgs a) {
    mid_body(a);
    mid_post(a);
}

__global__ void __launch_bounds__(kWThreads, 1) apsp_mid_wide_kernel(const MidArgs a) {
    mid_wide_body(a);
    mid_post(a);
}
}  // namespace

int apsp_mid_max_n() {
    // largest n btas_apsp sends here: above about 1800 vertices the tiled
    // product kernels have enough tiles to fill the GPU and win (measured:
    // 937 vs 1290 us at n = 1536, 2134 vs 1666 us at 2048);
    // BTAS_APSP_MID_MAX_N overrides it (up to 4096)
    static const int dflt = 1792;
    const char *e = getenv("BTAS_APSP_MID_MAX_N");
    if (!e || !*e) return dflt;
    const int v = atoi(e);
    return v < 0 ? 0 : v > 4096 ? 4096 : v;
}

bool apsp_mid_takes(long long n, int sms) {
    if (n <= apsp_mid_max_n()) return true;
    const char *e = getenv("BTAS_APSP_MID_MAX_N");
    if ((e && *e) || n > 3584 || sms < 1) return false;  // an explicit limit wins
    // the tiled packed squaring: 128 x 256 tiles, one CTA per SM
    const long long tiles = ((n + 127) / 128) * (((n + 1) / 2 + 127) / 128);
    const long long waves = (tiles + sms - 1) / sms;
    return 4 * tiles < 3 * waves * sms;
}

// workspace: three n x ldx matrices, then 512 bytes of barrier words and
// 256 bytes for the status words of a caller that passes info = null
size_t apsp_mid_workspace(long long n, int S) {
    (void)S;
    const size_t mat = ((size_t)n * ((n + 3) & ~3LL) * 4 + 255) & ~size_t(255);
    return 3 * mat + 1024;
}

int *apsp_mid_info(void *ws, long long n) {
    const size_t mat = ((size_t)n * ((n + 3) & ~3LL) * 4 + 255) & ~size_t(255);
    return reinterpret_cast<int *>(static_cast<char *>(ws) + 3 * mat + 512);
}

cudaError_t launch_apsp_mid(const int *W, long long ldw, int n, int S, bool early, bool packed_ok, int *D,
                            long long ldd, void *ws, int *info_out_dev, cudaStream_t st, int *mailbox) {
    // device facts and the kernel's occupancy, queried once per device
    DeviceInfo di{};
    int dev = 0;
    if (!current_device_info(&di, &dev)) return cudaErrorInvalidDevice;
    static std::mutex mu;
    static int cached_per_sm[64];
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && cached_per_sm[dev] > 0) {
            per_sm = cached_per_sm[dev];
        } else {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apsp_mid_kernel, kThreads, 0);
            if (e != cudaSuccess) return e;
            if (dev < 64) cached_per_sm[dev] = per_sm;
        }
    }
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // the wide form from n = 1408 up: measured on GB300 (p = 0.05, w in [1,
    // 100]) it ties the 64 x 64 form at n = 1280 (591 vs 592 us) and is 10 %
    // faster at 1536 (862 vs 955 us) and 1792 (1290 vs 1462 us); at 1024 it is
    // slower (396 vs 341 us).  BTAS_MID_WIDE_MIN_N overrides the boundary.
    const char *wmin = getenv("BTAS_MID_WIDE_MIN_N");
    const bool wide = n >= (wmin && *wmin ? atoi(wmin) : 1408);
    int per_sm_w = 0;
    if (wide) {
        cudaError_t e = set_smem_once(reinterpret_cast<const void *>(apsp_mid_wide_kernel), kWwSmem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_w, apsp_mid_wide_kernel, kWThreads, kWwSmem);
        if (e != cudaSuccess) return e;
        if (per_sm_w < 1) return cudaErrorCooperativeLaunchTooLarge;
    }
    if (S > 63) return cudaErrorInvalidValue;  // per-squaring maxima at bar[64 + s]
    const int sms = di.sms, clk_khz = di.clock_khz;
    const int tile = wide ? kWT : kT;
    const long long tiles = (n + tile - 1) / tile, KS = (n + kKc - 1) / kKc;
    const long long units = tiles * tiles * KS;
    const int grid = (int)std::max(1LL, std::min(units, (long long)(wide ? per_sm_w : per_sm) * sms));
    const long long ldx = (n + 3) & ~3LL;
    const size_t mat = ((size_t)n * ldx * 4 + 255) & ~size_t(255);
    char *base = static_cast<char *>(ws);
    const char *no_u16 = getenv("BTAS_MID_NO_U16");
    MidArgs a{};
    a.W = W;
    a.ldw = ldw;
    a.n = n;
    a.S = S;
    a.early = early ? 1 : 0;
    a.u16_ok = (!packed_ok || (no_u16 && *no_u16 && atoi(no_u16) != 0)) ? 0 : 1;
    const char *wh = getenv("BTAS_MID_WITHHOLD");
    a.withhold = (wh && *wh && atoi(wh) != 0 && grid > 1) ? 1 : 0;
    a.D = D;
    a.ldd = ldd;
    a.ldx = ldx;
    a.buf0 = reinterpret_cast<int *>(base);
    a.buf1 = reinterpret_cast<int *>(base + mat);
    a.buf2 = reinterpret_cast<int *>(base + 2 * mat);
    a.bar = reinterpret_cast<unsigned *>(base + 3 * mat);
    a.info = info_out_dev ? info_out_dev : apsp_mid_info(ws, n);
    a.mailbox = mailbox;
    a.timeout_cycles = (long long)(2.0 * (clk_khz > 0 ? clk_khz : 2000000) * 1e3);  // about 2 s
    // barrier words and per-squaring maxima, and the internal status words
    // when the caller passes none: one memset
    cudaError_t e = cudaMemsetAsync(base + 3 * mat, 0, info_out_dev ? 512 : 768, st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    if (wide)
        e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(apsp_mid_wide_kernel), dim3(grid), dim3(kWThreads),
                                        args, kWwSmem, st);
    else
        e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(apsp_mid_kernel), dim3(grid), dim3(kThreads), args,
                                        0, st);
    note_launch();
    return e;
}

}  // namespace btas
