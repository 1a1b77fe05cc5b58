// APSP by repeated squaring (Sec. III) for mid-size graphs in ONE
// cooperative launch.
//
// Between the one-block kernel (n <= 64) and the tiled product kernels (n >
// 1792; for graphs that fit the edge lists below, n > 4096) a solve is bound
// by launches and host round trips: a few dozen tiles per squaring cannot
// fill the GPU, and every squaring waits for the previous one's change flag.
// Here one cooperative grid runs the domain check and all squarings, with
// ONE grid barrier per squaring.
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
//
// Edge lists (from n = 384, when the workspace has room).  Phase 0 also
// builds per-row lists of W's edges.  When every row fits them, squaring 1
// runs as sparse products over them (sparse_first), and after a squaring
// that lowered few entries a closure certificate (certify) checks
// X_s (x) W >= X_s at the lowered entries only; when it holds, squaring
// s + 1 would change nothing and the solve stops.  Both give the results
// and squaring counts of the literal sequence.
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
    // Edge lists of W (null when the workspace has no room for them): row i's
    // edges (j + 1, W[i][j]), j != i, in lists[i * cap .. i * cap + deg[i]) in
    // no particular order; the other slots are zero.  aux: [0] set if a row has more than cap edges, [1]
    // edges in all, [64 + s] entries that squaring s lowered, counted per
    // piece (an over-estimate).  deg, aux and lists are zeroed by the launch.
    int *deg;
    int2 *lists;
    int *aux;
    int cap;
    int sparse;  // 1: the first squaring from the edge lists when they hold every edge
    int cert;    // 0: never; 1: the closure certificate where the estimate allows; 2: after every changing squaring
    int bail;    // 1: return after phase 0 (D untouched, info[4] = kMidDeclined) unless the lists hold every edge
};

constexpr int kBoundSat = (1 << 29) - 1;  // published values: a bound saturated to 29 bits, and one flag bit
constexpr int kFlagBit = 1 << 29;

struct MidSmem {
    int a[2][kKc][kLdA];  // A stage, k-major: a[k][row]; packed mode: duplicated 16-bit words
    int b[2][kKc][kT];    // B stage: b[k][col]; packed mode: b[k][pair] in the first kT / 2 words
};

__device__ __forceinline__ bool grid_barrier(const MidArgs &a, unsigned &gen, bool flag, const int *pval, int &v0,
                                             int &v1) {
    return btas::grid_barrier(GridSync{a.bar, a.info + 3, a.timeout_cycles}, gen, flag, pval, v0, v1);
}

__device__ __forceinline__ GridSync gsync_of(const MidArgs &a) { return GridSync{a.bar, a.info + 3, a.timeout_cycles}; }

__device__ __forceinline__ int *bufp(const MidArgs &a, int i) { return i == 0 ? a.buf0 : i == 1 ? a.buf1 : a.buf2; }

// Published after phase 0: the largest weight (saturated), and the flag bit
// when there are no usable edge lists (none, or a row longer than cap).
__device__ __forceinline__ unsigned phase0_value(const MidArgs &a) {
    const unsigned mw = (unsigned)gsync::ld_relaxed_i32(a.info + 1);
    const bool no_lists = a.lists == nullptr || gsync::ld_relaxed_i32(a.aux) != 0;
    return min(mw, (unsigned)kBoundSat) | (no_lists ? (unsigned)kFlagBit : 0u);
}

// Published after squaring s: the largest merged value (saturated; only its
// comparison with 16383 matters), and the flag bit when the closure
// certificate should be tried.  On random graphs the squaring that reaches
// the fixpoint follows one that lowered far fewer entries than the one
// before it (3-16 % of it at n = 256 ... 2048, p = 0.02 ... 0.1), while the
// earlier ones lower a similar share (20 % or more).  So the certificate is
// tried when squaring s lowered at most 1/6 as many entries as squaring s - 1
// (all n^2 for s = 1), and its edge-list reads, about (lowered) x (edges / n),
// are at most n^3 / 128.  (The counts are per piece, up to a few times the
// entries; a list read costs the time of about 180 product terms, so a
// certificate that fails costs at most about one squaring.)
__device__ __forceinline__ unsigned squaring_value(const MidArgs &a, int s) {
    const unsigned m = (unsigned)gsync::ld_relaxed_i32(reinterpret_cast<const int *>(a.bar + 64 + s));
    bool c = a.cert == 2;
    if (a.cert == 1 && a.aux != nullptr) {
        const long long n = a.n;
        const long long lowered = gsync::ld_relaxed_i32(a.aux + 64 + s), edges = gsync::ld_relaxed_i32(a.aux + 1);
        const long long before = s > 1 ? gsync::ld_relaxed_i32(a.aux + 64 + s - 1) : n * n;
        c = 6 * lowered <= before && lowered * edges <= n * n * n * n / 128;
    }
    return min(m, (unsigned)kBoundSat) | (c ? (unsigned)kFlagBit : 0u);
}

// A squaring's largest merged value and lowered-entry count, one atomic per warp.
__device__ __forceinline__ void report(const MidArgs &a, int s, int mx, int cnt) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx > 0) atomicMax(reinterpret_cast<int *>(a.bar + 64 + s), mx);
        if (cnt > 0 && a.aux != nullptr) atomicAdd(a.aux + 64 + s, cnt);
    }
}

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
                                         MidSmem &sm, int tid, bool &ch, int &mx, int &cnt) {
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
                cnt += p < o[c];
            }
        }
    }
}

// A block's share [u0, u1) of squaring s, unit u = k-step u % KS of tile
// u / KS, as pieces of consecutive units of one tile.
template <bool U16>
__device__ __forceinline__ void squaring(const MidArgs &a, const int *in, int *out, int tiles, int KS, long long u0,
                                         long long u1, MidSmem &sm, int tid, bool &ch, int &mx, int &cnt) {
    const int n = a.n;
    long long u = u0;
    while (u < u1) {
        const int tile = (int)(u / KS), ks = (int)(u % KS);
        const long long pe = min(u1, (long long)(tile + 1) * KS);
        const int k0 = ks * kKc, k1 = min(n, (int)(pe - (long long)tile * KS) * kKc);
        run_item<U16>(a, in, out, (tile / tiles) * kT, (tile % tiles) * kT, k0, k1, sm, tid, ch, mx, cnt);
        u = pe;
    }
}

// Phase 0 of both forms of the kernel: the domain check, W -> X_0 (buf2) and
// X_1's buffer (buf0) to INF; the entries outside the domain and the largest
// finite weight go to info[0] and info[1].  With edge lists, each warp also
// appends the edges of its 256-column row segments to its row's list (one
// atomicAdd on deg[i] per segment reserves the slots).  Returns whether this
// block found an entry outside the domain.
__device__ __forceinline__ bool mid_phase0(const MidArgs &a, long long gtid, long long gthreads) {
    const int n = a.n, lane = threadIdx.x & 31;
    const long long ldx = a.ldx;
    const int spr = (int)((ldx + 255) / 256);  // segments per row
    const long long nseg = (long long)n * spr, gw = gtid >> 5, nw = gthreads >> 5;
    int bad = 0, mx = 0, edges = 0;
    for (long long sg = gw; sg < nseg; sg += nw) {
        const int i = (int)(sg / spr), c0 = (int)(sg % spr) * 256;
        int v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = c0 + 32 * t + lane;
            v[t] = j < n ? a.W[(long long)i * a.ldw + j] : kInfI32;
        }
        unsigned m[8];
        int tot = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = c0 + 32 * t + lane;
            const bool fin = v[t] >= 0 && v[t] <= BTAS_I32_FINITE_MAX;  // false past column n - 1 (INF)
            if (j < n && ((!fin && v[t] != kInfI32) || (i == j && v[t] != 0))) ++bad;
            if (fin) mx = max(mx, v[t]);
            if (j < ldx) {
                a.buf2[(long long)i * ldx + j] = v[t];
                a.buf0[(long long)i * ldx + j] = kInfI32;
            }
            m[t] = __ballot_sync(0xffffffffu, fin && j != i);
            tot += __popc(m[t]);
        }
        if (a.lists != nullptr && tot > 0) {  // warp-uniform
            int base = 0;
            if (lane == 0) base = atomicAdd(a.deg + i, tot);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lane == 0 && base + tot > a.cap) atomicOr(a.aux, 1);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int q = base + __popc(m[t] & ((1u << lane) - 1u));
                if (((m[t] >> lane) & 1u) && q < a.cap)
                    a.lists[(long long)i * a.cap + q] = make_int2(c0 + 32 * t + lane + 1, v[t]);
                base += __popc(m[t]);
            }
            edges += tot;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        if (bad) atomicAdd(a.info + 0, bad);
        atomicMax(a.info + 1, mx);
        if (edges) atomicAdd(a.aux + 1, edges);
    }
    return __syncthreads_or(bad != 0) != 0;
}

// The rows of this block in the sparse first squaring and the closure
// certificate: an equal contiguous share of the n rows.
__device__ __forceinline__ void block_rows(int n, int &r0, int &r1) {
    r0 = (int)((long long)n * blockIdx.x / gridDim.x);
    r1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);
}

// Up to 64 rows of a block at a time in shared memory, and beside them the
// prefix sums of their degrees (65 words) or a list of entries.
constexpr int kRowsMax = 64;
constexpr int kPfxWords = 128;
// The 64 x 64 form reads 16 edge lists at once (measured against 8: 247.6 vs
// 252.4 us per call at n = 1024, 153.3 vs 155.0 at 768, and 96.1 vs 93.9 at
// 512, where the lists hold about 26 edges; both depths in one kernel spill).

// Rows of a chunk: each takes its X row (ldx words) and, in the sparse
// squaring, its own edge list (2 cap words).
__device__ __forceinline__ int sparse_rows(const MidArgs &a, int smem_words) {
    return min(kRowsMax, (smem_words - kPfxWords) / (int)(a.ldx + 2 * a.cap));
}
__device__ __forceinline__ bool sparse_fits(const MidArgs &a, int smem_words) { return sparse_rows(a, smem_words) >= 1; }
__device__ __forceinline__ bool certify_fits(const MidArgs &a, int smem_words) {
    return (smem_words / 2) / a.ldx >= 1 && smem_words / 2 > kPfxWords;
}

// The first 32 H entries of edge list k, H per lane.  Entries hold (j + 1,
// w) and unused slots are zero, so a list ends at its first zero slot (or at
// cap).
template <int H>
__device__ __forceinline__ void list_head(const MidArgs &a, int k, int lane, int2 (&ev)[H]) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int q = lane + 32 * h;
        ev[h] = q < a.cap ? __ldcg(a.lists + (long long)k * a.cap + q) : make_int2(0, 0);
    }
}

// Squaring 1 from the edge lists.  X_1[i][j] = min over k of X_0[i][k] +
// X_0[k][j]; the terms k = i and k = j are W[i][j] itself, and every other
// finite term is w_ik + w_kj over edges (i, k) and (k, j), at most 2^29, so
// no clamp applies.  A chunk of the block's rows starts as W[i][.] in shared
// memory, beside the rows' own edge lists; the block's warps take the (row,
// k) pairs (warp w: pairs w, w + warps, ...), read the lists of 8 k at once
// with the lanes along each list, and lower the row entries with
// shared-memory atomicMin.  The rows then go to out (whose padding columns
// stay INF), with the change test against X_0, the largest finite entry and
// the count of lowered entries.
template <int IF, int UN, int H>
__device__ __forceinline__ void sparse_first(const MidArgs &a, int *out, int *smem, int smem_words, bool &ch,
                                             int &mx, int &cnt) {
    const int n = a.n, cap = a.cap, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int ldx = (int)a.ldx;
    const int R = sparse_rows(a, smem_words);  // >= 1: checked by the caller
    int *pfx = smem + (smem_words - kPfxWords);
    int ra, rb;
    block_rows(n, ra, rb);
    for (int r0 = ra; r0 < rb; r0 += R) {
        const int nr = min(R, rb - r0);
        int2 *own = reinterpret_cast<int2 *>(smem + nr * ldx);  // nr x cap edges, 8-byte aligned
        // rows of X_0, the rows' own lists and their degrees: all loads in flight together
        const int rwords = nr * ldx, lwords = nr * cap * 2, total = rwords + lwords;
        if (warp == 0) {  // inclusive scan of the degrees: pfx[r + 1] = edges of rows r0 .. r0 + r
            int d0 = lane < nr ? __ldcg(a.deg + r0 + lane) : 0;
            int d1 = lane + 32 < nr ? __ldcg(a.deg + r0 + lane + 32) : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x0 = __shfl_up_sync(0xffffffffu, d0, o), x1 = __shfl_up_sync(0xffffffffu, d1, o);
                if (lane >= o) d0 += x0, d1 += x1;
            }
            d1 += __shfl_sync(0xffffffffu, d0, 31);
            pfx[lane + 1] = d0;
            pfx[lane + 33] = d1;
            if (lane == 0) pfx[0] = 0;
        }
        for (int e0 = 0; e0 < total; e0 += nthr * 4 * UN) {
            int4 w[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e < rwords) w[u] = __ldcg(reinterpret_cast<const int4 *>(a.buf2 + (long long)r0 * ldx + e));
                else if (e < total) w[u] = __ldcg(reinterpret_cast<const int4 *>(a.lists + (long long)r0 * cap) + (e - rwords) / 4);
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e < total) *reinterpret_cast<int4 *>(smem + e) = w[u];
            }
        }
        __syncthreads();
        const int P = pfx[nr];
        for (int g0 = warp; g0 < P; g0 += nwarp * 32) {
            // lane l sets up the warp's pair g0 + nwarp * l from shared memory
            const int p = g0 + nwarp * lane;
            int r = 0, k = 0, wik = 0;
            if (p < P) {
                int lo = 0, hi = nr;  // the row r with pfx[r] <= p < pfx[r + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pfx[mid] <= p) lo = mid;
                    else hi = mid;
                }
                r = lo;
                const int2 e = own[r * cap + (p - pfx[r])];
                k = e.x - 1;
                wik = e.y;
            }
            const int np = min(32, (P - g0 + nwarp - 1) / nwarp);
            for (int t = 0; t < np; t += IF) {
                int2 ev[IF][H];  // the heads of IF lists; the pairs' values are taken again below
#pragma unroll
                for (int u = 0; u < IF; ++u) {
                    const int kk = __shfl_sync(0xffffffffu, k, (t + u) & 31);
                    if (t + u < np) list_head<H>(a, kk, lane, ev[u]);
                    else {
#pragma unroll
                        for (int h = 0; h < H; ++h) ev[u][h] = make_int2(0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < IF; ++u) {
                    const int src = (t + u) & 31;
                    int *row = smem + __shfl_sync(0xffffffffu, r, src) * ldx;
                    const int ww = __shfl_sync(0xffffffffu, wik, src);
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        if (ev[u][h].x > 0) atomicMin(row + ev[u][h].x - 1, ww + ev[u][h].y);
                    // a full head: the rest of the list (warp-uniform test)
                    if (__shfl_sync(0xffffffffu, ev[u][H - 1].x, 31) > 0 && cap > 32 * H) {
                        const int kk = __shfl_sync(0xffffffffu, k, src);
                        const int dk = __ldcg(a.deg + kk);
                        for (int q = 32 * H + lane; q < dk; q += 32) {
                            const int2 e = __ldcg(a.lists + (long long)kk * cap + q);
                            atomicMin(row + e.x - 1, ww + e.y);
                        }
                    }
                }
            }
        }
        __syncthreads();
        for (int e0 = 0; e0 < rwords; e0 += nthr * 4 * UN) {
            int4 o[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e < rwords) o[u] = __ldcg(reinterpret_cast<const int4 *>(a.buf2 + (long long)r0 * ldx + e));
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e >= rwords) continue;
                const int4 v = *reinterpret_cast<const int4 *>(smem + e);
                *reinterpret_cast<int4 *>(out + (long long)r0 * ldx + e) = v;
                const int vv[4] = {v.x, v.y, v.z, v.w}, oo[4] = {o[u].x, o[u].y, o[u].z, o[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (vv[c] < kInfI32) mx = max(mx, vv[c]);
                    if (vv[c] < oo[c]) {
                        ch = true;
                        ++cnt;
                    }
                }
            }
        }
        __syncthreads();  // the chunk's shared memory is reused by the next chunk
    }
}

// Closure certificate after squaring s.  Y = X_s is the closure exactly when
// Y[i][j] <= c(Y[i][k] + W[k][j]) for all i, k, j, with c the clamp of the
// products (sums >= INF - 2^28 become INF): then Y (x) Y = Y, so squaring
// s + 1 would change nothing.  A pair (i, k) that squaring s left unchanged
// satisfies it: Y[i][j] <= c(X_{s-1}[i][k] + X_{s-1}[k][j]) and X_{s-1} <= W.
// So only the entries squaring s lowered are checked, against the edges
// (k, j), j != k, of their column k (j = k adds 0).  The block's rows go to
// shared memory with the list of their lowered entries; the warps take the
// entries (warp w: entries w, w + warps, ...) and read the edge lists of 8
// entries at once along the lanes.  Returns true if this block found a
// violation, or could not hold its list of lowered entries (then it
// certifies nothing).
template <int IF, int UN, int H>
__device__ __forceinline__ bool certify(const MidArgs &a, const int *Y, const int *Xp, int *smem, int smem_words) {
    const int n = a.n, cap = a.cap, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int ldx = (int)a.ldx;
    const int R = min(kRowsMax, (smem_words / 2) / ldx);  // >= 1: checked by the caller
    int *plist = smem + R * ldx;
    const int L = smem_words - R * ldx - kPfxWords;  // list capacity, >= smem_words / 2 - kPfxWords
    int *s_cnt = smem + (smem_words - kPfxWords);
    bool viol = false;
    int ra, rb;
    block_rows(n, ra, rb);
    for (int r0 = ra; r0 < rb; r0 += R) {
        const int nr = min(R, rb - r0);
        if (tid == 0) *s_cnt = 0;
        __syncthreads();
        const int total = nr * ldx;
        for (int e0 = 0; e0 < total; e0 += nthr * 4 * UN) {  // the same trip count in every lane
            int4 y[UN], x[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {  // all loads in flight first
                const int e = e0 + (u * nthr + tid) * 4;
                y[u] = x[u] = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
                if (e < total) {
                    const long long g = (long long)r0 * ldx + e;
                    y[u] = __ldcg(reinterpret_cast<const int4 *>(Y + g));
                    x[u] = __ldcg(reinterpret_cast<const int4 *>(Xp + g));
                }
            }
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e < total) *reinterpret_cast<int4 *>(smem + e) = y[u];
                const int yy[4] = {y[u].x, y[u].y, y[u].z, y[u].w}, xx[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool low = yy[c] < xx[c];
                    const unsigned m = __ballot_sync(0xffffffffu, low);
                    int base = 0;
                    if (lane == 0 && m) base = atomicAdd(s_cnt, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const int q = base + __popc(m & ((1u << lane) - 1u));
                    if (low && q < L) plist[q] = e + c;
                }
            }
        }
        __syncthreads();
        const int P = *s_cnt;
        if (P > L) viol = true;  // the list did not fit: no certificate from this block
        const int PP = P > L ? 0 : P;
        for (int g0 = warp; g0 < PP; g0 += nwarp * 32) {  // as in sparse_first
            const int p = g0 + nwarp * lane;
            const int idx = p < PP ? plist[p] : 0;
            const int np = min(32, (PP - g0 + nwarp - 1) / nwarp);
            for (int t = 0; t < np; t += IF) {
                int2 ev[IF][H];
#pragma unroll
                for (int u = 0; u < IF; ++u) {
                    const int k = __shfl_sync(0xffffffffu, idx, (t + u) & 31) % ldx;
                    if (t + u < np) list_head<H>(a, k, lane, ev[u]);
                    else {
#pragma unroll
                        for (int h = 0; h < H; ++h) ev[u][h] = make_int2(0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < IF; ++u) {
                    const int ii = __shfl_sync(0xffffffffu, idx, (t + u) & 31);
                    const int k = ii % ldx;
                    const int *row = smem + (ii - k);
                    const int yk = smem[ii];
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        if (ev[u][h].x > 0) {
                            const int sum = yk + ev[u][h].y;
                            viol |= sum < kClampI32 && sum < row[ev[u][h].x - 1];
                        }
                    }
                    if (__shfl_sync(0xffffffffu, ev[u][H - 1].x, 31) > 0 && cap > 32 * H) {  // a full head
                        const int dk = __ldcg(a.deg + k);
                        for (int q = 32 * H + lane; q < dk; q += 32) {
                            const int2 e = __ldcg(a.lists + (long long)k * cap + q);
                            const int sum = yk + e.y;
                            viol |= sum < kClampI32 && sum < row[e.x - 1];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    return viol;
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

    // phase 0: domain check, W -> X_0 (buf2), X_1's buffer to INF, edge lists
    const bool bad_block = mid_phase0(a, gtid, gthreads);
    int nbad = 0, v = 0;
    if (a.withhold && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier_fn(gsync_of(a), gen, bad_block, [&a]() { return phase0_value(a); }, nbad, v)) return;
    if (nbad != 0) return;  // D untouched
    int bound = v & kBoundSat;  // >= every finite entry of X_{s-1}
    const bool lists_ok = (v & kFlagBit) == 0;
    if (a.bail && !lists_ok) {  // too dense for the edge lists: the caller takes the tiled kernels
        if (blockIdx.x == 0 && threadIdx.x == 0) a.info[4] = kMidDeclined;
        return;
    }
    int *smem = reinterpret_cast<int *>(&sm);
    constexpr int smem_words = (int)(sizeof(MidSmem) / 4);

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
        const bool sparse = s == 1 && lists_ok && a.sparse && sparse_fits(a, smem_words);
        const bool u16 = a.u16_ok && bound <= kU16Max;
        path |= sparse ? 8 : u16 ? 4 : 1;
        bool ch = false;
        int mx = 0, cnt = 0;
        if (sparse)
            sparse_first<16, 2, 2>(a, out, smem, smem_words, ch, mx, cnt);
        else if (u16)
            squaring<true>(a, in, out, tiles, KS, u0, u1, sm, tid, ch, mx, cnt);
        else
            squaring<false>(a, in, out, tiles, KS, u0, u1, sm, tid, ch, mx, cnt);
        report(a, s, mx, cnt);
        int changed = 0;
        if (!grid_barrier_fn(gsync_of(a), gen, ch, [&a, s]() { return squaring_value(a, s); }, changed, v)) return;
        bound = v & kBoundSat;
        done += changed != 0;
        const int *prev = in;
        in = out;
        cur = (cur + 1) % 3;
        if (!changed && a.early) break;
        if ((v & kFlagBit) && lists_ok && a.early && s < a.S && certify_fits(a, smem_words)) {
            const bool viol = certify<16, 2, 2>(a, in, prev, smem, smem_words);
            int any = 0, unused = 0;
            if (!grid_barrier(a, gen, viol, nullptr, any, unused)) return;
            if (!any) break;  // X_s is the closure: squaring s + 1 would change nothing
        }
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
                                           long long u1, long long qbase, WwSmem &sm, int tid, bool &ch, int &mx,
                                           int &cnt) {
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
                    cnt += p < o[c];
                }
            }
        }
        u = pe;
    }
    return true;
}

extern __shared__ __align__(16) unsigned char ww_raw[];  // the wide form's dynamic shared memory

// The wide form's certificate and the grid barrier that combines it (barrier
// number gen + 1), on the ring's stages: 1 if X_s is the closure, 0 if not,
// -1 if the barrier gave up (status set).  Not inlined: it runs at most a few
// times per solve, and inside the squaring loop its code would take
// registers from the products.
__device__ __noinline__ int certify_step_wide(const MidArgs &a, unsigned gen, const int *Y, const int *Xp) {
    int *smem = reinterpret_cast<int *>(reinterpret_cast<WwSmem *>(ww_raw)->st);
    const bool viol = certify<8, 1, 4>(a, Y, Xp, smem, (int)(sizeof(WwStage) * kWStages / 4));
    int any = 0, unused = 0;
    if (!grid_barrier(a, gen, viol, nullptr, any, unused)) return -1;
    return any ? 0 : 1;
}

__device__ __forceinline__ void mid_wide_body(const MidArgs &a) {
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
    // phase 0: domain check, W -> X_0 (buf2), X_1's buffer to INF, edge lists
    const bool bad_block = mid_phase0(a, gtid, gthreads);
    int nbad = 0, v = 0;
    if (a.withhold && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier_fn(gsync_of(a), gen, bad_block, [&a]() { return phase0_value(a); }, nbad, v)) return;
    if (nbad != 0) return;  // D untouched
    int bound = v & kBoundSat;
    const bool lists_ok = (v & kFlagBit) == 0;
    if (a.bail && !lists_ok) {  // too dense for the edge lists: the caller takes the tiled kernels
        if (blockIdx.x == 0 && threadIdx.x == 0) a.info[4] = kMidDeclined;
        return;
    }
    constexpr int smem_words = (int)(sizeof(WwStage) * kWStages / 4);  // the ring's stages, idle between squarings

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
        const bool sparse = s == 1 && lists_ok && a.sparse && sparse_fits(a, smem_words);
        const bool u16 = a.u16_ok && bound <= kU16Max;
        path |= sparse ? 8 : u16 ? 4 : 1;
        bool ch = false;
        int mx = 0, cnt = 0;
        if (sparse) {
            sparse_first<8, 1, 4>(a, out, reinterpret_cast<int *>(sm.st), smem_words, ch, mx, cnt);
        } else {
            if (producer) {
                if (u16) ww_produce<true>(a, in, tiles, KS, u0, u1, qbase, sm, tid - kWConsumers);
                else ww_produce<false>(a, in, tiles, KS, u0, u1, qbase, sm, tid - kWConsumers);
            } else {
                if (u16) ww_consume<true>(a, in, out, tiles, KS, u0, u1, qbase, sm, tid, ch, mx, cnt);
                else ww_consume<false>(a, in, out, tiles, KS, u0, u1, qbase, sm, tid, ch, mx, cnt);
            }
            qbase += u1 - u0;  // units through the ring
        }
        report(a, s, mx, cnt);
        int changed = 0;
        if (!grid_barrier_fn(gsync_of(a), gen, ch, [&a, s]() { return squaring_value(a, s); }, changed, v)) return;
        bound = v & kBoundSat;
        done += changed != 0;
        const int *prev = in;
        in = out;
        cur = (cur + 1) % 3;
        if (!changed && a.early) break;
        if ((v & kFlagBit) && lists_ok && a.early && s < a.S && certify_fits(a, smem_words)) {
            const int c = certify_step_wide(a, gen++, in, prev);
            if (c < 0) return;
            if (c > 0) break;  // X_s is the closure: squaring s + 1 would change nothing
        }
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
    // largest n btas_apsp always sends here (and the server's whole solves
    // and the allocation-free entry point): above it, with 128 x 256 tiles
    // enough to fill the GPU, the tiled kernels win on dense graphs, and
    // btas_apsp keeps only graphs sparse enough for the edge lists here (up
    // to kMidSparseMaxN, see apsp_mid_takes); BTAS_APSP_MID_MAX_N overrides
    // it (up to 4096) and then is a plain limit
    static const int dflt = 1792;
    const char *e = getenv("BTAS_APSP_MID_MAX_N");
    if (!e || !*e) return dflt;
    const int v = atoi(e);
    return v < 0 ? 0 : v > 4096 ? 4096 : v;
}

bool apsp_mid_takes(long long n, int sms) {
    (void)sms;
    if (n <= apsp_mid_max_n()) return true;
    const char *e = getenv("BTAS_APSP_MID_MAX_N");
    if (e && *e) return false;  // an explicit limit wins
    return n <= kMidSparseMaxN;  // launched with bail_dense: dense graphs go to the tiled kernels
}

// workspace: three n x ldx matrices, then 512 bytes of barrier words and
// 256 bytes for the status words of a caller that passes info = null (the
// minimum); then 1 KiB of aux words, the row degrees and the edge lists.
namespace {
size_t mid_mat_bytes(long long n) { return ((size_t)n * ((n + 3) & ~3LL) * 4 + 255) & ~size_t(255); }
size_t mid_deg_bytes(long long n) { return ((size_t)n * 4 + 255) & ~size_t(255); }
}  // namespace

// Edges per row the lists hold: n / 4 rounded up to a multiple of 32, in [32,
// 256] (a first squaring with more edges per row gains little from them);
// BTAS_MID_LIST_CAP overrides it (tests), rounded up to an even number so
// that every row's list starts on a 16-byte boundary.
int apsp_mid_list_cap(long long n) {
    const char *e = getenv("BTAS_MID_LIST_CAP");
    if (e && *e) {
        const int v = atoi(e);
        return v < 2 ? 2 : v > 4096 ? 4096 : (v + 1) & ~1;
    }
    const long long c = ((n / 4 + 31) / 32) * 32;
    return (int)std::min(256LL, std::max(32LL, c));
}

size_t apsp_mid_workspace_min(long long n) { return 3 * mid_mat_bytes(n) + 1024; }

size_t apsp_mid_workspace(long long n, int S) {
    (void)S;
    return 3 * mid_mat_bytes(n) + 2048 + mid_deg_bytes(n) + (size_t)n * (size_t)apsp_mid_list_cap(n) * 8;
}

int *apsp_mid_info(void *ws, long long n) {
    return reinterpret_cast<int *>(static_cast<char *>(ws) + 3 * mid_mat_bytes(n) + 512);
}

cudaError_t launch_apsp_mid(const int *W, long long ldw, int n, int S, bool early, bool packed_ok, int *D,
                            long long ldd, void *ws, size_t ws_bytes, int *info_out_dev, cudaStream_t st,
                            int *mailbox, bool bail_dense) {
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
    const size_t mat = mid_mat_bytes(n);
    char *base = static_cast<char *>(ws);
    // The edge lists (sparse first squaring, closure certificate) from n =
    // 384 (BTAS_MID_LISTS_MIN_N): below it a squaring is a few microseconds,
    // bound by the grid barrier, and the list reads cost as much as they save.
    const char *lmin = getenv("BTAS_MID_LISTS_MIN_N");
    const bool lists = ws_bytes >= apsp_mid_workspace(n, S) && n >= (lmin && *lmin ? atoi(lmin) : 384);
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
    // BTAS_MID_NO_SPARSE, BTAS_MID_NO_CERT: the first squaring dense, no
    // closure certificate; BTAS_MID_CERT_ALWAYS: the certificate after every
    // changing squaring (tests)
    const char *no_sp = getenv("BTAS_MID_NO_SPARSE"), *no_ce = getenv("BTAS_MID_NO_CERT"),
               *ce_all = getenv("BTAS_MID_CERT_ALWAYS");
    a.cap = apsp_mid_list_cap(n);
    a.aux = lists ? reinterpret_cast<int *>(base + 3 * mat + 1024) : nullptr;
    a.deg = lists ? reinterpret_cast<int *>(base + 3 * mat + 2048) : nullptr;
    a.lists = lists ? reinterpret_cast<int2 *>(base + 3 * mat + 2048 + mid_deg_bytes(n)) : nullptr;
    a.sparse = (no_sp && *no_sp && atoi(no_sp) != 0) ? 0 : 1;
    a.cert = (no_ce && *no_ce && atoi(no_ce) != 0) ? 0 : (ce_all && *ce_all && atoi(ce_all) != 0) ? 2 : 1;
    a.bail = bail_dense && lists && a.sparse ? 1 : 0;
    // barrier words and per-squaring maxima, the internal status words when
    // the caller passes none, and with edge lists the aux words, degrees and
    // lists: one memset
    const size_t zero = lists ? apsp_mid_workspace(n, S) - 3 * mat : info_out_dev ? 512 : 768;
    cudaError_t e = cudaMemsetAsync(base + 3 * mat, 0, zero, st);
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
