// Batched tropical products and APSP solves in one persistent launch.
//
// Many independent problems of uneven size (APSP by repeated squaring,
// Sec. III, and single tropical products) are cut into 128 x 128 tile tasks.
// Tasks are ordered by level -- level 0: transposes into the k-contiguous
// B-operand layout; level s >= 1: the tiles of squaring s (a product has one
// level) -- and, within a level, by instance, largest first.  Persistent CTAs
// claim tasks from one global counter.  A task of level s waits until every
// task of level s-1 of its own instance is done (a per-(instance, level)
// completion counter).  Tasks are claimed in level order, so every task a CTA
// waits on was claimed earlier by a CTA that is running: the schedule cannot
// deadlock, and no co-residency assumption is needed.  Every wait is bounded
// (clock64 budget); on expiry the CTA records BTAS_ERR_TIMEOUT in a device
// status word and stops, and the other CTAs see the word and stop too.
//
// An APSP squaring tile also stores its output transposed (through shared
// memory), so the next squaring finds its B operand ready.  Early exit: the
// first squaring whose predecessor changed nothing copies that fixpoint into
// D, and the squarings after it do nothing (the result is unchanged).
// Closure certificate (graphs of n >= 256): level 0 also builds W's edge
// lists, and after squarings 2 .. S-1 certificate tasks, placed after all of
// their level's tiles, check X_s (x) W >= X_s at the entries squaring s
// lowered; when every block passes, squaring s + 1 copies X_s forward
// instead of computing it, and the early exit finishes the solve.  The
// launch (counter reset + kernel) is captured once in a CUDA graph and
// replayed.
#include <algorithm>
#include <map>
#include <tuple>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "batch_kernel.cuh"
#include "kernels.h"
#include "tgemm.cuh"
#include "u16_tile.cuh"

namespace btas {

using BCfg = TileCfg<128, 128, 32, 3, 2, 2, 1>;  // 2 CTAs/SM, <= 128 registers
// the small output tile: 64 x 64, 4 x 4 outputs per thread, same 256 threads
using BCfgS = TileCfg<kBTSmall, kBTSmall, 32, 3, 2, 2, 1, 4, 4>;
static_assert(BCfgS::kThreads == BCfg::kThreads, "both task tiles run on the same CTA");

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kListRows = 32;  // rows of W per edge-list task (4 per warp)

// The persistent kernel's dynamic shared memory, in words: a product tile's
// stages or a 128 x 128 transpose, whichever is larger.
__host__ __device__ constexpr int batch_smem_words() {
    return (BCfg::kSmemBytes > kBT * (kBT + 1) * 4 ? BCfg::kSmemBytes : kBT * (kBT + 1) * 4) / 4;
}

__host__ __device__ __forceinline__ int list_tasks(const BInst &I) { return (I.n + kListRows - 1) / kListRows; }
constexpr int kCertRows = 64;  // rows of D per certificate task, checked in chunks of cert_rows
__host__ __device__ __forceinline__ int cert_tasks(const BInst &I) {
    return I.cert_rows > 0 ? (I.n + kCertRows - 1) / kCertRows : 0;
}

// Certificate tasks follow squarings 2 .. levels - 1 (after the first one
// nearly every entry is lowered, and the last one ends the solve anyway).
__host__ __device__ __forceinline__ bool has_cert(const BInst &I, int level) {
    return I.cert && level >= 2 && level < I.levels;
}

// Tasks of an instance's level: level 0 the transposes (and an APSP's edge
// lists), level s >= 1 the output tiles (and, after an APSP squaring s <
// levels, the certificate tasks).
__device__ __forceinline__ int tasks_at(const BInst &I, int level) {
    if (level == 0)
        return (I.t0_rows > 0 ? ((I.t0_rows + kBT - 1) / kBT) * ((I.t0_cols + kBT - 1) / kBT) : 0) +
               (I.cert ? list_tasks(I) : 0);
    return I.tiles_m * I.tiles_n + (has_cert(I, level) ? cert_tasks(I) : 0);
}

// Edge lists of rows 32 t .. 32 t + 31 of W, four rows per warp: row i's
// edges (j + 1, w) in lists[i * cap ..] in column order, then zeros up to
// cap, and deg[i]; a row with more than cap edges sets *ovf.
__device__ __forceinline__ void lists_task(const BInst &I, int t, int tid, int *ovf) {
    const int lane = tid & 31, warp = tid >> 5, n = I.n, cap = I.cap;
    const int *W = static_cast<const int *>(I.A);
    for (int q = 0; q < kListRows / 8; ++q) {
        const int i = t * kListRows + warp * (kListRows / 8) + q;
        if (i >= n) break;  // warp-uniform
        int2 *L = I.lists + (long long)i * cap;
        int cnt = 0;
        for (int j0 = 0; j0 < n; j0 += 256) {
            int v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + 32 * u + lane;
                v[u] = j < n ? __ldg(W + (long long)i * I.lda + j) : kInfI32;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + 32 * u + lane;
                const bool e = j != i && v[u] >= 0 && v[u] <= BTAS_I32_FINITE_MAX;  // false past n - 1
                const unsigned m = __ballot_sync(0xffffffffu, e);
                const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (e && pos < cap) L[pos] = make_int2(j + 1, v[u]);
                cnt += __popc(m);
            }
        }
        for (int q2 = cnt + lane; q2 < cap; q2 += 32) L[q2] = make_int2(0, 0);
        if (lane == 0) {
            I.deg[i] = cnt;
            if (cnt > cap) atomicOr(ovf, 1);
        }
    }
}

// Closure certificate after squaring s >= 2 over rows 64 t .. 64 t + 63, in
// chunks of R = cert_rows rows: Y = D_s is the closure exactly when Y[i][j]
// <= c(Y[i][k] + W[k][j]) for all i, k, j (c: the products' clamp); pairs
// (i, k) that squaring s left unchanged satisfy it (Y[i][j] <= c(D_{s-1}[i][k]
// + D_{s-1}[k][j]) and D_{s-1} <= W), so only the lowered entries are
// checked, against the edges of column k.  Returns true (for every thread)
// on a violation, when a chunk's lowered entries exceed an eighth of its
// entries or the shared list, or when another task of this level has failed
// already (*failed): then it certifies nothing.
__device__ __forceinline__ bool cert_task(const BInst &I, int s, int t, int *smem, int smem_words, int tid,
                                          const int *failed) {
    const int n = I.n, cap = I.cap, ldx = (int)I.ldx, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int R = I.cert_rows;
    // s >= 2: D_s and D_{s-1} both live in X0 / X1 with the 16-byte pitch ldx
    const int *Y = static_cast<const int *>((s & 1) ? I.X0 : I.X1);
    const int *Xp = static_cast<const int *>((s & 1) ? I.X1 : I.X0);
    int *plist = smem + R * ldx;
    int *s_cnt = smem + (smem_words - 32);
    const int rend = min(n, (t + 1) * kCertRows);
    bool viol = false;
    for (int r0 = t * kCertRows; r0 < rend && !viol; r0 += R) {
        const int nr = min(R, rend - r0);
        const int L = min(smem_words - R * ldx - 32, nr * n / 8);
        if (tid == 0) {
            *s_cnt = 0;
            s_cnt[1] = ld_acquire(failed);  // another task of this level failed already: stop
        }
        __syncthreads();
        if (s_cnt[1] != 0) {  // s_cnt[1] is not written again before the next barrier
            viol = true;
            break;
        }
        const int total = nr * ldx;  // padding columns (n .. ldx - 1) are never written: masked below
        for (int e0 = 0; e0 < total; e0 += nthr * 16) {  // the same trip count in every lane
            int4 y[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {  // all loads in flight first
                const int e = e0 + (u * nthr + tid) * 4;
                y[u] = x[u] = make_int4(kInfI32, kInfI32, kInfI32, kInfI32);
                if (e < total) {
                    y[u] = __ldcg(reinterpret_cast<const int4 *>(Y + (long long)r0 * ldx + e));
                    x[u] = __ldcg(reinterpret_cast<const int4 *>(Xp + (long long)r0 * ldx + e));
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + (u * nthr + tid) * 4;
                if (e < total) *reinterpret_cast<int4 *>(smem + e) = y[u];
                const int col = e % ldx;  // a 16-byte vector stays inside its row (ldx % 4 == 0)
                const int yy[4] = {y[u].x, y[u].y, y[u].z, y[u].w}, xx[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool low = col + c < n && yy[c] < xx[c];
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
        viol = P > L;
        const int PP = viol ? 0 : P;
        bool v = false;
        for (int g0 = warp; g0 < PP; g0 += nwarp * 32) {  // warp w: entries w, w + warps, ...
            const int p = g0 + nwarp * lane;
            const int idx = p < PP ? plist[p] : 0;
            const int np = min(32, (PP - g0 + nwarp - 1) / nwarp);
            for (int t0 = 0; t0 < np; t0 += 8) {
                int2 ev[8][2];  // the first 64 entries of 8 lists
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = __shfl_sync(0xffffffffu, idx, (t0 + u) & 31) % ldx;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q = lane + 32 * h;
                        ev[u][h] =
                            (t0 + u < np && q < cap) ? __ldcg(I.lists + (long long)k * cap + q) : make_int2(0, 0);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int ii = __shfl_sync(0xffffffffu, idx, (t0 + u) & 31);
                    const int k = ii % ldx;
                    const int *row = smem + (ii - k);
                    const int yk = smem[ii];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (ev[u][h].x > 0) {
                            const int sum = yk + ev[u][h].y;
                            v |= sum < kClampI32 && sum < row[ev[u][h].x - 1];
                        }
                    }
                    if (__shfl_sync(0xffffffffu, ev[u][1].x, 31) > 0 && cap > 64) {  // a full head: the rest
                        const int dk = __ldcg(I.deg + k);
                        for (int q = 64 + lane; q < dk; q += 32) {
                            const int2 e = __ldcg(I.lists + (long long)k * cap + q);
                            const int sum = yk + e.y;
                            v |= sum < kClampI32 && sum < row[e.x - 1];
                        }
                    }
                }
            }
        }
        viol = __syncthreads_or((viol || v) ? 1 : 0) != 0;  // also: the chunk's shared memory is free again
    }
    return viol;
}

// 128 x 128 transpose of a 4-byte matrix through shared memory.  With Cd /
// Cu it also stores the tile's packed 16-bit forms (row-major, not
// transposed) and reports the largest finite int32 entry to *maxfin.
__device__ __forceinline__ void transpose_tile(const uint32_t *src, long long lds, int rows, int cols, uint32_t *dst,
                                               long long ldd, int tile, uint32_t *sm, int tid,
                                               uint32_t *Cd = nullptr, uint16_t *Cu = nullptr, long long ldcd = 0,
                                               long long ldcu = 0, int *maxfin = nullptr) {
    const int tiles_c = (cols + kBT - 1) / kBT;
    const int r0 = (tile / tiles_c) * kBT, c0 = (tile % tiles_c) * kBT;
    int mx = -1;
    // loads in batches of 16 per thread (coalesced along rows), so several
    // are in flight before the shared-memory and 16-bit-form stores
    constexpr int PER = kBT * kBT / BCfg::kThreads, BATCH = 16;
    static_assert(PER % BATCH == 0, "whole batches");
#pragma unroll 1
    for (int b0 = 0; b0 < PER; b0 += BATCH) {
        uint32_t v[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int idx = tid + (b0 + u) * BCfg::kThreads;
            const int r = idx / kBT, c = idx % kBT;
            v[u] = (r0 + r < rows && c0 + c < cols) ? __ldcg(src + (long long)(r0 + r) * lds + c0 + c) : 0u;
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int idx = tid + (b0 + u) * BCfg::kThreads;
            const int r = idx / kBT, c = idx % kBT;
            if (r0 + r < rows && c0 + c < cols) {
                sm[c * (kBT + 1) + r] = v[u];
                if (Cd != nullptr) {
                    const int iv = static_cast<int>(v[u]);
                    const uint32_t h = iv >= BTAS_INF_U16 ? BTAS_INF_U16 : (uint32_t)iv;
                    Cd[(long long)(r0 + r) * ldcd + c0 + c] = h * 0x10001u;
                    Cu[(long long)(r0 + r) * ldcu + c0 + c] = (uint16_t)h;
                    if (iv < kInfI32) mx = max(mx, iv);
                }
            }
        }
    }
    if (maxfin != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0 && mx >= 0) atomicMax(maxfin, mx);
    }
    __syncthreads();
    for (int idx = tid; idx < kBT * kBT; idx += BCfg::kThreads) {
        const int c = idx / kBT, r = idx % kBT;
        if (r0 + r < rows && c0 + c < cols) dst[(long long)(c0 + c) * ldd + r0 + r] = sm[c * (kBT + 1) + r];
    }
    __syncthreads();
}

// One output tile of a product or an int32 squaring, of either task tile
// size (the IMAD path on half of the thread's columns, as in the
// standalone kernels).
template <int VAR, int SR>
__device__ __forceinline__ bool gemm_tile(bool small, const GemmArgs &a, int bm, int bn, unsigned char *smem, int tid,
                                          void *Ct = nullptr, long long ldct = 0, uint32_t *Cd = nullptr,
                                          long long ldcd = 0, uint16_t *Cu = nullptr, long long ldcu = 0) {
    if (small) return nt_tile<BCfgS, VAR, SR, 2>(a, bm, bn, smem, tid, Ct, ldct, Cd, ldcd, Cu, ldcu);
    return nt_tile<BCfg, VAR, SR, 4>(a, bm, bn, smem, tid, Ct, ldct, Cd, ldcd, Cu, ldcu);
}

__device__ __forceinline__ void copy_task_tile(bool small, const GemmArgs &a, int bm, int bn, int tid) {
    if (small) copy_tile<BCfgS, int>(a, bm, bn, tid);
    else copy_tile<BCfg, int>(a, bm, bn, tid);
}

__device__ __forceinline__ bool u16_task_tile(bool small, const U16Tile &u, int bm, int bn, unsigned char *smem,
                                              int tid) {
    if (small) return u16_tile_t<u16t::Small>(u, bm, bn, smem, tid);
    return u16_tile_t<u16t::Big>(u, bm, bn, smem, tid);
}

__global__ void __launch_bounds__(BCfg::kThreads, BCfg::MINB) batch_kernel(const BatchParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task[4];
    __shared__ int s_flag;
    __shared__ int s_flag2;
    __shared__ int s_closed;
    __shared__ int s_m;
    __shared__ long long s_wait;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(p.next, 1);
            int4 w = make_int4(-1, 0, 0, 0);
            if (t < p.total && ld_acquire(p.status) == 0) w = p.tasks[t];
            s_task[0] = w.x; s_task[1] = w.y; s_task[2] = w.z; s_task[3] = w.w;
            s_flag = 1;
            s_flag2 = 1;
            s_closed = 0;
            s_m = 0x7FFFFFFF;
            s_wait = 0;
            if (w.x >= 0 && w.z > 0) {
                // wait until every task of the previous level of this instance
                // is done; a certificate task waits for the output tiles of its
                // own level (claimed before it)
                const BInst &I = p.insts[w.y];
                const bool cert = w.x == kTaskCert;
                const int need = (cert ? I.tiles_m * I.tiles_n : tasks_at(I, w.z - 1)) +
                                 (w.y == p.withhold_inst ? 1 : 0);
                const int *cnt = p.done + I.done_base + w.z - (cert ? 0 : 1);
                const long long t0 = clock64();
                while (ld_acquire(cnt) < need) {
                    if (ld_acquire(p.status) != 0) { s_task[0] = -1; break; }
                    if (clock64() - t0 > p.timeout_cycles) {
                        atomicCAS(p.status, 0, BTAS_ERR_TIMEOUT);
                        s_task[0] = -1;
                        break;
                    }
                    __nanosleep(200);
                }
                s_wait = clock64() - t0;
                if (s_task[0] >= 0 && cert) {
                    // squaring w.z changed something, and the lists hold every edge
                    s_flag = ld_acquire(p.changed + I.flag_base + w.z);
                    s_flag2 = ld_acquire(p.certfail + I.flag_base);
                } else {
                    if (s_task[0] >= 0 && I.kind == kInstApsp && w.z >= 2)
                        s_flag = ld_acquire(p.changed + I.flag_base + w.z - 1);
                    if (s_task[0] >= 0 && I.kind == kInstApsp && w.z >= 3)
                        s_flag2 = ld_acquire(p.changed + I.flag_base + w.z - 2);
                    if (s_task[0] >= 0 && I.kind == kInstApsp) s_m = ld_acquire(p.maxfin + I.flag_base + w.z - 1);
                    // the certificate after squaring w.z - 1 held
                    if (s_task[0] >= 0 && I.kind == kInstApsp && has_cert(I, w.z - 1))
                        s_closed = ld_acquire(p.certfail + I.flag_base + w.z - 1) == 0 ? 1 : 0;
                }
            }
        }
        __syncthreads();
        const int type = s_task[0], inst = s_task[1], level = s_task[2], tile = s_task[3];
        const int prev_changed = s_flag;
        const int prev_changed2 = s_flag2;
        const int prev_closed = s_closed;
        const int prev_max = s_m;
        __syncthreads();
        if (type < 0) break;
        const long long t_task = clock64();
        int slot = BTAS_BATCH_SLOT_COPY;
        const BInst I = p.insts[inst];
        const bool small = I.tile == kBTSmall;
        const int TT = small ? kBTSmall : kBT;  // output tile edge of this instance
        bool ch = false;
        if (type == kTaskTranspose) {
            slot = BTAS_BATCH_SLOT_TRANSPOSE;
            const uint32_t *src = static_cast<const uint32_t *>(I.kind == kInstGemm ? I.B : I.A);
            const long long lds = I.kind == kInstGemm ? I.ldb : I.lda;
            const bool forms = (I.kind == kInstApsp && I.use_u16) || (I.kind == kInstSquare && I.use_u16 == 2);
            transpose_tile(src, lds, I.t0_rows, I.t0_cols, static_cast<uint32_t *>(I.Q0), I.ldq, tile,
                           reinterpret_cast<uint32_t *>(smem_raw), tid, forms ? I.Ad0 : nullptr,
                           forms ? I.U0 : nullptr, I.ldq, I.ldu,
                           (forms && I.kind == kInstApsp) ? p.maxfin + I.flag_base : nullptr);
        } else if (type == kTaskLists) {
            slot = BTAS_BATCH_SLOT_LISTS;
            lists_task(I, tile, tid, p.certfail + I.flag_base);
        } else if (type == kTaskCert) {
            slot = BTAS_BATCH_SLOT_CERT;
            // prev_changed: squaring `level` changed something; prev_changed2:
            // a row had more edges than the lists hold.  Unchanged: the next
            // level copies the fixpoint anyway.
            if (prev_changed) {
                const bool fail = prev_changed2 != 0 || cert_task(I, level, tile, reinterpret_cast<int *>(smem_raw),
                                                                  batch_smem_words(), tid,
                                                                  p.certfail + I.flag_base + level);
                if (fail && tid == 0) atomicOr(p.certfail + I.flag_base + level, 1);
            }
        } else if (type == kTaskCopy) {
            // n <= 2: D = W
            const int bm = (tile / I.tiles_n) * TT, bn = (tile % I.tiles_n) * TT;
            GemmArgs a{};
            a.m = I.n; a.n = I.n;
            a.prev = I.A; a.ldp = I.lda;
            a.C = I.C; a.ldc = I.ldc;
            copy_task_tile(small, a, bm, bn, tid);
        } else if (type == kTaskApsp) {
            const int S = I.levels, s = level;  // squaring s (1-based) of S
            // D_1..D_{S-1} alternate between X0 and X1 (aligned pitch ldx);
            // the last squaring writes D
            const void *cur = s == 1 ? I.A : ((s - 1) & 1 ? I.X0 : I.X1);
            const long long ldcur = s == 1 ? I.lda : I.ldx;
            void *out = s == S ? I.C : (s & 1 ? I.X0 : I.X1);
            const int bm = (tile / I.tiles_n) * TT, bn = (tile % I.tiles_n) * TT;
            GemmArgs a{};
            a.m = a.n = a.k = I.n;
            a.A = cur; a.lda = ldcur;
            a.Bt = (s & 1) ? I.Q0 : I.Q1; a.ldb = I.ldq;
            a.C = out; a.ldc = s == S ? I.ldc : I.ldx;
            a.prev = cur; a.ldp = ldcur;
            a.one = 1;
            a.vec_a = ((reinterpret_cast<uintptr_t>(cur) & 15) == 0) && ((ldcur & 3) == 0);
            a.vec_b = 1;
            a.ro_a = s == 1;  // W; later iterates are written by this launch
            // forms of D_{s-1} are in set (s-1) & 1, D_s goes to set s & 1
            const bool more = s < S && I.use_u16;
            // every finite entry of D_s is <= 2 max(D_{s-1}); if even 4 max(D_{s-1})
            // < 0x7FFF, squaring s+1 is certain to run packed and needs no
            // transposed int32 operand
            const bool next_u16 = I.use_u16 && 4LL * prev_max < BTAS_INF_U16;
            int *Ct = (s < S && !next_u16) ? static_cast<int *>((s & 1) ? I.Q1 : I.Q0) : nullptr;
            uint32_t *Cd = more ? ((s & 1) ? I.Ad1 : I.Ad0) : nullptr;
            uint16_t *Cu = more ? ((s & 1) ? I.U1 : I.U0) : nullptr;
            if (more) a.maxfin = p.maxfin + I.flag_base + s;
            if (s >= 2 && prev_changed == 0) {
                // D_{s-1} == D_{s-2}: a fixpoint of the squaring.  The first
                // such level copies it into D; the levels after it have
                // nothing left to do.
                slot = BTAS_BATCH_SLOT_APSP_DONE;
                if (prev_changed2 != 0) {
                    a.C = I.C;
                    a.ldc = I.ldc;
                    copy_task_tile(small, a, bm, bn, tid);
                }
            } else if (prev_closed) {
                // the certificate after squaring s - 1 held: D_{s-1} is the
                // closure, so D_s = D_{s-1}, with no change; the next level
                // copies it into D as after a converged squaring
                slot = BTAS_BATCH_SLOT_APSP_DONE;
                copy_task_tile(small, a, bm, bn, tid);
            } else if (I.use_u16 && 2LL * prev_max < BTAS_INF_U16) {
                slot = BTAS_BATCH_SLOT_APSP_U16;
                // every finite entry of D_{s-1} is < 0x7FFF / 2: the packed squaring is exact
                U16Tile u{};
                u.n = I.n;
                u.Ad = ((s - 1) & 1) ? I.Ad1 : I.Ad0; u.ldad = I.ldq;
                u.U = ((s - 1) & 1) ? I.U1 : I.U0; u.ldu = I.ldu;
                u.prev = static_cast<const int *>(cur); u.ldp = ldcur;
                u.C = static_cast<int *>(out); u.ldc = a.ldc;
                u.Ct = Ct; u.ldct = I.ldq;
                u.Cd = Cd; u.ldcd = I.ldq;
                u.Cu = Cu; u.ldcu = I.ldu;
                u.maxfin = a.maxfin;
                ch = u16_task_tile(small, u, bm, bn, smem_raw, tid);
            } else {
                slot = BTAS_BATCH_SLOT_APSP_I32;
                ch = gemm_tile<kI32Mix, kMin>(small, a, bm, bn, smem_raw, tid, Ct, I.ldq, Cd, I.ldq, Cu, I.ldu);
            }
        } else if (type == kTaskSquare) {
            const int bm = (tile / I.tiles_n) * TT, bn = (tile % I.tiles_n) * TT;
            GemmArgs a{};
            a.m = a.n = a.k = I.n;
            a.A = I.A; a.lda = I.lda;
            a.Bt = I.Q0; a.ldb = I.ldq;
            a.C = I.C; a.ldc = I.ldc;
            a.prev = I.A; a.ldp = I.lda;
            a.one = 1;
            a.vec_a = ((reinterpret_cast<uintptr_t>(I.A) & 15) == 0) && ((I.lda & 3) == 0);
            a.vec_b = 1;
            a.ro_a = 1;  // this step's input, written by an earlier launch
            a.maxfin = I.maxfin_ptr;
            // packed when asked, or (use_u16 == 2) when every finite entry of the
            // input is < 0x7FFF / 2 (exact; the forms were written at level 0)
            const bool packed = I.use_u16 == 1 || (I.use_u16 == 2 && 2LL * __ldcg(I.maxfin_in) < BTAS_INF_U16);
            if (packed) {
                slot = BTAS_BATCH_SLOT_SQUARE_U16;
                U16Tile u{};
                u.n = I.n;
                u.Ad = I.Ad0; u.ldad = I.ldq;
                u.U = I.U0; u.ldu = I.ldu;
                u.prev = static_cast<const int *>(I.A); u.ldp = I.lda;
                u.C = static_cast<int *>(I.C); u.ldc = I.ldc;
                u.Ct = static_cast<int *>(I.Q1); u.ldct = I.ldq;
                u.Cd = I.Ad1; u.ldcd = I.ldq;
                u.Cu = I.U1; u.ldcu = I.ldu;
                u.maxfin = I.maxfin_ptr;
                ch = u16_task_tile(small, u, bm, bn, smem_raw, tid);
            } else {
                slot = BTAS_BATCH_SLOT_SQUARE_I32;
                ch = gemm_tile<kI32Mix, kMin>(small, a, bm, bn, smem_raw, tid, I.Q1, I.ldq, I.Ad1, I.ldq, I.U1, I.ldu);
            }
        } else {  // kTaskGemm
            const int bm = (tile / I.tiles_n) * TT, bn = (tile % I.tiles_n) * TT;
            GemmArgs a{};
            a.m = I.m; a.n = I.n; a.k = I.k;
            a.A = I.A; a.lda = I.lda;
            a.Bt = I.trans_b ? I.B : I.Q0; a.ldb = I.trans_b ? I.ldb : I.ldq;
            a.C = I.C; a.ldc = I.ldc;
            a.one = 1;
            a.vec_a = ((reinterpret_cast<uintptr_t>(I.A) & 15) == 0) && ((I.lda & 3) == 0);
            a.vec_b = ((reinterpret_cast<uintptr_t>(a.Bt) & 15) == 0) && ((a.ldb & 3) == 0);
            a.ro_a = 1;                // the caller's A
            a.ro_b = I.trans_b ? 1 : 0;  // the caller's B^T, or Q0 from this launch's transposes
            slot = I.dtype == BTAS_I32 ? BTAS_BATCH_SLOT_GEMM_I32 : BTAS_BATCH_SLOT_GEMM_F32;
            if (I.dtype == BTAS_I32) {
                if (I.sr == kMin) gemm_tile<kI32Mix, kMin>(small, a, bm, bn, smem_raw, tid);
                else gemm_tile<kI32Mix, kMax>(small, a, bm, bn, smem_raw, tid);
            } else {
                if (I.sr == kMin) gemm_tile<kF32X2, kMin>(small, a, bm, bn, smem_raw, tid);
                else gemm_tile<kF32X2, kMax>(small, a, bm, bn, smem_raw, tid);
            }
        }
        if (type == kTaskApsp && __any_sync(0xffffffffu, ch) && (tid & 31) == 0)
            atomicOr(p.changed + I.flag_base + level, 1);
        if (type == kTaskSquare && __any_sync(0xffffffffu, ch) && (tid & 31) == 0) atomicOr(I.changed_ptr, 1);
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            atomicAdd(p.done + I.done_base + level, 1);
            if (p.prof != nullptr) {
                atomicAdd(p.prof + 2 * slot, (unsigned long long)(clock64() - t_task));
                atomicAdd(p.prof + 2 * slot + 1, 1ULL);
                if (level > 0) {
                    atomicAdd(p.prof + 2 * BTAS_BATCH_SLOT_WAIT, (unsigned long long)s_wait);
                    atomicAdd(p.prof + 2 * BTAS_BATCH_SLOT_WAIT + 1, 1ULL);
                }
            }
        }
    }
}


int batch_kernel_smem() { return batch_smem_words() * 4; }
int batch_kernel_threads() { return BCfg::kThreads; }

cudaError_t batch_kernel_prepare(int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_kernel_smem());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, batch_kernel, BCfg::kThreads,
                                                         batch_kernel_smem());
}

cudaError_t launch_batch_kernel(const BatchParams &p, int grid, cudaStream_t st) {
    batch_kernel<<<grid, BCfg::kThreads, batch_kernel_smem(), st>>>(p);
    note_launch();
    return cudaGetLastError();
}

long long batch_timeout_cycles(int device) {
    (void)device;  // the current device
    DeviceInfo d{};
    long long c = (long long)(2.0 * (current_device_info(&d) ? d.clock_khz : 2000000) * 1e3);
    const char *tmo = getenv("BTAS_BATCH_TIMEOUT_CYCLES");
    if (tmo && *tmo) c = atoll(tmo);
    return c;
}

namespace {

// Synthetic inputs of the tile autotuner (timing only): kind 0 a random
// digraph (edge probability 0.1, weights 1..100, zero diagonal, INF
// elsewhere), kind 1 int32 values in [0, 10^6], kind 2 fp32 values in [0, 1).
__global__ void tile_tune_fill_kernel(uint32_t *X, long long n, int kind, unsigned long long seed) {
    const long long total = n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        unsigned long long h = seed + (unsigned long long)idx * 0x9e3779b97f4a7c15ULL;
        h = (h ^ (h >> 30)) * 0xbf58476d1ce4e5b9ULL;
        h = (h ^ (h >> 27)) * 0x94d049bb133111ebULL;
        h ^= h >> 31;
        uint32_t v;
        if (kind == 0) {
            const long long r = idx / n, c = idx % n;
            v = r == c ? 0u : ((h & 1023) < 102 ? 1u + (uint32_t)((h >> 16) % 100) : (uint32_t)kInfI32);
        } else if (kind == 1) {
            v = (uint32_t)((h >> 20) % 1000001ULL);
        } else {
            v = __float_as_uint((float)(h >> 40) * 5.9604644775390625e-8f);
        }
        X[idx] = v;
    }
}

}  // namespace

// The batch tuner below needs the batch object's internals.
btas_status batch_tune_impl(int64_t n_max, cudaStream_t st, double *ms_out, int max_entries);
}  // namespace btas

using namespace btas;

// ------------------------------------------------------------------ host side

struct btas_batch_t {
    struct Req {
        BInst inst;
        long long work;  // terms, for ordering
    };
    std::vector<Req> reqs;
    int flags = 0;
    bool dirty = true;
    // plan
    void *dev_mem = nullptr;  // tasks | insts | counters | workspace
    size_t dev_bytes = 0;
    int total = 0;
    int *d_counters = nullptr;  // next | status | done[] | changed[]
    unsigned long long *d_prof = nullptr;  // BTAS_BATCH_PROFILE: (cycles, count) per slot
    size_t counter_bytes = 0;
    BatchParams params{};
    int grid = 0;
    int smem = 0;
    int device = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    long long workspace_bytes = 0;
    int force_tile = 0;  // the tuner's timing batches: this output tile for every instance
};

namespace {

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

int squarings_of(long long n) {
    int s = 0;
    long long reach = 1;
    while (reach < n - 1) {
        reach *= 2;
        ++s;
    }
    return s;
}

// Output task tile per instance: the autotuner's table, keyed by (device,
// kind, size bucket of 32), with BTAS_BATCH_TILE=64|128 overriding it and
// 128 x 128 when neither says otherwise.  kind: 0 APSP, 1 int32 product,
// 2 fp32 product; the bucket is that of the larger output side.
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int>, int> g_tile_table;

int tile_kind(const BInst &I) { return I.kind == kInstApsp ? 0 : (I.dtype == BTAS_I32 ? 1 : 2); }
int tile_bucket(long long n) { return (int)((std::max(1LL, n) - 1) / 32); }

int table_tile(int dev, int kind, long long n) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_table.find(std::make_tuple(dev, kind, tile_bucket(n)));
    return it == g_tile_table.end() ? 0 : it->second;
}

int choose_tile(const btas_batch_t *b, int dev, const BInst &I) {
    if (b->force_tile) return b->force_tile;
    const char *e = getenv("BTAS_BATCH_TILE");
    if (e && *e) return atoi(e) == kBTSmall ? kBTSmall : kBT;
    const int t = table_tile(dev, tile_kind(I), std::max(I.m, I.n));
    return t == kBTSmall ? kBTSmall : kBT;
}

void release_plan(btas_batch_t *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dev_mem) cudaFree(b->dev_mem);
    b->exec = nullptr;
    b->graph = nullptr;
    b->dev_mem = nullptr;
    b->d_prof = nullptr;
}

btas_status bfail(btas_status s, const char *msg) {
    record_error(msg);
    return s;
}

btas_status build_plan(btas_batch_t *b) {
    release_plan(b);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bfail(BTAS_ERR_CUDA, "btas_batch: cudaGetDevice failed");
    b->device = dev;
    const size_t ninst = b->reqs.size();
    // order instances by work, largest first
    std::vector<int> order(ninst);
    for (size_t i = 0; i < ninst; ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->reqs[x].work > b->reqs[y].work; });
    // workspace per instance and counter bases
    std::vector<BInst> insts(ninst);
    size_t ws = 0;
    int counters = 0, max_level = 0;
    std::vector<size_t> ws_off(ninst);
    // BTAS_BATCH_NO_U16 keeps every batched squaring in int32
    const char *no16 = getenv("BTAS_BATCH_NO_U16");
    const int allow16 = (no16 && *no16 && atoi(no16) != 0) ? 0 : 1;
    // The closure certificate for graphs from n = 256 (BTAS_BATCH_CERT_MIN_N;
    // BTAS_BATCH_NO_CERT=1 turns it off): below that a squaring is one or
    // two tiles, no dearer than the certificate tasks.
    const char *no_cert = getenv("BTAS_BATCH_NO_CERT"), *cert_min = getenv("BTAS_BATCH_CERT_MIN_N");
    const bool allow_cert = !(no_cert && *no_cert && atoi(no_cert) != 0);
    const long long cert_min_n = (cert_min && *cert_min) ? atoll(cert_min) : 256;
    for (size_t i = 0; i < ninst; ++i) {
        BInst I = b->reqs[i].inst;
        I.tile = choose_tile(b, dev, I);
        I.tiles_m = (I.m + I.tile - 1) / I.tile;
        I.tiles_n = (I.n + I.tile - 1) / I.tile;
        ws_off[i] = ws;
        if (I.kind == kInstApsp) {
            if (I.levels > 0) {
                I.ldq = (I.n + 3) & ~3LL;
                I.ldx = I.ldq;
                I.ldu = (I.n + 7) & ~7LL;
                I.use_u16 = allow16;
                // X0, X1, Q0, Q1 (int32), Ad0, Ad1 (duplicated words), U0, U1 (uint16)
                ws += 6 * al256((size_t)I.n * I.ldq * 4) + 2 * al256((size_t)I.n * I.ldu * 2);
                // the certificate: rows per task that fit shared memory with their list of
                // lowered entries; edge lists of up to min(256, max(32, n / 4)) edges per row
                const int rows = std::min(16, (batch_smem_words() / 2) / (int)I.ldx);
                I.cert = allow_cert && I.levels >= 3 && I.n >= cert_min_n && rows >= 1 ? 1 : 0;
                if (I.cert) {
                    I.cert_rows = rows;
                    I.cap = (int)std::min(256LL, std::max(32LL, ((I.n / 4 + 31) / 32) * 32LL));
                    ws += al256((size_t)I.n * I.cap * 8) + al256((size_t)I.n * 4);
                }
            }
        } else if (!I.trans_b) {
            I.ldq = (I.k + 3) & ~3LL;
            ws += al256((size_t)I.n * I.ldq * 4);
        }
        I.done_base = counters;
        I.flag_base = counters;
        counters += (I.levels > 0 ? I.levels : 1) + 1;
        max_level = std::max(max_level, I.levels > 0 ? I.levels : 1);
        insts[i] = I;
    }
    // tasks
    std::vector<int4> tasks;
    for (int level = 0; level <= max_level; ++level) {
        for (int oi : order) {
            const BInst &I = insts[oi];
            if (level == 0) {
                if (I.t0_rows > 0) {
                    const int nt = ((I.t0_rows + kBT - 1) / kBT) * ((I.t0_cols + kBT - 1) / kBT);
                    for (int t = 0; t < nt; ++t) tasks.push_back(make_int4(kTaskTranspose, oi, 0, t));
                }
                if (I.cert)
                    for (int t = 0; t < list_tasks(I); ++t) tasks.push_back(make_int4(kTaskLists, oi, 0, t));
                continue;
            }
            const int nt = I.tiles_m * I.tiles_n;
            if (I.kind == kInstApsp && I.levels == 0) {
                if (level == 1)
                    for (int t = 0; t < nt; ++t) tasks.push_back(make_int4(kTaskCopy, oi, 1, t));
            } else if (I.kind == kInstApsp && level <= I.levels) {
                for (int t = 0; t < nt; ++t) tasks.push_back(make_int4(kTaskApsp, oi, level, t));
            } else if (I.kind == kInstGemm && level == 1) {
                for (int t = 0; t < nt; ++t) tasks.push_back(make_int4(kTaskGemm, oi, 1, t));
            }
        }
        // the certificates of this level after every instance's tiles of it:
        // each waits only for tasks claimed before it
        for (int oi : order) {
            const BInst &I = insts[oi];
            if (I.kind == kInstApsp && has_cert(I, level))
                for (int t = 0; t < cert_tasks(I); ++t) tasks.push_back(make_int4(kTaskCert, oi, level, t));
        }
    }
    b->total = (int)tasks.size();
    const size_t task_bytes = al256(tasks.size() * sizeof(int4));
    const size_t inst_bytes = al256(ninst * sizeof(BInst));
    b->counter_bytes = al256((size_t)(2 + 4 * counters) * 4);
    b->workspace_bytes = (long long)ws;
    const size_t prof_bytes = (b->flags & BTAS_BATCH_PROFILE) ? al256(2 * BTAS_BATCH_PROFILE_SLOTS * 8) : 0;
    b->dev_bytes = task_bytes + inst_bytes + b->counter_bytes + prof_bytes + ws;
    if (cudaMalloc(&b->dev_mem, b->dev_bytes ? b->dev_bytes : 256) != cudaSuccess)
        return bfail(BTAS_ERR_NOMEM, "btas_batch: workspace allocation failed");
    char *base = static_cast<char *>(b->dev_mem);
    int4 *d_tasks = reinterpret_cast<int4 *>(base);
    BInst *d_insts = reinterpret_cast<BInst *>(base + task_bytes);
    b->d_counters = reinterpret_cast<int *>(base + task_bytes + inst_bytes);
    b->d_prof = prof_bytes ? reinterpret_cast<unsigned long long *>(base + task_bytes + inst_bytes + b->counter_bytes)
                           : nullptr;
    if (b->d_prof && cudaMemset(b->d_prof, 0, prof_bytes) != cudaSuccess)
        return bfail(BTAS_ERR_CUDA, "btas_batch: profile reset");
    char *d_ws = base + task_bytes + inst_bytes + b->counter_bytes + prof_bytes;
    for (size_t i = 0; i < ninst; ++i) {
        BInst &I = insts[i];
        char *w = d_ws + ws_off[i];
        if (I.kind == kInstApsp && I.levels > 0) {
            const size_t blk = al256((size_t)I.n * I.ldq * 4);
            I.X0 = w;
            I.X1 = w + blk;
            I.Q0 = w + 2 * blk;
            I.Q1 = w + 3 * blk;
            I.Ad0 = reinterpret_cast<uint32_t *>(w + 4 * blk);
            I.Ad1 = reinterpret_cast<uint32_t *>(w + 5 * blk);
            I.U0 = reinterpret_cast<uint16_t *>(w + 6 * blk);
            I.U1 = reinterpret_cast<uint16_t *>(w + 6 * blk + al256((size_t)I.n * I.ldu * 2));
            if (I.cert) {
                char *l = w + 6 * blk + 2 * al256((size_t)I.n * I.ldu * 2);
                I.lists = reinterpret_cast<int2 *>(l);
                I.deg = reinterpret_cast<int *>(l + al256((size_t)I.n * I.cap * 8));
            }
        } else if (I.kind == kInstGemm && !I.trans_b) {
            I.Q0 = w;
        }
    }
    if (cudaMemcpy(d_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_insts, insts.data(), ninst * sizeof(BInst), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(BTAS_ERR_CUDA, "btas_batch: plan upload failed");
    BatchParams &p = b->params;
    p.tasks = d_tasks;
    p.total = b->total;
    p.next = b->d_counters;
    p.status = b->d_counters + 1;
    p.done = b->d_counters + 2;
    p.changed = b->d_counters + 2 + counters;
    p.maxfin = b->d_counters + 2 + 2 * counters;
    p.certfail = b->d_counters + 2 + 3 * counters;
    p.insts = d_insts;
    p.timeout_cycles = batch_timeout_cycles(dev);
    p.prof = b->d_prof;
    // Fault injection (tests only): BTAS_BATCH_WITHHOLD=i makes the host
    // withhold one completion of instance i (in add order), so its bounded
    // waits run out and the launch ends with BTAS_ERR_TIMEOUT.
    const char *wh = getenv("BTAS_BATCH_WITHHOLD");
    p.withhold_inst = (wh && *wh) ? atoi(wh) : -1;
    // grid: resident CTAs
    b->smem = batch_kernel_smem();
    int per_sm = 0, sms = 0;
    if (batch_kernel_prepare(&per_sm) != cudaSuccess) return bfail(BTAS_ERR_CUDA, "btas_batch: kernel attributes");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(per_sm * sms, std::max(1, b->total)));
    // capture: counter reset + persistent kernel
    if (!(b->flags & BTAS_BATCH_NO_GRAPH)) {
        if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
            return bfail(BTAS_ERR_CUDA, "btas_batch: stream create");
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(BTAS_ERR_CUDA, "btas_batch: begin capture");
        cudaMemsetAsync(b->d_counters, 0, b->counter_bytes, b->cap);
        launch_batch_kernel(p, b->grid, b->cap);
        const cudaError_t e1 = cudaStreamEndCapture(b->cap, &b->graph);
        if (e1 != cudaSuccess) return bfail(BTAS_ERR_CUDA, "btas_batch: end capture");
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
            return bfail(BTAS_ERR_CUDA, "btas_batch: graph instantiate");
    }
    b->dirty = false;
    return BTAS_OK;
}

}  // namespace

extern "C" {

btas_status btas_batch_create(btas_batch_t **out, int flags) {
    if (!out) return bfail(BTAS_ERR_ARG, "btas_batch_create: NULL out");
    if (flags & ~(BTAS_BATCH_NO_GRAPH | BTAS_BATCH_PROFILE))
        return bfail(BTAS_ERR_ARG, "btas_batch_create: unknown flags");
    btas_batch_t *b = new btas_batch_t();
    b->flags = flags;
    *out = b;
    return BTAS_OK;
}

btas_status btas_batch_destroy(btas_batch_t *b) {
    if (!b) return BTAS_OK;
    release_plan(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return BTAS_OK;
}

btas_status btas_batch_add_apsp(btas_batch_t *b, int64_t n, const int32_t *W, int32_t *D) {
    if (!b) return bfail(BTAS_ERR_ARG, "btas_batch_add_apsp: NULL batch");
    if (n < 1 || n > 46340) return bfail(BTAS_ERR_ARG, "btas_batch_add_apsp: n out of range");
    if (!W || !D) return bfail(BTAS_ERR_ARG, "btas_batch_add_apsp: NULL pointer");
    const char *wb = reinterpret_cast<const char *>(W), *db = reinterpret_cast<const char *>(D);
    const size_t bytes = (size_t)n * n * 4;
    if (wb < db + bytes && db < wb + bytes) return bfail(BTAS_ERR_ARG, "btas_batch_add_apsp: W and D overlap");
    BInst I{};
    I.kind = kInstApsp;
    I.sr = kMin;
    I.dtype = BTAS_I32;
    I.m = I.n = I.k = (int)n;
    I.levels = squarings_of(n);
    I.tiles_m = I.tiles_n = (int)((n + kBT - 1) / kBT);
    if (I.levels > 0) {
        I.t0_rows = I.t0_cols = (int)n;
    }
    I.A = W;
    I.lda = n;
    I.C = D;
    I.ldc = n;
    b->reqs.push_back({I, (long long)n * n * n * std::max(1, I.levels)});
    b->dirty = true;
    return BTAS_OK;
}

btas_status btas_batch_add_gemm(btas_batch_t *b, int semiring, int dtype, int64_t m, int64_t n, int64_t k,
                                const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc) {
    if (!b) return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: NULL batch");
    const int sr = semiring & 0xff;
    const bool trans_b = (semiring & BTAS_GEMM_TRANS_B) != 0;
    if (semiring & ~(0xff | BTAS_GEMM_TRANS_B)) return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: flags");
    if (sr != kMin && sr != kMax) return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return bfail(BTAS_ERR_UNSUPPORTED, "btas_batch_add_gemm: dtype");
    if (m < 1 || n < 1 || k < 1 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
        return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: sizes must be >= 1");
    if (lda < k || ldc < n || ldb < (trans_b ? k : n)) return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: ld");
    if (!A || !B || !C) return bfail(BTAS_ERR_ARG, "btas_batch_add_gemm: NULL pointer");
    BInst I{};
    I.kind = kInstGemm;
    I.sr = sr;
    I.dtype = dtype;
    I.m = (int)m;
    I.n = (int)n;
    I.k = (int)k;
    I.levels = 1;
    I.tiles_m = (int)((m + kBT - 1) / kBT);
    I.tiles_n = (int)((n + kBT - 1) / kBT);
    I.trans_b = trans_b ? 1 : 0;
    if (!trans_b) {
        I.t0_rows = (int)k;
        I.t0_cols = (int)n;
    }
    I.A = A;
    I.lda = lda;
    I.B = B;
    I.ldb = ldb;
    I.C = C;
    I.ldc = ldc;
    b->reqs.push_back({I, (long long)m * n * k});
    b->dirty = true;
    return BTAS_OK;
}

btas_status btas_batch_launch(btas_batch_t *b, void *stream) {
    if (!b) return bfail(BTAS_ERR_ARG, "btas_batch_launch: NULL batch");
    if (b->reqs.empty()) return BTAS_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (b->dirty || dev != b->device) {
        const btas_status s = build_plan(b);
        if (s != BTAS_OK) return s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (b->exec) {
        e = cudaGraphLaunch(b->exec, st);
        note_launch();
    } else {
        e = cudaMemsetAsync(b->d_counters, 0, b->counter_bytes, st);
        if (e == cudaSuccess) e = launch_batch_kernel(b->params, b->grid, st);
    }
    if (e != cudaSuccess) return bfail(BTAS_ERR_CUDA, cudaGetErrorString(e));
    return BTAS_OK;
}

btas_status btas_batch_wait(btas_batch_t *b, void *stream) {
    if (!b) return bfail(BTAS_ERR_ARG, "btas_batch_wait: NULL batch");
    if (!b->d_counters) return BTAS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, b->params.status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail(BTAS_ERR_CUDA, cudaGetErrorString(e));
    if (status != 0) return bfail(static_cast<btas_status>(status), "btas_batch: a bounded device wait expired");
    return BTAS_OK;
}

int64_t btas_batch_workspace_bytes(btas_batch_t *b) { return b ? b->workspace_bytes : 0; }

int btas_batch_tasks(btas_batch_t *b) { return b ? b->total : 0; }

btas_status btas_batch_tune(int64_t n_max, void *stream, double *ms_out, int max_entries) {
    return batch_tune_impl(n_max, static_cast<cudaStream_t>(stream), ms_out, max_entries);
}

btas_status btas_batch_select_tiles(btas_batch_t *b, void *stream, int *mode, double *ms_out) {
    if (!b) return bfail(BTAS_ERR_ARG, "btas_batch_select_tiles: NULL batch");
    if (b->reqs.empty()) {
        if (mode) *mode = 0;
        return BTAS_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // mode 0: the table (and BTAS_BATCH_TILE), 1: 128 x 128, 2: 64 x 64 for every instance
    const int force[3] = {0, kBT, kBTSmall};
    double ms[3] = {0, 0, 0};
    btas_status r = BTAS_OK;
    for (int m = 0; m < 3 && r == BTAS_OK; ++m) {
        b->force_tile = force[m];
        b->dirty = true;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && r == BTAS_OK; ++rep) {
            cudaEventRecord(e0, st);
            r = btas_batch_launch(b, st);
            cudaEventRecord(e1, st);
            if (r == BTAS_OK) r = btas_batch_wait(b, st);
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) best = std::min(best, t);
        }
        ms[m] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != BTAS_OK) {
        b->force_tile = 0;
        b->dirty = true;
        return r;
    }
    int best = 0;
    for (int m = 1; m < 3; ++m)
        if (ms[m] < ms[best]) best = m;
    b->force_tile = force[best];
    b->dirty = true;  // the next launch plans with the chosen tiles
    if (mode) *mode = best;
    if (ms_out)
        for (int m = 0; m < 3; ++m) ms_out[m] = ms[m];
    return BTAS_OK;
}

int btas_batch_tile(int kind, int64_t n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || kind < 0 || kind > 2 || n < 1) return 0;
    return table_tile(dev, kind, n);
}

void btas_batch_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_table.clear();
}

btas_status btas_batch_profile(btas_batch_t *b, uint64_t *cycles, uint64_t *counts, int slots) {
    if (!b || !(b->flags & BTAS_BATCH_PROFILE))
        return bfail(BTAS_ERR_ARG, "btas_batch_profile: batch created without BTAS_BATCH_PROFILE");
    if (!b->d_prof) return bfail(BTAS_ERR_ARG, "btas_batch_profile: batch not launched yet");
    if (slots < 0 || ((!cycles || !counts) && slots > 0)) return bfail(BTAS_ERR_ARG, "btas_batch_profile: outputs");
    unsigned long long h[2 * BTAS_BATCH_PROFILE_SLOTS];
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h, b->d_prof, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bfail(BTAS_ERR_CUDA, "btas_batch_profile: read back");
    for (int i = 0; i < std::min(slots, BTAS_BATCH_PROFILE_SLOTS); ++i) {
        cycles[i] = h[2 * i];
        counts[i] = h[2 * i + 1];
    }
    return BTAS_OK;
}

}  // extern "C"

namespace btas {

// For each kind and size bucket of 32 vertices (rows) up to n_max: one
// synthetic batch of three sizes in the bucket, with enough instances that
// every level holds several waves of 128 x 128 tasks (4 waves of the
// persistent grid per squaring level, 8 for products) -- the regime of a
// large batch, where per-term speed and padding decide, not the number of
// tasks -- timed (best of 3 graph-captured launches, after one warm-up)
// with the 128 x 128 and with the 64 x 64 output tile.  The small tile is
// kept only if it is at least 3 % faster.
btas_status batch_tune_impl(int64_t n_max, cudaStream_t st, double *ms_out, int max_entries) {
    if (n_max < 1 || n_max > 2048) return bfail(BTAS_ERR_ARG, "btas_batch_tune: n_max must be in [1, 2048]");
    if (max_entries < 0 || (max_entries > 0 && !ms_out)) return bfail(BTAS_ERR_ARG, "btas_batch_tune: ms_out");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bfail(BTAS_ERR_CUDA, "btas_batch_tune: cudaGetDevice failed");
    const int buckets = (int)((n_max + 31) / 32);
    int per_sm = 0;
    DeviceInfo di{};
    if (batch_kernel_prepare(&per_sm) != cudaSuccess || !current_device_info(&di))
        return bfail(BTAS_ERR_CUDA, "btas_batch_tune: device query failed");
    const double grid = std::max(1, per_sm) * (double)di.sms;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    btas_status result = BTAS_OK;
    for (int kind = 0; kind < 3 && result == BTAS_OK; ++kind) {
        for (int bk = 0; bk < buckets && result == BTAS_OK; ++bk) {
            std::vector<long long> sizes;
            for (int off : {8, 20, 32}) {
                const long long n = std::min<long long>(n_max, 32LL * bk + off);
                if (n >= 3 && (sizes.empty() || sizes.back() != n)) sizes.push_back(n);
            }
            if (sizes.empty()) continue;
            // instances per size: several waves of 128 x 128 tasks per level
            std::vector<int> count;
            size_t bytes = 0;
            for (long long n : sizes) {
                const double tiles = (double)((n + kBT - 1) / kBT) * ((n + kBT - 1) / kBT);
                const double waves = kind == 0 ? 4.0 : 8.0;
                const int c = (int)std::max(2.0, std::min(4096.0, std::ceil(waves * grid / (sizes.size() * tiles))));
                count.push_back(c);
                bytes += (size_t)c * (kind == 0 ? 2 : 3) * al256((size_t)n * n * 4);
            }
            void *buf = nullptr;
            if (cudaMalloc(&buf, bytes) != cudaSuccess) {
                result = bfail(BTAS_ERR_NOMEM, "btas_batch_tune: allocation failed");
                break;
            }
            char *p = static_cast<char *>(buf);
            std::vector<std::pair<long long, char *>> mats;
            unsigned long long seed = 0x170104733ULL + 977ULL * (kind * 64 + bk);
            for (size_t z = 0; z < sizes.size(); ++z)
                for (int c = 0; c < count[z]; ++c) {
                    const long long n = sizes[z];
                    const size_t mb = al256((size_t)n * n * 4);
                    const int inputs = kind == 0 ? 1 : 2;
                    for (int q = 0; q < inputs; ++q) {
                        const long long blocks = std::min<long long>(1024, (n * n + 255) / 256);
                        tile_tune_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<uint32_t *>(p + q * mb),
                                                                               n, kind, seed++);
                        note_launch();
                    }
                    mats.push_back({n, p});
                    p += (kind == 0 ? 2 : 3) * mb;
                }
            double ms[2] = {0, 0};
            for (int ti = 0; ti < 2 && result == BTAS_OK; ++ti) {
                btas_batch_t *b = nullptr;
                btas_batch_create(&b, 0);
                b->force_tile = ti == 0 ? kBT : kBTSmall;
                for (auto &m : mats) {
                    const long long n = m.first;
                    const size_t mb = al256((size_t)n * n * 4);
                    if (kind == 0)
                        btas_batch_add_apsp(b, n, reinterpret_cast<const int32_t *>(m.second),
                                            reinterpret_cast<int32_t *>(m.second + mb));
                    else
                        btas_batch_add_gemm(b, kind == 1 ? BTAS_MINPLUS : BTAS_MAXPLUS, kind == 1 ? BTAS_I32 : BTAS_F32,
                                            n, n, n, m.second, n, m.second + mb, n, m.second + 2 * mb, n);
                }
                float best = 1e30f;
                for (int rep = 0; rep < 4 && result == BTAS_OK; ++rep) {
                    cudaEventRecord(e0, st);
                    result = btas_batch_launch(b, st);
                    cudaEventRecord(e1, st);
                    if (result == BTAS_OK) result = btas_batch_wait(b, st);
                    float t = 0;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) best = std::min(best, t);
                }
                ms[ti] = best;
                btas_batch_destroy(b);
            }
            cudaStreamSynchronize(st);
            cudaFree(buf);
            if (result != BTAS_OK) break;
            const int choice = ms[1] < 0.97 * ms[0] ? kBTSmall : kBT;
            {
                std::lock_guard<std::mutex> lk(g_tile_mu);
                g_tile_table[std::make_tuple(dev, kind, bk)] = choice;
            }
            const int slot = kind * buckets + bk;
            if (2 * slot + 1 < max_entries) {
                ms_out[2 * slot] = ms[0];
                ms_out[2 * slot + 1] = ms[1];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

}  // namespace btas
