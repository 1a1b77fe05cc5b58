// Continuous-batching request server for tropical products and APSP solves.
//
// Requests (a tropical product, or an APSP solve by repeated squaring,
// Sec. III) arrive with HOST buffers at any time.  One executor thread owns
// the device:
//   admit   - in arrival order, while the device-memory footprint of the
//             admitted requests stays within the budget: allocate the
//             request's device block (stream-ordered) and copy its inputs in
//             on a copy stream;
//   step    - active requests contribute their next unit of work (a
//             product: the whole product; APSP: its next squaring), oldest
//             first, up to a work cap per step (default 1.5e10 terms, about
//             1 ms; BTAS_SERVER_STEP_TERMS), and these units run together in
//             ONE launch of the persistent tile-task kernel
//             (batch_kernel.cuh).  A unit larger than what is left of the
//             cap contributes a chunk of its 128 x 128 output tiles and
//             continues in the next step, so every step stays short; units
//             below 5 % of the cap always join.  Short steps let finished
//             requests leave and new ones join often.  An APSP request with
//             n <= 1792 is one unit instead when the rest of the work is
//             light: the whole solve, by the one-block or the cooperative
//             kernel, launched after the persistent kernel;
//   retire  - a product is finished after its step; an APSP solve after its
//             last squaring or as soon as a squaring changed nothing (early
//             exit, same result).  Its result is copied back on the copy
//             stream and its memory returned once the copy has completed.
// Requests too large for one launch of either kind of kernel to bring any
// batching gain -- APSP above the cooperative kernel's size limit, products
// of more than BTAS_SERVER_BULK_TERMS terms (default 4e9) -- take a second
// lane instead: a bulk thread runs them one at a time, in arrival order,
// through the library's single calls (btas_apsp, btas_gemm) on a compute
// stream of its own, of higher priority than the step loop's: the large
// requests set the latency tail, and the small ones, batched in the step
// loop, never queue behind them but take the SMs the large kernels leave
// free (and the gaps of the bulk lane's read-backs and set-up).  While the
// bulk lane holds work the step loop does not launch the cooperative
// whole-solve kernel, whose grid must be co-resident on every SM.  The bulk
// lane's copies run on a copy stream of their own.
// Requests that arrive while a step runs are admitted at once (their device
// memory is taken on the copy stream, so their input copies overlap the
// step) and join the next step, so their work overlaps with the squarings
// of requests already in flight (iteration-level continuous batching).  The arithmetic is the library's
// single-call arithmetic: every result is bit-identical to the one computed
// alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_kernel.cuh"
#include "common.cuh"
#include "kernels.h"

using namespace btas;

namespace {

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }
long long r4(long long v) { return (v + 3) & ~3LL; }

enum ReqState : int { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Req {
    int64_t id = 0;
    int kind = 0;  // 0 APSP, 1 product
    int sr = 0, dtype = 0;
    int m = 0, n = 0, k = 0;
    const void *hA = nullptr, *hB = nullptr;
    void *hC = nullptr;
    size_t bytes = 0;
    char *dmem = nullptr;
    // APSP: P[0], P[1] ping-pong (pitch ldp), Q[0], Q[1] transposes (pitch ldp), flags
    // product: A (pitch lda_d), B (pitch ldb_d), Bt (pitch ldq), C (pitch ldc_d)
    void *P[2] = {nullptr, nullptr}, *Q[2] = {nullptr, nullptr};
    int *dflag = nullptr;
    long long ldp = 0;
    void *dA = nullptr, *dB = nullptr, *dBt = nullptr, *dC = nullptr;
    long long lda_d = 0, ldb_d = 0, ldq = 0, ldc_d = 0;
    int S = 0, s = 1;  // APSP squarings, next squaring (1-based)
    // APSP: packed 16-bit operand forms of D (two sets) and the largest
    // finite entry of the latest D (-1: not known yet)
    uint32_t *Ad[2] = {nullptr, nullptr};
    uint16_t *U[2] = {nullptr, nullptr};
    long long ldu = 0;
    int last_max = -1;
    int result_buf = 0;
    cudaEvent_t in_ready = nullptr, out_ready = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = kQueued;
    int steps = 0;
    int tile_next = 0;   // output tiles of the current unit done in earlier steps
    int take = 0;        // output tiles of the current unit in this step
    bool finished = false;
    bool whole = false;  // APSP solved in one unit (small / cooperative kernel) in this step
    bool bulk = false;   // large request: runs in the bulk lane through the single calls
    bool bad = false;    // W outside the domain (checked on the device before the first squaring): the request fails
    // terms of this request's next unit of work
    double unit_terms() const { return kind == 0 ? (double)n * n * n : (double)m * n * k; }
    int unit_tiles() const { return ((m + 127) / 128) * ((n + 127) / 128); }
    double tile_terms() const { return 128.0 * 128.0 * (double)k; }
    double remaining_terms() const { return unit_terms() * (1.0 - (double)tile_next / unit_tiles()); }
};

}  // namespace

struct btas_server_t {
    int device = 0;
    long long budget = 0;
    long long used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;             // waiting for admission
    std::deque<Req *> bulk_queue;        // large requests waiting for the bulk lane
    std::vector<Req *> active;           // admitted, work remaining
    std::vector<Req *> retiring;         // result copy in flight
    std::map<int64_t, Req *> all;        // every request ever submitted
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker, bulk_worker;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t compute = nullptr, copy = nullptr;      // the step loop's streams
    cudaStream_t bulk = nullptr, bulk_compute = nullptr;  // the bulk lane's copy and compute streams
    double bulk_terms = 4e9;   // products above this many terms take the bulk lane
    int64_t bulk_runs = 0;
    bool bulk_busy = false;  // the bulk lane holds a request
    void *bulk_buf = nullptr;  // the bulk lane's device block, grown as needed, kept until destroy
    size_t bulk_cap = 0;
    // per-step device/pinned staging (double-buffered by step parity)
    void *d_stage[2] = {nullptr, nullptr};
    void *h_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    int *h_flags = nullptr;  // pinned mailbox: change flags, maxima or barrier status, domain-scan results
    int *d_flag_slots = nullptr;
    int flag_slots = 0;
    cudaEvent_t step_done[2] = {nullptr, nullptr};
    int grid = 0;
    long long timeout_cycles = 0;
    int step_parity = 0;
    double step_terms = 1.5e10;  // work cap of one step (terms), keeps steps short
    int allow_u16 = 1;         // BTAS_SERVER_NO_U16=1 keeps every squaring in int32
    int allow_whole = 1;       // BTAS_SERVER_NO_WHOLE=1 runs every APSP squaring by squaring
    double whole_below = 1.5e10;  // whole solves only when the other pending work is below this (terms)
    int64_t steps = 0;
    int64_t units = 0;
    int64_t completed = 0;
    int last_error = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

btas_status sfail(btas_status s, const char *msg) {
    record_error(msg);
    return s;
}

int squarings_of(long long n) {
    int s = 0;
    long long reach = 1;
    while (reach < n - 1) {
        reach *= 2;
        ++s;
    }
    return s;
}

size_t footprint(const Req &r) {
    if (r.kind == 0) {
        const long long ld = r4(r.n), ldu = (r.n + 7) & ~7LL;
        return 6 * a256((size_t)r.n * ld * 4) + 2 * a256((size_t)r.n * ldu * 2) + a256((size_t)(2 * r.S + 6) * 4);
    }
    return a256((size_t)r.m * r4(r.k) * 4) + a256((size_t)r.k * r4(r.n) * 4) + a256((size_t)r.n * r4(r.k) * 4) +
           a256((size_t)r.m * r4(r.n) * 4);
}

// Allocate the request's device block and start its input copies.
// The block is taken on the copy stream, so the copies start at once even
// while a step runs on the compute stream; the compute stream waits for
// in_ready before it touches the block.
bool admit(btas_server_t *sv, Req *r) {
    if (ws_alloc(reinterpret_cast<void **>(&r->dmem), r->bytes, sv->copy) != cudaSuccess) return false;
    char *p = r->dmem;
    if (r->kind == 0) {
        const long long ld = r4(r->n);
        const size_t blk = a256((size_t)r->n * ld * 4);
        r->ldp = ld;
        r->P[0] = p;
        r->P[1] = p + blk;
        r->Q[0] = p + 2 * blk;
        r->Q[1] = p + 3 * blk;
        r->Ad[0] = reinterpret_cast<uint32_t *>(p + 4 * blk);
        r->Ad[1] = reinterpret_cast<uint32_t *>(p + 5 * blk);
        r->ldu = (r->n + 7) & ~7LL;
        const size_t ublk = a256((size_t)r->n * r->ldu * 2);
        r->U[0] = reinterpret_cast<uint16_t *>(p + 6 * blk);
        r->U[1] = reinterpret_cast<uint16_t *>(p + 6 * blk + ublk);
        // change flags [0, S+2), largest finite entries [S+2, 2S+4), the
        // domain scan of W [2S+4, 2S+6)
        r->dflag = reinterpret_cast<int *>(p + 6 * blk + 2 * ublk);
        cudaMemsetAsync(r->dflag, 0, (size_t)(2 * r->S + 6) * 4, sv->copy);
        cudaMemcpy2DAsync(r->P[0], ld * 4, r->hA, (size_t)r->n * 4, (size_t)r->n * 4, r->n, cudaMemcpyHostToDevice,
                          sv->copy);
    } else {
        r->lda_d = r4(r->k);
        r->ldb_d = r4(r->n);
        r->ldq = r4(r->k);
        r->ldc_d = r4(r->n);
        r->dA = p;
        p += a256((size_t)r->m * r->lda_d * 4);
        r->dB = p;
        p += a256((size_t)r->k * r->ldb_d * 4);
        r->dBt = p;
        p += a256((size_t)r->n * r->ldq * 4);
        r->dC = p;
        cudaMemcpy2DAsync(r->dA, r->lda_d * 4, r->hA, (size_t)r->k * 4, (size_t)r->k * 4, r->m,
                          cudaMemcpyHostToDevice, sv->copy);
        cudaMemcpy2DAsync(r->dB, r->ldb_d * 4, r->hB, (size_t)r->n * 4, (size_t)r->n * 4, r->k,
                          cudaMemcpyHostToDevice, sv->copy);
    }
    cudaEventCreateWithFlags(&r->in_ready, cudaEventDisableTiming);
    cudaEventRecord(r->in_ready, sv->copy);
    return true;
}

void release(btas_server_t *sv, Req *r) {
    if (r->dmem) ws_free(r->dmem, sv->copy);
    r->dmem = nullptr;
    if (r->in_ready) cudaEventDestroy(r->in_ready);
    if (r->out_ready) cudaEventDestroy(r->out_ready);
    r->in_ready = r->out_ready = nullptr;
}

// Build and launch one step over the active requests.  Returns the number
// of units launched.
int launch_step(btas_server_t *sv, std::vector<Req *> &units) {
    // oldest admitted requests first, until the step's work cap (at least one)
    units.clear();
    double terms = 0, pending = 0;
    for (Req *r : sv->active) pending += r->remaining_terms();
    bool bulk_busy;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        bulk_busy = sv->bulk_busy || !sv->bulk_queue.empty();
    }
    const double cap = sv->step_terms;
    const double small = 0.05 * cap;
    for (Req *r : sv->active) {
        // an APSP request that fits the one-block or cooperative kernel is
        // solved whole, in one unit, instead of one squaring per step -- when
        // the rest of the work is light.  Under load its squarings are
        // batched with the other requests' work instead, which keeps the GPU
        // busier than a whole solve's grid barriers do.
        r->whole = sv->allow_whole && r->kind == 0 && r->s == 1 && r->tile_next == 0 && r->n <= apsp_mid_max_n() &&
                   pending - r->unit_terms() < sv->whole_below && (r->n <= apsp_small_limit() || !bulk_busy);
        r->take = 0;
        if (r->whole) {
            const double w = r->unit_terms() * std::min(r->S, 6);
            if (!units.empty() && terms + w > cap && w >= small) continue;
            units.push_back(r);
            terms += w;
            continue;
        }
        // the rest of the current unit, or the chunk of its output tiles that
        // fits what is left of the cap; small units always join
        const int rem = r->unit_tiles() - r->tile_next;
        const double tt = r->tile_terms(), rem_terms = rem * tt, left = cap - terms;
        int take;
        if (rem_terms <= left || rem_terms < small) take = rem;
        else if (left >= tt) take = std::min(rem, std::max(1, (int)(left / tt)));
        else if (units.empty()) take = 1;
        else continue;
        r->take = take;
        units.push_back(r);
        terms += take * tt;
    }
    if (units.empty()) return 0;
    // batched units first (largest first), whole solves after them
    std::stable_sort(units.begin(), units.end(), [](const Req *a, const Req *b) {
        if (a->whole != b->whole) return !a->whole;
        const long long wa = (long long)a->m * a->n * a->k, wb = (long long)b->m * b->n * b->k;
        return wa > wb;
    });
    int ninst = 0;
    while (ninst < (int)units.size() && !units[ninst]->whole) ++ninst;
    std::vector<BInst> insts(ninst);
    std::vector<int4> tasks;
    for (int i = 0; i < ninst; ++i) {
        Req *r = units[i];
        cudaStreamWaitEvent(sv->compute, r->in_ready, 0);
        BInst I{};
        I.done_base = 2 * i;
        I.flag_base = 2 * i;
        I.levels = 1;
        const bool first_chunk = r->tile_next == 0;
        if (r->kind == 0) {
            const int s = r->s;
            I.kind = kInstSquare;
            I.sr = kMin;
            I.dtype = BTAS_I32;
            I.m = I.n = I.k = r->n;
            I.tiles_m = I.tiles_n = (r->n + kBT - 1) / kBT;
            I.A = r->P[(s - 1) & 1];
            I.lda = r->ldp;
            I.C = r->P[s & 1];
            I.ldc = r->ldp;
            I.Q0 = r->Q[(s - 1) & 1];
            I.Q1 = s < r->S ? r->Q[s & 1] : nullptr;
            I.ldq = r->ldp;
            I.changed_ptr = r->dflag + s;
            if (s == 1 && first_chunk) {
                I.t0_rows = I.t0_cols = r->n;  // transpose W into Q[0] first
                // the weight domain, checked on the device; a violation fails the
                // request.  The scan also finds W's largest weight.
                if (launch_apsp_scan(static_cast<const int *>(r->P[0]), r->n, r->dflag + 2 * r->S + 4, sv->compute,
                                     r->ldp) != cudaSuccess)
                    return -1;
            }
            // packed squaring when every finite entry of D_{s-1} is < 0x7FFF / 2
            // (exact); the forms of D_s are written for the next squaring.  For
            // the first squaring the device decides from W's largest weight (the
            // level-0 transposes also write W's 16-bit forms).
            if (s == 1) {
                I.use_u16 = sv->allow_u16 ? 2 : 0;
                I.maxfin_in = r->dflag + 2 * r->S + 4;
            } else {
                I.use_u16 = (r->last_max >= 0 && 2LL * r->last_max < BTAS_INF_U16 && sv->allow_u16) ? 1 : 0;
            }
            I.Ad0 = r->Ad[(s - 1) & 1];
            I.U0 = r->U[(s - 1) & 1];
            I.Ad1 = s < r->S ? r->Ad[s & 1] : nullptr;
            I.U1 = s < r->S ? r->U[s & 1] : nullptr;
            I.ldu = r->ldu;
            I.maxfin_ptr = s < r->S ? r->dflag + r->S + 2 + s : nullptr;
        } else {
            I.kind = kInstGemm;
            I.sr = r->sr;
            I.dtype = r->dtype;
            I.m = r->m;
            I.n = r->n;
            I.k = r->k;
            I.tiles_m = (r->m + kBT - 1) / kBT;
            I.tiles_n = (r->n + kBT - 1) / kBT;
            I.A = r->dA;
            I.lda = r->lda_d;
            I.B = r->dB;
            I.ldb = r->ldb_d;
            I.C = r->dC;
            I.ldc = r->ldc_d;
            I.Q0 = r->dBt;
            I.ldq = r->ldq;
            if (first_chunk) {  // B^T into Q0 with the first chunk
                I.t0_rows = r->k;
                I.t0_cols = r->n;
            }
        }
        insts[i] = I;
    }
    const int par = sv->step_parity;
    // the staging buffer of this parity was used two steps ago: that step is done
    cudaEventSynchronize(sv->step_done[par]);
    if (ninst > 0) {
    for (int level = 0; level <= 1; ++level)
        for (int i = 0; i < ninst; ++i) {
            const BInst &I = insts[i];
            if (level == 0) {
                if (I.t0_rows > 0) {
                    const int nt = ((I.t0_rows + kBT - 1) / kBT) * ((I.t0_cols + kBT - 1) / kBT);
                    for (int t = 0; t < nt; ++t) tasks.push_back(make_int4(kTaskTranspose, i, 0, t));
                }
            } else {
                // this step's chunk of the unit's output tiles
                const int type = I.kind == kInstSquare ? kTaskSquare : kTaskGemm;
                const int t0 = units[i]->tile_next, t1 = t0 + units[i]->take;
                for (int t = t0; t < t1; ++t) tasks.push_back(make_int4(type, i, 1, t));
            }
        }
    // staging: [counters (next, status, done[2*ninst], changed[2*ninst]) | insts | tasks]
    const size_t cnt_bytes = a256((size_t)(2 + 4 * ninst) * 4);
    const size_t inst_bytes = a256((size_t)ninst * sizeof(BInst));
    const size_t task_bytes = a256(tasks.size() * sizeof(int4));
    const size_t need = cnt_bytes + inst_bytes + task_bytes;
    if (need > sv->stage_bytes) {
        for (int q = 0; q < 2; ++q) {
            cudaEventSynchronize(sv->step_done[q]);
            if (sv->d_stage[q]) cudaFree(sv->d_stage[q]);
            if (sv->h_stage[q]) cudaFreeHost(sv->h_stage[q]);
            sv->d_stage[q] = sv->h_stage[q] = nullptr;
        }
        sv->stage_bytes = std::max(need, sv->stage_bytes * 2);
        for (int q = 0; q < 2; ++q) {
            if (cudaMalloc(&sv->d_stage[q], sv->stage_bytes) != cudaSuccess ||
                cudaMallocHost(&sv->h_stage[q], sv->stage_bytes) != cudaSuccess)
                return -1;
        }
    }
    char *h = static_cast<char *>(sv->h_stage[par]);
    char *d = static_cast<char *>(sv->d_stage[par]);
    memset(h, 0, cnt_bytes);
    memcpy(h + cnt_bytes, insts.data(), (size_t)ninst * sizeof(BInst));
    memcpy(h + cnt_bytes + inst_bytes, tasks.data(), tasks.size() * sizeof(int4));
    cudaMemcpyAsync(d, h, need, cudaMemcpyHostToDevice, sv->compute);
    BatchParams p{};
    int *cnt = reinterpret_cast<int *>(d);
    p.next = cnt;
    p.status = cnt + 1;
    p.done = cnt + 2;
    p.changed = cnt + 2 + 2 * ninst;
    p.insts = reinterpret_cast<const BInst *>(d + cnt_bytes);
    p.tasks = reinterpret_cast<const int4 *>(d + cnt_bytes + inst_bytes);
    p.total = (int)tasks.size();
    p.timeout_cycles = sv->timeout_cycles;
    p.withhold_inst = -1;
    const int grid = std::max(1, std::min(sv->grid, p.total));
    if (launch_batch_kernel(p, grid, sv->compute) != cudaSuccess) return -1;
    // change flags and largest finite entries of this step's squarings ->
    // pinned mailbox
    for (int i = 0; i < ninst; ++i) {
        if (units[i]->kind != 0) continue;
        sv->h_flags[2 * sv->flag_slots + 1 + i] = 0;
        if (units[i]->s == 1)
            cudaMemcpyAsync(sv->h_flags + 2 * sv->flag_slots + 1 + i, units[i]->dflag + 2 * units[i]->S + 5, 4,
                            cudaMemcpyDeviceToHost, sv->compute);
        cudaMemcpyAsync(sv->h_flags + i, units[i]->dflag + units[i]->s, 4, cudaMemcpyDeviceToHost, sv->compute);
        cudaMemcpyAsync(sv->h_flags + sv->flag_slots + 1 + i, units[i]->dflag + units[i]->S + 2 + units[i]->s, 4,
                        cudaMemcpyDeviceToHost, sv->compute);
    }
    cudaMemcpyAsync(sv->h_flags + sv->flag_slots, p.status, 4, cudaMemcpyDeviceToHost, sv->compute);
    } else {
        sv->h_flags[sv->flag_slots] = 0;
    }
    // whole solves: domain check and every squaring in one launch each; the
    // result lands in P[1]; mailbox slot i <- entries outside the domain,
    // slot flag_slots + 1 + i <- barrier status
    for (int i = ninst; i < (int)units.size(); ++i) {
        Req *r = units[i];
        cudaStreamWaitEvent(sv->compute, r->in_ready, 0);
        int *info = r->dflag;  // 2S + 4 >= S + 5 ints
        cudaMemsetAsync(info, 0, (size_t)(2 * r->S + 4) * 4, sv->compute);
        cudaError_t e;
        if (r->n <= apsp_small_limit())
            e = launch_apsp_small(static_cast<const int *>(r->P[0]), r->ldp, r->n, r->S, true,
                                  static_cast<int *>(r->P[1]), r->ldp, info, sv->compute);
        else
            e = launch_apsp_mid(static_cast<const int *>(r->P[0]), r->ldp, r->n, r->S, true, true,
                                static_cast<int *>(r->P[1]), r->ldp, r->Q[0],
                                (size_t)(reinterpret_cast<char *>(r->dflag) - static_cast<char *>(r->Q[0])), info,
                                sv->compute);
        if (e != cudaSuccess) return -1;
        cudaMemcpyAsync(sv->h_flags + i, info, 4, cudaMemcpyDeviceToHost, sv->compute);
        cudaMemcpyAsync(sv->h_flags + sv->flag_slots + 1 + i, info + 3, 4, cudaMemcpyDeviceToHost, sv->compute);
    }
    cudaEventRecord(sv->step_done[par], sv->compute);
    sv->step_parity ^= 1;
    ++sv->steps;
    sv->units += (int)units.size();
    return (int)units.size();
}

void start_retire(btas_server_t *sv, Req *r) {
    if (r->bad) {
        // failed (W outside the domain): the caller's D is not written
    } else if (r->kind == 0) {
        cudaMemcpy2DAsync(r->hC, (size_t)r->n * 4, r->P[r->result_buf], r->ldp * 4, (size_t)r->n * 4, r->n,
                          cudaMemcpyDeviceToHost, sv->copy);
    } else {
        cudaMemcpy2DAsync(r->hC, (size_t)r->n * 4, r->dC, r->ldc_d * 4, (size_t)r->n * 4, r->m,
                          cudaMemcpyDeviceToHost, sv->copy);
    }
    cudaEventCreateWithFlags(&r->out_ready, cudaEventDisableTiming);
    cudaEventRecord(r->out_ready, sv->copy);
    sv->retiring.push_back(r);
}

void poll_retiring(btas_server_t *sv, bool block) {
    std::vector<Req *> keep;
    for (Req *r : sv->retiring) {
        const cudaError_t q = block ? cudaEventSynchronize(r->out_ready) : cudaEventQuery(r->out_ready);
        if (q == cudaSuccess) {
            const double t = sv->now();
            release(sv, r);
            std::lock_guard<std::mutex> lk(sv->mu);
            r->t_done = t;
            r->state = r->bad ? kFailed : kDone;
            sv->used -= (long long)r->bytes;
            ++sv->completed;
        } else {
            keep.push_back(r);
        }
    }
    sv->retiring.swap(keep);
    sv->cv.notify_all();
}

// The bulk lane: one large request at a time, in arrival order and within
// the budget, through the library's single calls on the bulk stream.  The
// result is the single call's result by construction.
void bulk_loop(btas_server_t *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                return (sv->stop && sv->bulk_queue.empty()) ||
                       (!sv->bulk_queue.empty() &&
                        sv->used + (long long)sv->bulk_queue.front()->bytes <= sv->budget);
            });
            if (sv->bulk_queue.empty()) break;
            r = sv->bulk_queue.front();
            sv->bulk_queue.pop_front();
            sv->bulk_busy = true;
            sv->used += (long long)r->bytes;
            r->state = kRunning;
            r->t_admit = sv->now();
        }
        // memory and copies on the lane's copy stream; the single call on the
        // compute stream, ordered by events in both directions
        const cudaStream_t cp = sv->bulk, cs = sv->bulk_compute;
        const double t_pick = sv->now();
        cudaEvent_t in_ev = nullptr, out_ev = nullptr;
        cudaEventCreateWithFlags(&in_ev, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&out_ev, cudaEventDisableTiming);
        bool ok = true;
        // the lane's own device block, reused by every large request
        const size_t need = r->kind == 0 ? 2 * a256((size_t)r->n * r->n * 4)
                                         : a256((size_t)r->m * r->k * 4) + a256((size_t)r->k * r->n * 4) +
                                               a256((size_t)r->m * r->n * 4);
        if (need > sv->bulk_cap) {
            if (sv->bulk_buf) cudaFreeAsync(sv->bulk_buf, cp);
            sv->bulk_buf = nullptr;
            sv->bulk_cap = 0;
            if (ws_alloc(&sv->bulk_buf, need, cp) == cudaSuccess) sv->bulk_cap = need;
            else ok = false;
        }
        void *dmem = ok ? sv->bulk_buf : nullptr;
        if (r->kind == 0) {
            const size_t nn = (size_t)r->n * r->n * 4;
            if (ok) {
                int32_t *W = static_cast<int32_t *>(dmem);
                int32_t *D = reinterpret_cast<int32_t *>(static_cast<char *>(dmem) + a256(nn));
                ok = cudaMemcpyAsync(W, r->hA, nn, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                     cudaEventRecord(in_ev, cp) == cudaSuccess && cudaStreamWaitEvent(cs, in_ev, 0) == cudaSuccess &&
                     btas_apsp(r->n, W, D, cs) == BTAS_OK && cudaEventRecord(out_ev, cs) == cudaSuccess &&
                     cudaStreamWaitEvent(cp, out_ev, 0) == cudaSuccess &&
                     cudaMemcpyAsync(r->hC, D, nn, cudaMemcpyDeviceToHost, cp) == cudaSuccess;
            }
        } else {
            const size_t ba = (size_t)r->m * r->k * 4, bb = (size_t)r->k * r->n * 4, bc = (size_t)r->m * r->n * 4;
            if (ok) {
                char *p = static_cast<char *>(dmem);
                void *A = p, *B = p + a256(ba), *C = p + a256(ba) + a256(bb);
                ok = cudaMemcpyAsync(A, r->hA, ba, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                     cudaMemcpyAsync(B, r->hB, bb, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                     cudaEventRecord(in_ev, cp) == cudaSuccess && cudaStreamWaitEvent(cs, in_ev, 0) == cudaSuccess &&
                     btas_gemm(r->sr, r->dtype, r->m, r->n, r->k, A, r->k, B, r->n, C, r->n, cs) == BTAS_OK &&
                     cudaEventRecord(out_ev, cs) == cudaSuccess && cudaStreamWaitEvent(cp, out_ev, 0) == cudaSuccess &&
                     cudaMemcpyAsync(r->hC, C, bc, cudaMemcpyDeviceToHost, cp) == cudaSuccess;
            }
        }
        if (!ok) {
            // the compute stream may still hold work of this request: the copy
            // stream waits for it before the block is returned
            cudaEventRecord(out_ev, cs);
            cudaStreamWaitEvent(cp, out_ev, 0);
        }
        const double t_call = sv->now();
        if (cudaStreamSynchronize(cp) != cudaSuccess) ok = false;
        if (log_level() >= 1)
            log_event("server bulk lane: %s n=%d: call returned after %.3f ms, result in host memory %.3f ms later",
                      r->kind == 0 ? "apsp" : "product", r->n, (t_call - t_pick) * 1e3, (sv->now() - t_call) * 1e3);
        cudaEventDestroy(in_ev);
        cudaEventDestroy(out_ev);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->t_done = sv->now();
            r->state = ok ? kDone : kFailed;
            sv->used -= (long long)r->bytes;
            ++sv->completed;
            ++sv->bulk_runs;
            sv->bulk_busy = false;
        }
        sv->cv.notify_all();
    }
}

// Admission: queued requests in arrival order while their device footprint
// fits the budget.  Worker thread only.
void admit_queued(btas_server_t *sv, bool wait_if_idle) {
    std::vector<Req *> admitted;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        if (wait_if_idle && sv->queue.empty() && sv->active.empty() && sv->retiring.empty() && !sv->stop)
            sv->cv.wait_for(lk, std::chrono::milliseconds(2));
        while (!sv->queue.empty() && sv->used + (long long)sv->queue.front()->bytes <= sv->budget) {
            Req *r = sv->queue.front();
            sv->queue.pop_front();
            sv->used += (long long)r->bytes;
            admitted.push_back(r);
        }
    }
    for (Req *r : admitted) {
        const double t = sv->now();
        const bool ok = admit(sv, r);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->t_admit = t;
            if (!ok) {
                r->state = kFailed;
                sv->used -= (long long)r->bytes;
            } else {
                r->state = kRunning;
            }
        }
        if (ok) sv->active.push_back(r);
    }
    if (!admitted.empty()) sv->cv.notify_all();
}

void worker_loop(btas_server_t *sv) {
    cudaSetDevice(sv->device);
    std::vector<Req *> units;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->stop && sv->queue.empty() && sv->active.empty() && sv->retiring.empty()) break;
        }
        admit_queued(sv, true);
        const int launched = launch_step(sv, units);
        poll_retiring(sv, false);
        if (launched < 0) {
            sv->last_error = BTAS_ERR_CUDA;
            break;
        }
        if (launched == 0) {
            // nothing to launch: result copies may still be in flight
            if (!sv->retiring.empty()) std::this_thread::yield();
            continue;
        }
        // while the step runs: admit arrivals (their input copies overlap the
        // step) and retire finished copies; then advance every unit
        const cudaEvent_t step_ev = sv->step_done[sv->step_parity ^ 1];
        while (cudaEventQuery(step_ev) == cudaErrorNotReady) {
            admit_queued(sv, false);
            poll_retiring(sv, false);
            std::this_thread::yield();
        }
        if (sv->h_flags[sv->flag_slots] != 0) sv->last_error = sv->h_flags[sv->flag_slots];
        for (int i = 0; i < (int)units.size(); ++i) {
            Req *r = units[i];
            ++r->steps;
            bool finished = true;
            if (r->whole) {
                // the one-block kernel reports no barrier status (its slot stays 0)
                r->bad = sv->h_flags[i] != 0 || (r->n > apsp_small_limit() && sv->h_flags[sv->flag_slots + 1 + i] != 0);
                r->result_buf = 1;
                r->s = r->S + 1;
            } else {
                // a unit that ran a chunk of its tiles continues in the next step
                // (a domain violation ends the request at once)
                const bool bad = r->kind == 0 && r->s == 1 && sv->h_flags[2 * sv->flag_slots + 1 + i] != 0;
                r->tile_next += r->take;
                if (!bad && r->tile_next < r->unit_tiles()) continue;
                r->tile_next = 0;
                if (r->kind == 0) {
                    const bool changed = sv->h_flags[i] != 0;
                    r->last_max = r->s < r->S ? sv->h_flags[sv->flag_slots + 1 + i] : -1;
                    r->result_buf = r->s & 1;
                    r->bad = bad;
                    finished = r->bad || !changed || r->s >= r->S;
                    ++r->s;
                }
            }
            if (finished) {
                r->finished = true;
                start_retire(sv, r);
            }
        }
        // keep admission order for the requests with work left
        std::vector<Req *> still;
        for (Req *r : sv->active)
            if (!r->finished) still.push_back(r);
        sv->active.swap(still);
    }
    poll_retiring(sv, true);
}

}  // namespace

extern "C" {

btas_status btas_server_create(btas_server_t **out, int64_t hbm_budget_bytes, int flags) {
    if (!out || hbm_budget_bytes <= 0) return sfail(BTAS_ERR_ARG, "btas_server_create: bad arguments");
    if (flags != 0) return sfail(BTAS_ERR_ARG, "btas_server_create: unknown flags");
    btas_server_t *sv = new btas_server_t();
    sv->budget = hbm_budget_bytes;
    sv->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&sv->device);
    int per_sm = 0, sms = 0;
    // the bulk lane's streams get the highest priority, the step loop's the lowest
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (batch_kernel_prepare(&per_sm) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sv->compute, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sv->copy, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sv->bulk, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sv->bulk_compute, cudaStreamNonBlocking, prio_high) != cudaSuccess) {
        delete sv;
        return sfail(BTAS_ERR_CUDA, "btas_server_create: CUDA set-up failed");
    }
    sv->grid = std::max(1, per_sm * sms);
    // memory freed by retired requests stays cached in the library's pool up
    // to the budget (plus the single calls' workspace): otherwise every
    // synchronisation above the pool's threshold hands memory back to the
    // driver and the next large allocation maps it again
    ws_keep_at_least((uint64_t)hbm_budget_bytes + (4ULL << 30));
    if (const char *e = getenv("BTAS_SERVER_STEP_TERMS")) sv->step_terms = atof(e) > 0 ? atof(e) : sv->step_terms;
    if (const char *e = getenv("BTAS_SERVER_NO_U16")) sv->allow_u16 = (*e && atoi(e) != 0) ? 0 : 1;
    if (const char *e = getenv("BTAS_SERVER_NO_WHOLE")) sv->allow_whole = (*e && atoi(e) != 0) ? 0 : 1;
    if (const char *e = getenv("BTAS_SERVER_BULK_TERMS")) sv->bulk_terms = atof(e);
    sv->timeout_cycles = batch_timeout_cycles(sv->device);
    sv->flag_slots = 1 << 16;
    if (cudaMallocHost(reinterpret_cast<void **>(&sv->h_flags), (size_t)(3 * sv->flag_slots + 1) * 4) != cudaSuccess) {
        delete sv;
        return sfail(BTAS_ERR_NOMEM, "btas_server_create: pinned mailbox");
    }
    for (int q = 0; q < 2; ++q) {
        cudaEventCreateWithFlags(&sv->step_done[q], cudaEventDisableTiming);
        cudaEventRecord(sv->step_done[q], sv->compute);
    }
    sv->worker = std::thread(worker_loop, sv);
    sv->bulk_worker = std::thread(bulk_loop, sv);
    *out = sv;
    return BTAS_OK;
}

static btas_status enqueue(btas_server_t *sv, Req *r, int64_t *ticket) {
    r->bytes = footprint(*r);
    if ((long long)r->bytes > sv->budget) {
        delete r;
        return sfail(BTAS_ERR_BUDGET, "btas_server: request larger than the device-memory budget");
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
        delete r;
        return sfail(BTAS_ERR_ARG, "btas_server: server is stopping");
    }
    if ((int64_t)sv->active.size() + (int64_t)sv->queue.size() + (int64_t)sv->bulk_queue.size() >= sv->flag_slots) {
        delete r;
        return sfail(BTAS_ERR_BUDGET, "btas_server: too many requests in flight");
    }
    r->id = sv->next_id++;
    r->t_submit = sv->now();
    // large requests take the bulk lane (BTAS_SERVER_BULK_TERMS <= 0 turns it off)
    r->bulk = sv->bulk_terms > 0 && (r->kind == 0 ? r->n > apsp_mid_max_n() : r->unit_terms() > sv->bulk_terms);
    if (r->bulk) sv->bulk_queue.push_back(r);
    else sv->queue.push_back(r);
    sv->all[r->id] = r;
    if (ticket) *ticket = r->id;
    sv->cv.notify_all();
    return BTAS_OK;
}

btas_status btas_server_submit_apsp(btas_server_t *sv, int64_t n, const int32_t *W, int32_t *D, int64_t *ticket) {
    if (!sv || !W || !D || n < 1 || n > 46340) return sfail(BTAS_ERR_ARG, "btas_server_submit_apsp: bad arguments");
    Req *r = new Req();
    r->kind = 0;
    r->m = r->n = r->k = (int)n;
    r->S = squarings_of(n);
    if (r->S == 0) r->S = 1;  // n <= 2: one squaring leaves W unchanged (zero diagonal)
    r->hA = W;
    r->hC = D;
    return enqueue(sv, r, ticket);
}

btas_status btas_server_submit_gemm(btas_server_t *sv, int semiring, int dtype, int64_t m, int64_t n, int64_t k,
                                    const void *A, const void *B, void *C, int64_t *ticket) {
    if (!sv || !A || !B || !C || m < 1 || n < 1 || k < 1 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
        return sfail(BTAS_ERR_ARG, "btas_server_submit_gemm: bad arguments");
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) return sfail(BTAS_ERR_ARG, "semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return sfail(BTAS_ERR_UNSUPPORTED, "dtype");
    Req *r = new Req();
    r->kind = 1;
    r->sr = semiring;
    r->dtype = dtype;
    r->m = (int)m;
    r->n = (int)n;
    r->k = (int)k;
    r->hA = A;
    r->hB = B;
    r->hC = C;
    return enqueue(sv, r, ticket);
}

btas_status btas_server_poll(btas_server_t *sv, int64_t ticket, int *state, double *t_submit, double *t_admit,
                             double *t_done) {
    if (!sv) return sfail(BTAS_ERR_ARG, "btas_server_poll: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return sfail(BTAS_ERR_ARG, "btas_server_poll: unknown ticket");
    const Req *r = it->second;
    if (state) *state = r->state;
    if (t_submit) *t_submit = r->t_submit;
    if (t_admit) *t_admit = r->t_admit;
    if (t_done) *t_done = r->t_done;
    return BTAS_OK;
}

btas_status btas_server_wait_all(btas_server_t *sv, double timeout_s) {
    if (!sv) return sfail(BTAS_ERR_ARG, "btas_server_wait_all: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        bool busy = !sv->queue.empty() || !sv->bulk_queue.empty();
        for (auto &kv : sv->all)
            if (kv.second->state == kQueued || kv.second->state == kRunning) busy = true;
        if (!busy) break;
        if (sv->last_error) return sfail(static_cast<btas_status>(sv->last_error), "btas_server: device error");
        if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout)
            return sfail(BTAS_ERR_TIMEOUT, "btas_server_wait_all: timed out");
    }
    if (sv->last_error) return sfail(static_cast<btas_status>(sv->last_error), "btas_server: device error");
    return BTAS_OK;
}

btas_status btas_server_stats(btas_server_t *sv, int64_t *steps, int64_t *units, int64_t *completed,
                              int64_t *bytes_in_use) {
    if (!sv) return sfail(BTAS_ERR_ARG, "btas_server_stats: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (steps) *steps = sv->steps;
    if (units) *units = sv->units;
    if (completed) *completed = sv->completed;
    if (bytes_in_use) *bytes_in_use = sv->used;
    return BTAS_OK;
}

btas_status btas_server_destroy(btas_server_t *sv) {
    if (!sv) return BTAS_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->bulk_worker.joinable()) sv->bulk_worker.join();
    cudaStreamSynchronize(sv->compute);
    cudaStreamSynchronize(sv->copy);
    cudaStreamSynchronize(sv->bulk);
    cudaStreamSynchronize(sv->bulk_compute);
    if (sv->bulk_buf) ws_free(sv->bulk_buf, sv->bulk);
    for (auto &kv : sv->all) {
        release(sv, kv.second);
        delete kv.second;
    }
    for (int q = 0; q < 2; ++q) {
        if (sv->d_stage[q]) cudaFree(sv->d_stage[q]);
        if (sv->h_stage[q]) cudaFreeHost(sv->h_stage[q]);
        if (sv->step_done[q]) cudaEventDestroy(sv->step_done[q]);
    }
    if (sv->h_flags) cudaFreeHost(sv->h_flags);
    cudaStreamSynchronize(sv->copy);
    cudaStreamDestroy(sv->compute);
    cudaStreamDestroy(sv->copy);
    cudaStreamDestroy(sv->bulk);
    cudaStreamDestroy(sv->bulk_compute);
    delete sv;
    return BTAS_OK;
}

}  // extern "C"
