// C-ABI entry points declared in include/btas.h: argument validation, kernel
// selection, stream-ordered workspace, and the APSP squaring driver.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "kernels.h"

namespace btas {
extern const GemmKernel kGemmI32Dpx[];
extern const int kGemmI32DpxCount;
extern const GemmKernel kGemmI32Mix[];
extern const int kGemmI32MixCount;
extern const GemmKernel kGemmF32[];
extern const int kGemmF32Count;
}  // namespace btas

using namespace btas;

namespace btas {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// One workspace pool per device, created on first use, with a release
// threshold so that freed blocks stay cached between calls.
static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;

static cudaError_t device_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        const char *keep = getenv("BTAS_POOL_KEEP_MB");
        uint64_t thr = (uint64_t)((keep && *keep) ? atoll(keep) : 4096) << 20;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr)) != cudaSuccess) return e;
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

cudaError_t ws_alloc(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

cudaError_t ws_free(void *p, cudaStream_t st) { return cudaFreeAsync(p, st); }

cudaError_t ws_keep_at_least(uint64_t bytes) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    uint64_t cur = 0;
    if ((e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur)) != cudaSuccess) return e;
    if (cur >= bytes) return cudaSuccess;
    return cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
}

// BTAS_LOG=1 (read once) prints each entry point's execution choices to
// stderr; 0 or unset prints nothing.
int log_level() {
    static const int level = [] {
        const char *v = getenv("BTAS_LOG");
        return v && *v ? atoi(v) : 0;
    }();
    return level;
}

void log_event(const char *fmt, ...) {
    if (log_level() <= 0) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fprintf(stderr, "[btas] %s\n", buf);
}

static std::mutex g_dev_mu;
static std::vector<DeviceInfo> g_dev_info;
static std::set<std::pair<int, const void *>> g_smem_set;

bool current_device_info(DeviceInfo *out, int *device) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (device) *device = dev;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if ((int)g_dev_info.size() <= dev) g_dev_info.resize(dev + 1, DeviceInfo{0, 0, 0});
    DeviceInfo &d = g_dev_info[dev];
    if (d.sms == 0) {
        int ma = 0, mi = 0, sms = 0, khz = 0;
        if (cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
            return false;
        d = DeviceInfo{ma * 10 + mi, sms, khz > 0 ? khz : 2000000};
    }
    *out = d;
    return true;
}

cudaError_t set_smem_once(const void *func, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (g_smem_set.count({dev, func})) return cudaSuccess;
    }
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    g_smem_set.insert({dev, func});
    return cudaSuccess;
}
}  // namespace btas

namespace {

thread_local std::string g_err = "no error";

// A small device -> host read-back followed by a wait for the stream, through
// a per-thread pinned mailbox (a copy into pageable memory is staged by the
// driver and takes longer).
cudaError_t read_back(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    struct Mailbox {
        void *p = nullptr;
        ~Mailbox() {
            if (p) cudaFreeHost(p);
        }
    };
    thread_local Mailbox mb;
    constexpr size_t kCap = 4096;
    if (bytes <= kCap && !mb.p && cudaMallocHost(&mb.p, kCap) != cudaSuccess) {
        cudaGetLastError();
        mb.p = nullptr;
    }
    void *tgt = (bytes <= kCap && mb.p) ? mb.p : dst;
    cudaError_t e = cudaMemcpyAsync(tgt, src, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && tgt != dst) memcpy(dst, tgt, bytes);
    return e;
}

btas_status fail(btas_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

btas_status cuda_fail(cudaError_t e, const char *what) {
    return fail(BTAS_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define BTAS_CUDA(call, what)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Stream-ordered scratch that is released on the same stream when it goes
// out of scope.
struct Workspace {
    void *p = nullptr;
    cudaStream_t st;
    explicit Workspace(cudaStream_t s) : st(s) {}
    cudaError_t alloc(size_t bytes) { return bytes ? ws_alloc(&p, bytes, st) : cudaSuccess; }
    ~Workspace() {
        if (p) ws_free(p, st);
    }
};

// An NVTX range around one entry point (visible to Nsight tools; a no-op
// without one attached).
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool aligned16(const void *p, long long ld) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld & 3) == 0;
}

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v && *v ? atoi(v) : dflt;
}

// Kernel choice.  Explicit environment overrides win: BTAS_I32_VARIANT (0 =
// DPX, 1 = mixed), BTAS_I32_NS, BTAS_F32_VARIANT (2 = f32x2, 3 = scalar, 4 =
// two scalar adds + 3-input min) and BTAS_CFG.  Otherwise an autotuner entry
// for the problem's size buckets (tune.cu), else the defaults measured on
// GB300 at 8192^3, where the 2-CTA/SM, 64-bit-fragment tiles reach the
// measured issue ceilings of their instruction mixes: int32 = IMAD/3-input-min
// mix on 4 of 8 columns, fp32 = add.f32x2 + 3-input min; 64 x 64 tiles when
// the 128 x 128 tiles would not fill one wave of 2 CTAs per SM.
const GemmKernel *select_kernel(int dtype, int sr, long long m, long long n, long long k, cudaStream_t st,
                                int *group_m) {
    *group_m = 8;
    const bool forced = getenv("BTAS_I32_VARIANT") || getenv("BTAS_I32_NS") || getenv("BTAS_F32_VARIANT") ||
                        getenv("BTAS_CFG");
    TuneChoice c{};
    if (!forced && tune_choice(sr, dtype, m, n, k, st, &c)) {
        const GemmKernel *t = find_gemm_kernel(c.var, sr, c.ns, c.cfg);
        if (t) {
            *group_m = c.group_m;
            log_event("product %lldx%lldx%lld %s %s: variant %d ns %d cfg %d group %d (autotuner)", m, n, k,
                      dtype == BTAS_F32 ? "fp32" : "int32", sr == kMin ? "min-plus" : "max-plus", t->var, t->ns,
                      t->cfg, c.group_m);
            return t;
        }
    }
    int var, ns = 0;
    if (dtype == BTAS_F32) {
        var = env_int("BTAS_F32_VARIANT", kF32X2);
    } else {
        var = env_int("BTAS_I32_VARIANT", kI32Mix);
        ns = var == kI32Mix ? env_int("BTAS_I32_NS", 4) : 0;
    }
    // 128 x 128 tiles at 2 CTAs/SM once they fill at least one full wave
    DeviceInfo di{};
    const int sms = current_device_info(&di) ? di.sms : 152;
    const long long big_tiles = ((m + 127) / 128) * ((n + 127) / 128);
    int cfg = env_int("BTAS_CFG", big_tiles >= 2LL * sms ? 4 : 2);
    const GemmKernel *kk = find_gemm_kernel(var, sr, ns, cfg);
    if (!kk && dtype == BTAS_I32) kk = find_gemm_kernel(kI32Mix, sr, 5, cfg);
    if (!kk) kk = find_gemm_kernel(var, sr, ns, 0);
    if (!kk && dtype == BTAS_I32) kk = find_gemm_kernel(kI32Mix, sr, 5, 0);
    if (!kk && dtype == BTAS_I32) kk = find_gemm_kernel(kI32Dpx, sr, 0, 0);
    if (!kk && dtype == BTAS_F32) kk = find_gemm_kernel(kF32X2, sr, 0, 0);
    if (kk)
        log_event("product %lldx%lldx%lld %s %s: variant %d ns %d cfg %d group 8 (%s)", m, n, k,
                  dtype == BTAS_F32 ? "fp32" : "int32", sr == kMin ? "min-plus" : "max-plus", kk->var, kk->ns,
                  kk->cfg, forced ? "environment" : "defaults");
    return kk;
}

// IMAD/DPX split of the packed u16x2 kernel: BTAS_U16_NS, else the
// autotuner's entry, else 5.
int u16_ns(long long m, long long n, long long k, cudaStream_t st) {
    if (getenv("BTAS_U16_NS")) return env_int("BTAS_U16_NS", 5);
    TuneChoice c{};
    if (tune_choice(kMin, BTAS_U16, m, n, k, st, &c)) return c.ns;
    return 5;
}

// Run the NT kernel on A (m x k) and Bt (n x k).
btas_status run_nt(int dtype, int sr, const GemmArgs &a, cudaStream_t st) {
    int group_m = 8;
    const GemmKernel *k = select_kernel(dtype, sr, a.m, a.n, a.k, st, &group_m);
    if (!k) return fail(BTAS_ERR_UNSUPPORTED, "no kernel for dtype %d semiring %d", dtype, sr);
    GemmArgs args = a;
    args.group_m = group_m;
    args.one = 1;
    {
        // Grids of two or more waves: groups of 16 tile columns and k run
        // backwards in every other wave (GemmArgs::kwave), which cuts the
        // DRAM re-reads of the operand panels by a fifth to a quarter at the
        // same speed.  BTAS_KWAVE=0 keeps the row-group raster.
        DeviceInfo di{};
        const int sms = current_device_info(&di) ? di.sms : 152;
        const long long tiles = (long long)((a.m + k->bm - 1) / k->bm) * ((a.n + k->bn - 1) / k->bn);
        if (tiles >= 4LL * sms && env_int("BTAS_KWAVE", 1) != 0) {
            args.kwave = sms;
            args.group_m = 16;
        }
    }
    // one standalone launch never writes its own operands
    args.ro_a = args.ro_b = 1;
    BTAS_CUDA(k->launch(args, st), "tropical gemm launch");
    return BTAS_OK;
}

uint32_t ident_bits(int dtype, int sr) {
    if (dtype == BTAS_I32) return static_cast<uint32_t>(sr == kMin ? kInfI32 : kNinfI32);
    return sr == kMin ? 0x7f800000u : 0xff800000u;
}

}  // namespace

namespace btas {
void record_error(const char *msg) { g_err = msg; }

const GemmKernel *find_gemm_kernel(int var, int sr, int ns, int cfg) {
    for (int i = 0; i < gemm_kernel_count(); ++i) {
        const GemmKernel &k = *gemm_kernel_at(i);
        if (k.var == var && k.sr == sr && k.cfg == cfg && (var != kI32Mix || k.ns == ns)) return &k;
    }
    return nullptr;
}

int gemm_kernel_count() { return kGemmI32DpxCount + kGemmI32MixCount + kGemmF32Count; }

const GemmKernel *gemm_kernel_at(int i) {
    if (i < 0) return nullptr;
    if (i < kGemmI32DpxCount) return &kGemmI32Dpx[i];
    i -= kGemmI32DpxCount;
    if (i < kGemmI32MixCount) return &kGemmI32Mix[i];
    i -= kGemmI32MixCount;
    if (i < kGemmF32Count) return &kGemmF32[i];
    return nullptr;
}
}  // namespace btas

extern "C" {

int btas_version(void) { return 100; }

int64_t btas_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t btas_workspace_reserved(void) {
    cudaMemPool_t pool = nullptr;
    if (device_pool(&pool) != cudaSuccess) return -1;
    uint64_t v = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) return -1;
    return (int64_t)v;
}

btas_status btas_workspace_trim(void) {
    cudaMemPool_t pool = nullptr;
    BTAS_CUDA(device_pool(&pool), "workspace pool");
    BTAS_CUDA(cudaDeviceSynchronize(), "synchronise");
    BTAS_CUDA(cudaMemPoolTrimTo(pool, 0), "trim");
    return BTAS_OK;
}

const char *btas_last_error_string(void) { return g_err.c_str(); }

int btas_apsp_squarings(int64_t n) {
    int s = 0;
    int64_t reach = 1;
    while (reach < n - 1) {
        reach *= 2;
        ++s;
    }
    return s;
}

btas_status btas_gemm(int semiring, int dtype, int64_t m, int64_t n, int64_t k, const void *A, int64_t lda,
                      const void *B, int64_t ldb, void *C, int64_t ldc, void *stream) {
    Trace trace_("btas_gemm");
    const int sr = semiring & 0xff;
    const bool accumulate = (semiring & BTAS_GEMM_ACCUMULATE) != 0;
    const bool trans_b = (semiring & BTAS_GEMM_TRANS_B) != 0;
    const bool packed = (semiring & BTAS_GEMM_PACKED) != 0;
    const bool checked = (semiring & BTAS_GEMM_CHECKED) != 0;
    if (semiring & ~(0xff | BTAS_GEMM_ACCUMULATE | BTAS_GEMM_TRANS_B | BTAS_GEMM_NO_CARRIER | BTAS_GEMM_PACKED |
                     BTAS_GEMM_CHECKED))
        return fail(BTAS_ERR_ARG, "btas_gemm: unknown flag bits 0x%x", semiring);
    if (sr != BTAS_MINPLUS && sr != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "btas_gemm: unknown semiring %d", sr);
    if (dtype != BTAS_I32 && dtype != BTAS_F32 && dtype != BTAS_U16)
        return fail(BTAS_ERR_ARG, "btas_gemm: unknown dtype %d", dtype);
    if (m < 0 || n < 0 || k < 0) return fail(BTAS_ERR_ARG, "btas_gemm: negative size");
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return fail(BTAS_ERR_ARG, "btas_gemm: size beyond 2^31-1");
    if (lda < (k > 1 ? k : 1)) return fail(BTAS_ERR_ARG, "btas_gemm: lda %lld < k", (long long)lda);
    if (ldb < (trans_b ? (k > 1 ? k : 1) : (n > 1 ? n : 1)))
        return fail(BTAS_ERR_ARG, "btas_gemm: ldb %lld too small", (long long)ldb);
    if (ldc < (n > 1 ? n : 1)) return fail(BTAS_ERR_ARG, "btas_gemm: ldc %lld < n", (long long)ldc);
    if (m == 0 || n == 0) return BTAS_OK;
    if (!C || (k > 0 && (!A || !B))) return fail(BTAS_ERR_ARG, "btas_gemm: NULL pointer");
    if (dtype == BTAS_U16 && sr != BTAS_MINPLUS)
        return fail(BTAS_ERR_UNSUPPORTED, "btas_gemm: BTAS_U16 is min-plus only");
    if (checked && dtype == BTAS_U16)
        return fail(BTAS_ERR_UNSUPPORTED, "btas_gemm: BTAS_GEMM_CHECKED takes BTAS_I32 or BTAS_F32");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    if (dtype == BTAS_U16) {
        if (trans_b) return fail(BTAS_ERR_UNSUPPORTED, "btas_gemm: BTAS_U16 takes B untransposed");
        if (k == 0) {
            if (accumulate) return BTAS_OK;
            return fail(BTAS_ERR_UNSUPPORTED, "btas_gemm: BTAS_U16 with k == 0");
        }
        U16Args a{};
        a.m = (int)m; a.n = (int)n; a.k = (int)k;
        a.A = static_cast<const uint16_t *>(A); a.lda = lda;
        a.B = static_cast<const uint16_t *>(B); a.ldb = ldb;
        a.C = static_cast<uint16_t *>(C); a.ldc = ldc;
        a.one = 1;
        if (accumulate) return fail(BTAS_ERR_UNSUPPORTED, "btas_gemm: BTAS_U16 accumulate");
        Workspace ws(st);
        BTAS_CUDA(ws.alloc((size_t)m * ((k + 3) & ~3LL) * 4), "workspace alloc");
        BTAS_CUDA(launch_tgemm_u16_ws(a, static_cast<uint32_t *>(ws.p), u16_ns(m, n, k, st), st),
                  "u16 gemm launch");
        return BTAS_OK;
    }

    if (k == 0) {
        if (accumulate) return BTAS_OK;
        BTAS_CUDA(launch_fill4(C, ldc, (int)m, (int)n, ident_bits(dtype, sr), st), "fill");
        return BTAS_OK;
    }

    // BTAS_GEMM_CHECKED: count the operand entries outside the domain on the
    // device; a call that finds any leaves C unwritten, and btas_sync_status
    // reports it.  chk[0] = this call's count, chk[1] = skip word of the
    // product kernels.
    Workspace chk_ws(st);
    int *chk = nullptr;
    unsigned long long *status = nullptr;
    if (checked) {
        status = device_status_words();
        if (!status) return fail(BTAS_ERR_CUDA, "btas_gemm: device status words unavailable");
        BTAS_CUDA(chk_ws.alloc(256), "workspace alloc");
        chk = static_cast<int *>(chk_ws.p);
        BTAS_CUDA(cudaMemsetAsync(chk, 0, 8, st), "memset");
        const int is_f = dtype == BTAS_F32 ? 1 : 0;
        BTAS_CUDA(launch_domain_check(A, lda, (int)m, (int)k, is_f, sr, chk, status, st), "domain check");
        BTAS_CUDA(launch_domain_check(B, ldb, trans_b ? (int)n : (int)k, trans_b ? (int)k : (int)n, is_f, sr, chk,
                                      status, st),
                  "domain check");
        if (accumulate)
            BTAS_CUDA(launch_domain_check(C, ldc, (int)m, (int)n, is_f, sr, chk, status, st), "domain check");
    }

    Workspace ws(st);
    const void *Bt = B;
    long long ldbt = ldb;
    const long long ldt = (k + 3) & ~3LL;
    const size_t bt_bytes = trans_b ? 0 : align256((size_t)n * ldt * 4);
    int *pack_state = nullptr;
    if (packed && dtype == BTAS_I32) {
        log_event("product %lldx%lldx%lld int32: packed path requested (range check and choice on the device)",
                  (long long)m, (long long)n, (long long)k);
        // exact packed path, chosen on the device (pack.cu); the int32 path
        // below is enqueued too and bypassed when the packed one runs
        const long long ldad = (k + 3) & ~3LL, ldbu = (n + 7) & ~7LL;
        const size_t s_state = align256(kPackStateInts * 4), s_ad = align256((size_t)m * ldad * 4),
                     s_bu = align256((size_t)k * ldbu * 2), s_cu = align256((size_t)m * ldbu * 2);
        BTAS_CUDA(ws.alloc(bt_bytes + s_state + s_ad + s_bu + s_cu), "workspace alloc");
        char *base = static_cast<char *>(ws.p) + bt_bytes;
        pack_state = reinterpret_cast<int *>(base);
        uint32_t *adup = reinterpret_cast<uint32_t *>(base + s_state);
        uint16_t *bu = reinterpret_cast<uint16_t *>(base + s_state + s_ad);
        uint16_t *cu = reinterpret_cast<uint16_t *>(base + s_state + s_ad + s_bu);
        BTAS_CUDA(launch_pack_prepare(sr, (int)m, (int)n, (int)k, static_cast<const int *>(A), lda,
                                      static_cast<const int *>(B), ldb, trans_b, pack_state, adup, bu, ldbu, st,
                                      chk),
                  "packed operands");
        if (checked) BTAS_CUDA(launch_checked_gate(chk, pack_state, chk + 1, status, st), "checked gate");
        U16Args a{};
        a.m = (int)m; a.n = (int)n; a.k = (int)k;
        a.B = bu; a.ldb = ldbu;
        a.C = cu; a.ldc = ldbu;
        a.one = 1;
        a.gate = pack_state + kPackStateUse;
        a.adup_ready = true;
        BTAS_CUDA(launch_tgemm_u16_ws(a, adup, u16_ns(m, n, k, st), st), "packed product");
        BTAS_CUDA(launch_pack_finish(sr, (int)m, (int)n, cu, ldbu, pack_state, static_cast<int *>(C), ldc,
                                     accumulate, st),
                  "packed result");
    } else if (!trans_b) {
        BTAS_CUDA(ws.alloc(bt_bytes), "workspace alloc");
    }
    if (!trans_b) {
        BTAS_CUDA(launch_transpose4(B, ldb, (int)k, (int)n, ws.p, ldt, 0,
                                    pack_state ? pack_state + kPackStateNotUse : nullptr, st),
                  "transpose B");
        Bt = ws.p;
        ldbt = ldt;
    }
    GemmArgs a{};
    a.m = (int)m; a.n = (int)n; a.k = (int)k;
    a.A = A; a.lda = lda;
    a.Bt = Bt; a.ldb = ldbt;
    a.C = C; a.ldc = ldc;
    a.accumulate = accumulate ? 1 : 0;
    a.vec_a = aligned16(A, lda);
    a.vec_b = aligned16(Bt, ldbt);
    a.bypass = pack_state ? pack_state + kPackStateUse : nullptr;
    if (checked) {
        if (!pack_state) BTAS_CUDA(launch_checked_gate(chk, nullptr, chk + 1, status, st), "checked gate");
        a.bypass = chk + 1;
    }
    return run_nt(dtype, sr, a, st);
}

btas_status btas_sync_status(void *stream, int64_t *out_of_domain, int64_t *calls) {
    unsigned long long *status = device_status_words();
    if (!status) return fail(BTAS_ERR_CUDA, "btas_sync_status: device status words unavailable");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long h[2] = {0, 0};
    BTAS_CUDA(cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, st), "status read");
    BTAS_CUDA(cudaStreamSynchronize(st), "synchronise");
    BTAS_CUDA(cudaMemsetAsync(status, 0, sizeof h, st), "status clear");
    if (out_of_domain) *out_of_domain = (int64_t)h[0];
    if (calls) *calls = (int64_t)h[1];
    if (h[0] != 0)
        return fail(BTAS_ERR_ARG, "btas_sync_status: %llu checked product(s) found %llu operand entries outside the "
                    "domain and left C unwritten", h[1], h[0]);
    return BTAS_OK;
}

int64_t btas_packed_products(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    return packed_products(dev);
}

// ----------------------------------------------------------------- level 2

btas_status btas_gemv(int semiring, int dtype, int trans, int64_t m, int64_t n, const void *A, int64_t lda,
                      const void *x, void *y, void *stream) {
    Trace trace_("btas_gemv");
    const int sr = semiring & 0xff;
    const bool accumulate = (semiring & BTAS_GEMM_ACCUMULATE) != 0;
    if (semiring & ~(0xff | BTAS_GEMM_ACCUMULATE)) return fail(BTAS_ERR_ARG, "btas_gemv: unknown flags");
    if (sr != BTAS_MINPLUS && sr != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "btas_gemv: semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return fail(BTAS_ERR_ARG, "btas_gemv: dtype");
    if (trans != 0 && trans != 1) return fail(BTAS_ERR_ARG, "btas_gemv: trans must be 0 or 1");
    if (m < 0 || n < 0 || m > INT32_MAX || n > INT32_MAX) return fail(BTAS_ERR_ARG, "btas_gemv: sizes");
    if (lda < (n > 1 ? n : 1)) return fail(BTAS_ERR_ARG, "btas_gemv: lda < n");
    const int64_t ylen = trans ? n : m, xlen = trans ? m : n;
    if (ylen == 0) return BTAS_OK;
    if (!y || (xlen > 0 && (!A || !x))) return fail(BTAS_ERR_ARG, "btas_gemv: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (xlen == 0) {
        if (accumulate) return BTAS_OK;
        BTAS_CUDA(launch_fill4(y, ylen, 1, (int)ylen, ident_bits(dtype, sr), st), "fill");
        return BTAS_OK;
    }
    BTAS_CUDA(launch_gemv(sr, dtype, trans, (int)m, (int)n, A, lda, x, y, accumulate ? 1 : 0, nullptr, st), "gemv");
    return BTAS_OK;
}

btas_status btas_sssp(int64_t n, const int32_t *W, int64_t src, int32_t *dist, int *iterations, void *stream) {
    Trace trace_("btas_sssp");
    if (n < 0 || n > INT32_MAX) return fail(BTAS_ERR_ARG, "btas_sssp: n out of range");
    if (n == 0) {
        if (iterations) *iterations = 0;
        return BTAS_OK;
    }
    if (src < 0 || src >= n) return fail(BTAS_ERR_ARG, "btas_sssp: source out of range");
    if (!W || !dist) return fail(BTAS_ERR_ARG, "btas_sssp: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Relaxations are enqueued in groups of kGroup with one read-back per
    // group: relaxation t does nothing unless t - 1 changed d (its flag is
    // the next launch's gate), so the group's tail after the fixpoint costs
    // only empty launches and copies of an unchanged d.
    constexpr int kGroup = 8;
    Workspace ws(st);
    const size_t vb = align256((size_t)n * 4);
    BTAS_CUDA(ws.alloc(256 + 2 * vb), "workspace alloc");
    int *flag = static_cast<int *>(ws.p);  // [0, kGroup) change flags of a group, [8, 10) scan, [16] the constant 1
    int *d[2] = {reinterpret_cast<int *>(static_cast<char *>(ws.p) + 256),
                 reinterpret_cast<int *>(static_cast<char *>(ws.p) + 256 + vb)};
    // d_0 = e_src; d_{t+1} = d_t (x) W until unchanged (at most n-1 products):
    // in one cooperative launch (one grid barrier per product; the first
    // product checks the domain on its way through W), else
    // (BTAS_SSSP_NO_COOP=1, or no cooperative launch on this device) below
    if (n > 1 && n <= INT32_MAX / 4 && env_int("BTAS_SSSP_NO_COOP", 0) == 0) {
        Workspace cw(st);
        BTAS_CUDA(cw.alloc(sssp_coop_workspace(n) + 256), "workspace alloc");
        int *info = reinterpret_cast<int *>(static_cast<char *>(cw.p) + sssp_coop_workspace(n));
        BTAS_CUDA(cudaMemsetAsync(info, 0, 16, st), "memset");
        const cudaError_t le = launch_sssp_coop(W, n, (int)src, dist, cw.p, info, st);
        if (le == cudaSuccess) {
            int host[4] = {0, 0, 0, 0};
            BTAS_CUDA(read_back(host, info, 16, st), "info readback");
            if (host[1] != 0) return fail(BTAS_ERR_TIMEOUT, "btas_sssp: a bounded grid barrier wait expired");
            if (host[2] != 0) return fail(BTAS_ERR_ARG, "btas_sssp: %d entries outside the domain", host[2]);
            if (iterations) *iterations = host[0];
            log_event("sssp n=%lld: cooperative kernel, %d changing products", (long long)n, host[0]);
            return BTAS_OK;
        }
        if (le != cudaErrorCooperativeLaunchTooLarge && le != cudaErrorNotSupported)
            return fail(BTAS_ERR_CUDA, "btas_sssp: %s", cudaGetErrorString(le));
        cudaGetLastError();
    }
    {
        int host[2] = {0, 0};
        BTAS_CUDA(cudaMemsetAsync(flag, 0, 256, st), "memset");
        BTAS_CUDA(launch_apsp_scan(W, n, flag + 8, st), "domain scan");
        BTAS_CUDA(read_back(host, flag + 8, 8, st), "scan readback");
        if (host[1] != 0) return fail(BTAS_ERR_ARG, "btas_sssp: %d entries outside the domain", host[1]);
    }
    BTAS_CUDA(launch_fill4(d[0], n, 1, (int)n, static_cast<uint32_t>(kInfI32), st), "init");
    BTAS_CUDA(launch_fill4(flag + 16, 1, 1, 1, 1u, st), "init");
    const int zero = 0;
    BTAS_CUDA(cudaMemcpyAsync(d[0] + src, &zero, 4, cudaMemcpyHostToDevice, st), "init source");
    int cur = 0, steps = 0;
    bool done = false;
    for (int64_t t0 = 0; t0 + 1 < n && !done; t0 += kGroup) {
        const int g = (int)std::min<int64_t>(kGroup, n - 1 - t0);
        BTAS_CUDA(cudaMemsetAsync(flag, 0, kGroup * 4, st), "flag reset");
        for (int q = 0; q < g; ++q) {
            // the first relaxation of a group runs: the host saw the last one change d
            const int *gate = q == 0 ? flag + 16 : flag + q - 1;
            BTAS_CUDA(cudaMemcpyAsync(d[cur ^ 1], d[cur], (size_t)n * 4, cudaMemcpyDeviceToDevice, st), "copy");
            BTAS_CUDA(launch_gemv(kMin, BTAS_I32, 1, (int)n, (int)n, W, n, d[cur], d[cur ^ 1], 1, flag + q, st, gate),
                      "relax");
            cur ^= 1;
        }
        int host[kGroup] = {};
        BTAS_CUDA(read_back(host, flag, (size_t)g * 4, st), "flag readback");
        for (int q = 0; q < g; ++q) {
            if (!host[q]) {
                done = true;
                break;
            }
            ++steps;
        }
    }
    BTAS_CUDA(cudaMemcpyAsync(dist, d[cur], (size_t)n * 4, cudaMemcpyDeviceToDevice, st), "copy out");
    if (iterations) *iterations = steps;
    return BTAS_OK;
}

// ----------------------------------------------------------------- vectors

btas_status btas_dot(int semiring, int dtype, int64_t n, const void *x, int64_t incx, const void *y,
                     int64_t incy, void *result, void *stream) {
    Trace trace_("btas_dot");
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "btas_dot: semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return fail(BTAS_ERR_ARG, "btas_dot: dtype");
    if (n < 0 || incx < 1 || incy < 1) return fail(BTAS_ERR_ARG, "btas_dot: size or stride");
    if (!result || (n > 0 && (!x || !y))) return fail(BTAS_ERR_ARG, "btas_dot: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        BTAS_CUDA(launch_fill4(result, 1, 1, 1, ident_bits(dtype, semiring), st), "fill");
        return BTAS_OK;
    }
    long long nb = (n + 2047) / 2048;
    if (nb > 2 * 152) nb = 2 * 152;
    Workspace ws(st);
    BTAS_CUDA(ws.alloc((size_t)nb * 4), "workspace alloc");
    BTAS_CUDA(launch_dot(semiring, dtype, n, x, incx, y, incy, result, ws.p, (int)nb, st), "dot");
    return BTAS_OK;
}

btas_status btas_axpy(int semiring, int dtype, int64_t n, const void *alpha, const void *x, int64_t incx, void *y,
                      int64_t incy, void *stream) {
    Trace trace_("btas_axpy");
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "btas_axpy: semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return fail(BTAS_ERR_ARG, "btas_axpy: dtype");
    if (n < 0 || incx < 1 || incy < 1) return fail(BTAS_ERR_ARG, "btas_axpy: size or stride");
    if (n == 0) return BTAS_OK;
    if (!alpha || !x || !y) return fail(BTAS_ERR_ARG, "btas_axpy: NULL pointer");
    uint32_t bits;
    memcpy(&bits, alpha, 4);
    BTAS_CUDA(launch_axpy(semiring, dtype, n, bits, x, incx, y, incy, static_cast<cudaStream_t>(stream)), "axpy");
    return BTAS_OK;
}

static btas_status ewise(int op, int semiring, int dtype, int64_t n, const void *x, const void *y, void *z,
                         void *stream) {
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return fail(BTAS_ERR_ARG, "dtype");
    if (n < 0) return fail(BTAS_ERR_ARG, "negative size");
    if (n == 0) return BTAS_OK;
    if (!x || !y || !z) return fail(BTAS_ERR_ARG, "NULL pointer");
    BTAS_CUDA(launch_ewise(op, semiring, dtype, n, x, y, z, static_cast<cudaStream_t>(stream)), "elementwise");
    return BTAS_OK;
}

btas_status btas_add(int semiring, int dtype, int64_t n, const void *x, const void *y, void *z, void *stream) {
    return ewise(0, semiring, dtype, n, x, y, z, stream);
}

btas_status btas_mul(int semiring, int dtype, int64_t n, const void *x, const void *y, void *z, void *stream) {
    return ewise(1, semiring, dtype, n, x, y, z, stream);
}

// -------------------------------------------------------------------- APSP

// Squaring loop on 4-byte data (int32 or the fp32 carrier).  cur0 holds D_0
// (may be W itself).  bufs[0], bufs[1] are n x n ping-pong outputs; the
// last squaring writes bufs[last].  T is an n x n transpose buffer.  flags[s]
// is set when squaring s changed D.
static btas_status squaring_loop(int dtype, long long n, int S, const void *cur0, void *const bufs[2], void *T,
                                 int *flags, bool early_exit, cudaStream_t st) {
    const void *cur = cur0;
    const long long ldt = (n + 3) & ~3LL;
    for (int s = 0; s < S; ++s) {
        void *out = bufs[(S - 1 - s) & 1];
        const int *skip = (early_exit && s > 0) ? &flags[s - 1] : nullptr;
        BTAS_CUDA(launch_transpose4(cur, n, (int)n, (int)n, T, ldt, 0, skip, st), "transpose");
        GemmArgs a{};
        a.m = a.n = a.k = (int)n;
        a.A = cur; a.lda = n;
        a.Bt = T; a.ldb = ldt;
        a.C = out; a.ldc = n;
        a.prev = cur; a.ldp = n;
        a.changed = &flags[s];
        a.skip = skip;
        a.vec_a = aligned16(cur, n);
        a.vec_b = aligned16(T, ldt);
        btas_status r = run_nt(dtype, kMin, a, st);
        if (r != BTAS_OK) return r;
        cur = out;
    }
    return BTAS_OK;
}

// The cooperative mid-size solve (mid.cu).  Returns a btas_status, or
// kMidFallback if the grid cannot be co-resident on this device (e.g. a
// shared device); the tiled path then computes the same result.
constexpr int kMidFallback = -1;
constexpr int kMidDense = -2;  // the graph is too dense for the cooperative kernel's edge lists: tiled path

// Per host thread, for the one-block and cooperative solves: a host-mapped
// mailbox that the kernel leaves its status words in (no device-to-host copy
// after the kernel), and, for cooperative workspaces up to 32 MiB on the
// first device used, one cached workspace (no pool allocation and release
// per call).  Both are
// idle between calls: a call synchronises its stream before it returns.
// Measured on GB300 (p = 0.1, w in [1, 100]): 66.3 -> 61.7 us per call at
// n = 256, 103 -> 96 us at n = 512.
struct MidThreadState {
    int *mbox = nullptr;  // host pointer; the device writes it through UVA
    bool mbox_tried = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int ws_dev = -1;
    ~MidThreadState() {
        if (mbox) cudaFreeHost(mbox);
        if (ws) cudaFree(ws);
    }
};
constexpr size_t kMidCachedWs = size_t(32) << 20;

static MidThreadState &thread_state() {
    thread_local MidThreadState ts;
    if (!ts.mbox_tried) {
        ts.mbox_tried = true;
        void *p = nullptr;
        if (cudaHostAlloc(&p, 64, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
            void *d = nullptr;
            if (cudaHostGetDevicePointer(&d, p, 0) == cudaSuccess && d == p) ts.mbox = static_cast<int *>(p);
            else cudaFreeHost(p);
        }
        cudaGetLastError();
    }
    return ts;
}

static int apsp_mid_solve(int64_t n, const int32_t *W, int32_t *D, int S, bool early, bool packed_ok,
                          int *squarings_done, int64_t *bound_out, int *path_out, cudaStream_t st) {
    MidThreadState &ts = thread_state();
    int dev = 0;
    BTAS_CUDA(cudaGetDevice(&dev), "device");
    const size_t need = apsp_mid_workspace(n, S);
    Workspace ws(st);
    void *wsp = nullptr;
    if (need <= kMidCachedWs && (ts.ws_dev < 0 || ts.ws_dev == dev)) {
        if (ts.ws_bytes < need) {
            if (ts.ws) cudaFree(ts.ws);
            ts.ws = nullptr;
            ts.ws_bytes = 0;
            BTAS_CUDA(cudaMalloc(&ts.ws, kMidCachedWs), "workspace alloc");
            ts.ws_bytes = kMidCachedWs;
            ts.ws_dev = dev;
        }
        wsp = ts.ws;
    } else {
        BTAS_CUDA(ws.alloc(need), "workspace alloc");
        wsp = ws.p;
    }
    // the status words inside the workspace: zeroed by the launch
    int *info = apsp_mid_info(wsp, n);
    if (ts.mbox) ts.mbox[3] = -1;  // overwritten by the kernel as it ends
    const bool bail = n > apsp_mid_max_n();  // above it only graphs that fit the edge lists stay here
    const cudaError_t le =
        launch_apsp_mid(W, n, (int)n, S, early, packed_ok, D, n, wsp, need, nullptr, st, ts.mbox, bail);
    if (le == cudaErrorCooperativeLaunchTooLarge || le == cudaErrorNotSupported) {
        cudaGetLastError();
        return kMidFallback;
    }
    BTAS_CUDA(le, "mid apsp");
    int host[5] = {0, 0, 0, 0, 0};
    if (ts.mbox) {
        BTAS_CUDA(cudaStreamSynchronize(st), "mid apsp");
        memcpy(host, ts.mbox, sizeof host);
        if (host[3] == -1)
            return fail((btas_status)BTAS_ERR_INTERNAL, "btas_apsp: the cooperative kernel left no status");
    } else {
        BTAS_CUDA(read_back(host, info, 20, st), "info readback");
    }
    if (host[3] != 0) return fail(BTAS_ERR_TIMEOUT, "btas_apsp: a bounded grid barrier wait expired");
    if (host[0] != 0) {
        if (bound_out) *bound_out = -1;
        return fail(BTAS_ERR_ARG,
                    "btas_apsp: %d entries outside the domain (negative weight, weight > 2^28, or non-zero "
                    "diagonal)",
                    host[0]);
    }
    if (host[4] == kMidDeclined) {
        log_event("apsp n=%lld: too dense for the cooperative kernel's edge lists", (long long)n);
        return kMidDense;
    }
    if (bound_out) *bound_out = (long long)(n - 1) * host[1];
    if (squarings_done) *squarings_done = host[2];
    if (path_out) *path_out = host[4];
    log_event("apsp n=%lld: cooperative kernel, representations 0x%x, %d changing squarings", (long long)n, host[4],
              host[2]);
    return BTAS_OK;
}

static btas_status apsp_impl(int64_t n, const int32_t *W, int32_t *D, int flags, int *squarings_done,
                             int64_t *bound_out, int *path_out, cudaStream_t st) {
    Trace trace_("btas_apsp");
    if (n < 0) return fail(BTAS_ERR_ARG, "btas_apsp: negative n");
    if (n > 46340) return fail(BTAS_ERR_ARG, "btas_apsp: n too large");
    if (n == 0) {
        if (squarings_done) *squarings_done = 0;
        if (bound_out) *bound_out = 0;
        if (path_out) *path_out = 0;
        return BTAS_OK;
    }
    if (!W || !D) return fail(BTAS_ERR_ARG, "btas_apsp: NULL pointer");
    const int known = BTAS_APSP_EARLY_EXIT | BTAS_APSP_FORCE_I32 | BTAS_APSP_FORCE_U16 | BTAS_APSP_FORCE_CARRIER;
    if (flags & ~known) return fail(BTAS_ERR_ARG, "btas_apsp: unknown flags 0x%x", flags);
    const int forced = (flags & BTAS_APSP_FORCE_I32 ? 1 : 0) + (flags & BTAS_APSP_FORCE_U16 ? 1 : 0) +
                       (flags & BTAS_APSP_FORCE_CARRIER ? 1 : 0);
    if (forced > 1) return fail(BTAS_ERR_ARG, "btas_apsp: more than one FORCE flag");
    const int S = btas_apsp_squarings(n);
    const bool early = (flags & BTAS_APSP_EARLY_EXIT) != 0;
    const size_t nn = (size_t)n * (size_t)n;

    // small graphs: the whole solve in one thread block (one launch, one
    // read-back) on the int32 arithmetic; BTAS_APSP_NO_SMALL=1 disables it
    if (S >= 1 && n <= apsp_small_limit() && !(flags & (BTAS_APSP_FORCE_U16 | BTAS_APSP_FORCE_CARRIER)) &&
        env_int("BTAS_APSP_NO_SMALL", 0) == 0) {
        // the status words straight into the thread's host-mapped mailbox
        // (the kernel writes them once, from one thread, as it ends), else
        // into workspace read back
        MidThreadState &ts = thread_state();
        Workspace ws(st);
        int *info = ts.mbox;
        if (!info) {
            BTAS_CUDA(ws.alloc(256), "workspace alloc");
            info = static_cast<int *>(ws.p);
        }
        int host[3] = {0, 0, 0};
        if (ts.mbox) ts.mbox[2] = -1;  // overwritten by the kernel as it ends
        BTAS_CUDA(launch_apsp_small(W, n, (int)n, S, early, D, n, info, st), "small apsp");
        if (ts.mbox) {
            BTAS_CUDA(cudaStreamSynchronize(st), "small apsp");
            memcpy(host, ts.mbox, sizeof host);
            if (host[2] == -1)
                return fail((btas_status)BTAS_ERR_INTERNAL, "btas_apsp: the one-block kernel left no status");
        } else {
            BTAS_CUDA(read_back(host, info, 12, st), "info readback");
        }
        if (host[0] != 0) {
            if (bound_out) *bound_out = -1;
            return fail(BTAS_ERR_ARG,
                        "btas_apsp: %d entries outside the domain (negative weight, weight > 2^28, or non-zero "
                        "diagonal)",
                        host[0]);
        }
        if (bound_out) *bound_out = (long long)(n - 1) * host[1];
        if (squarings_done) *squarings_done = host[2];
        if (path_out) *path_out = 1;
        log_event("apsp n=%lld: one-block kernel, int32, %d changing squarings", (long long)n, host[2]);
        return BTAS_OK;
    }

    // mid-size graphs: every squaring in one cooperative launch (one
    // read-back); BTAS_APSP_NO_MID=1 disables it
    DeviceInfo dinfo{};
    const int dev_sms = current_device_info(&dinfo) ? dinfo.sms : 0;
    if (S >= 1 && n > apsp_small_limit() && apsp_mid_takes(n, dev_sms) &&
        !(flags & (BTAS_APSP_FORCE_U16 | BTAS_APSP_FORCE_CARRIER)) && env_int("BTAS_APSP_NO_MID", 0) == 0) {
        const int r = apsp_mid_solve(n, W, D, S, early, !(flags & BTAS_APSP_FORCE_I32), squarings_done, bound_out,
                                     path_out, st);
        if (r != kMidFallback && r != kMidDense) return static_cast<btas_status>(r);
        if (r == kMidFallback) log_event("apsp n=%lld: cooperative launch not possible here, tiled path", (long long)n);
    }

    Workspace ws(st);
    // flags: [0, S) change flags of the device-exit path, [S+1, S+2] the domain
    // scan, [2S+8, 4S+8) (change flag, largest finite entry) of each squaring
    // of the adaptive path, adjacent so that one read-back fetches both
    const size_t flag_bytes = align256((size_t)(4 * S + 8) * 4);
    // layout: [flags | X | Y | T]; T holds a transpose (or the duplicated
    // 16-bit operand) with a leading dimension rounded up to 4 elements
    const long long ldt = (n + 3) & ~3LL;
    const size_t t_bytes = align256((size_t)n * (size_t)ldt * 4);
    BTAS_CUDA(ws.alloc(flag_bytes + 2 * align256(nn * 4) + t_bytes), "workspace alloc");
    char *base = static_cast<char *>(ws.p);
    int *dflags = reinterpret_cast<int *>(base);
    char *X = base + flag_bytes;
    char *Y = X + align256(nn * 4);
    char *T = Y + align256(nn * 4);
    BTAS_CUDA(cudaMemsetAsync(dflags, 0, flag_bytes, st), "memset");

    // domain scan and bound: (n-1) * max finite weight
    long long bound = -1;
    const bool need_scan = !(flags & BTAS_APSP_FORCE_I32) || bound_out != nullptr;
    if (need_scan) {
        int host[2] = {0, 0};
        int *scan = dflags + S + 1;
        BTAS_CUDA(launch_apsp_scan(W, n, scan, st), "domain scan");
        BTAS_CUDA(read_back(host, scan, 8, st), "scan readback");
        if (host[1] != 0) {
            if (bound_out) *bound_out = -1;
            return fail(BTAS_ERR_ARG,
                        "btas_apsp: %d entries outside the domain (negative weight, weight > 2^28, or non-zero "
                        "diagonal)",
                        host[1]);
        }
        bound = (long long)(n - 1) * host[0];
        if (bound_out) *bound_out = bound;
    }
    if (S == 0) {
        if (D != W) BTAS_CUDA(cudaMemcpyAsync(D, W, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
        if (squarings_done) *squarings_done = 0;
        if (path_out) *path_out = 0;
        return BTAS_OK;
    }

    if ((flags & BTAS_APSP_FORCE_I32) && !need_scan) {
        // int32 only, no host synchronisation: the early exit is decided on
        // the device (a converged squaring copies its input through)
        const void *cur0 = W;
        if ((const void *)W == (const void *)D && ((S - 1) & 1) == 0) {
            // the first squaring would write D == W while reading it
            BTAS_CUDA(cudaMemcpyAsync(Y, W, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
            cur0 = Y;
        }
        void *bufs[2] = {D, X};
        btas_status r = squaring_loop(BTAS_I32, n, S, cur0, bufs, T, dflags, early, st);
        if (r != BTAS_OK) return r;
        if (path_out) *path_out = 1;
        if (squarings_done) {
            int host[64];
            BTAS_CUDA(read_back(host, dflags, (size_t)S * 4, st), "flags readback");
            int done = 0;
            for (int q = 0; q < S; ++q) done += host[q] != 0;
            *squarings_done = done;
        }
        return BTAS_OK;
    }

    // Representation per squaring: 0 = int32, 1 = exact fp32 carrier, 2 =
    // packed u16x2.  With m the largest finite entry of D_s, every finite
    // entry of D_{s+1} = D_s (x) D_s is at most 2m, and so is every pairwise
    // sum.  Hence 2m < 0x7FFF makes the 16-bit squaring exact, and 2m < 2^24
    // makes the fp32 one exact (all values and sums are exact integers).  The
    // squaring's epilogue reports the next m.  FORCE flags pin one
    // representation and require the static bound (n-1) * max w instead.
    int force_rep = -1;
    if (flags & BTAS_APSP_FORCE_U16) {
        if (bound >= BTAS_INF_U16) return fail(BTAS_ERR_BOUND, "btas_apsp: bound %lld >= 0x7FFF", bound);
        force_rep = 2;
    } else if (flags & BTAS_APSP_FORCE_CARRIER) {
        if (bound >= (1LL << 23)) return fail(BTAS_ERR_BOUND, "btas_apsp: bound %lld >= 2^23", bound);
        force_rep = 1;
    } else if (flags & BTAS_APSP_FORCE_I32) {
        force_rep = 0;
    }
    const bool no_u16 = env_int("BTAS_APSP_NO_U16", 0) != 0;
    const bool no_carrier = env_int("BTAS_APSP_NO_CARRIER", 0) != 0;
    int *pairs = dflags + 2 * S + 8;  // squaring s: pairs[2s] changed, pairs[2s + 1] largest finite entry
    int ns16 = -1;                    // looked up at the first packed squaring
    auto other = [&](const void *p) -> void * { return p == (const void *)X ? (void *)Y : (void *)X; };
    // convert an n x n matrix between representations (T is free scratch here)
    auto convert = [&](int from, int to, const void *src, void *dst) -> cudaError_t {
        if (from == to) return cudaSuccess;
        const void *s32 = src;
        cudaError_t e = cudaSuccess;
        if (from == 1) e = launch_convert4(src, n, (int)n, (int)n, (to == 0 ? dst : T), n, 2, st);
        if (from == 2) e = launch_widen_u16_i32(static_cast<const uint16_t *>(src), (long long)nn,
                                                static_cast<int *>(to == 0 ? dst : (void *)T), st);
        if (e != cudaSuccess || to == 0) return e;
        if (from != 0) s32 = T;
        if (to == 1) return launch_convert4(s32, n, (int)n, (int)n, dst, n, 1, st);
        return launch_narrow_u16(static_cast<const int *>(s32), (long long)nn, static_cast<uint16_t *>(dst), st);
    };

    int rep = 0, used = 0, done = 0;
    long long m = bound >= 0 ? (n > 1 ? bound / (n - 1) : 0) : 0;
    const void *cur = W;
    for (int s = 0; s < S; ++s) {
        int want = force_rep;
        if (want < 0) want = (2 * m < BTAS_INF_U16 && !no_u16) ? 2 : (2 * m < (1LL << 24) && !no_carrier) ? 1 : 0;
        if (want != rep) {
            void *dst = other(cur);
            BTAS_CUDA(convert(rep, want, cur, dst), "representation change");
            cur = dst;
            rep = want;
        }
        void *out = other(cur);
        if (rep == 2) {
            U16Args a{};
            a.m = a.n = a.k = (int)n;
            a.A = static_cast<const uint16_t *>(cur); a.lda = n;
            a.B = static_cast<const uint16_t *>(cur); a.ldb = n;
            a.C = static_cast<uint16_t *>(out); a.ldc = n;
            a.prev = static_cast<const uint16_t *>(cur); a.ldp = n;
            a.changed = &pairs[2 * s];
            a.one = 1;
            a.maxfin = &pairs[2 * s + 1];
            if (ns16 < 0) ns16 = u16_ns(n, n, n, st);
            BTAS_CUDA(launch_tgemm_u16_ws(a, reinterpret_cast<uint32_t *>(T), ns16, st), "u16 squaring");
        } else {
            const long long ldt = (n + 3) & ~3LL;
            BTAS_CUDA(launch_transpose4(cur, n, (int)n, (int)n, T, ldt, 0, nullptr, st), "transpose");
            GemmArgs a{};
            a.m = a.n = a.k = (int)n;
            a.A = cur; a.lda = n;
            a.Bt = T; a.ldb = ldt;
            a.C = out; a.ldc = n;
            a.prev = cur; a.ldp = n;
            a.changed = &pairs[2 * s];
            a.maxfin = &pairs[2 * s + 1];
            a.vec_a = aligned16(cur, n);
            a.vec_b = aligned16(T, ldt);
            btas_status r = run_nt(rep == 1 ? BTAS_F32 : BTAS_I32, kMin, a, st);
            if (r != BTAS_OK) return r;
        }
        used |= 1 << rep;
        int host[2] = {0, 0};  // one read-back through the pinned mailbox: change flag and maximum
        BTAS_CUDA(read_back(host, &pairs[2 * s], 8, st), "flag readback");
        cur = out;
        m = host[1] < 0 ? 0 : host[1];
        if (host[0]) ++done;
        if (early && !host[0]) break;
    }
    if (rep == 0) {
        if (cur != (const void *)D) BTAS_CUDA(cudaMemcpyAsync(D, cur, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
    } else {
        BTAS_CUDA(convert(rep, 0, cur, D), "final conversion");
    }
    if (squarings_done) *squarings_done = done;
    if (path_out) *path_out = used;
    log_event("apsp n=%lld: tiled kernels, representations %s%s%s, %d changing squarings", (long long)n,
              used & 1 ? "int32 " : "", used & 2 ? "fp32-carrier " : "", used & 4 ? "u16x2" : "", done);
    return BTAS_OK;
}

btas_status btas_closure(int semiring, int dtype, int64_t n, const void *A, void *Astar, int flags,
                         int *squarings_done, void *stream) {
    Trace trace_("btas_closure");
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) return fail(BTAS_ERR_ARG, "btas_closure: semiring");
    if (dtype != BTAS_I32 && dtype != BTAS_F32) return fail(BTAS_ERR_ARG, "btas_closure: dtype");
    if (n < 0 || n > 46340) return fail(BTAS_ERR_ARG, "btas_closure: n out of range");
    if (flags & ~BTAS_APSP_EARLY_EXIT) return fail(BTAS_ERR_ARG, "btas_closure: unknown flags");
    if (n == 0) {
        if (squarings_done) *squarings_done = 0;
        return BTAS_OK;
    }
    if (!A || !Astar) return fail(BTAS_ERR_ARG, "btas_closure: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a squaring that changes nothing is a fixpoint, so stopping there (the
    // early exit) never changes the result; the flag is accepted either way
    const int S = btas_apsp_squarings(n);
    const size_t nn = (size_t)n * (size_t)n;
    const long long ldt = (n + 3) & ~3LL;
    Workspace ws(st);
    const size_t flag_bytes = align256((size_t)(S + 4) * 4);
    BTAS_CUDA(ws.alloc(flag_bytes + 2 * align256(nn * 4) + align256((size_t)n * ldt * 4)), "workspace alloc");
    char *base = static_cast<char *>(ws.p);
    int *dflags = reinterpret_cast<int *>(base);
    void *X = base + flag_bytes;
    void *Y = static_cast<char *>(X) + align256(nn * 4);
    void *T = static_cast<char *>(Y) + align256(nn * 4);
    BTAS_CUDA(cudaMemsetAsync(dflags, 0, flag_bytes, st), "memset");
    BTAS_CUDA(launch_ident_oplus(A, n, (int)n, X, n, semiring, dtype == BTAS_F32, st), "E (+) A");
    // Square E (+) A: S = ceil(log2(n-1)) squarings reach every walk of
    // <= n-1 edges, which is A* when no cycle improves a walk; a squaring
    // that changes nothing is a fixpoint and ends the loop early.  If all S
    // squarings changed the matrix, one more squaring covers walks of
    // >= n edges: a negative (min-plus) / positive (max-plus) diagonal entry
    // there proves such a cycle, and A* does not exist.  The result is D_S.
    void *cur = X;
    int done = 0;
    bool converged = false;
    auto square = [&](const void *in, void *out, int *flag) -> btas_status {
        BTAS_CUDA(launch_transpose4(in, n, (int)n, (int)n, T, ldt, 0, nullptr, st), "transpose");
        GemmArgs a{};
        a.m = a.n = a.k = (int)n;
        a.A = in; a.lda = n;
        a.Bt = T; a.ldb = ldt;
        a.C = out; a.ldc = n;
        a.prev = in; a.ldp = n;
        a.changed = flag;
        a.vec_a = aligned16(in, n);
        a.vec_b = aligned16(T, ldt);
        return run_nt(dtype, semiring, a, st);
    };
    for (int s = 0; s < S; ++s) {
        void *out = cur == X ? Y : X;
        btas_status r = square(cur, out, &dflags[s]);
        if (r != BTAS_OK) return r;
        int changed = 1;
        BTAS_CUDA(read_back(&changed, &dflags[s], 4, st), "flag readback");
        if (!changed) {
            converged = true;
            break;
        }
        cur = out;
        ++done;
    }
    if (!converged) {
        void *chk = cur == X ? Y : X;
        btas_status r = square(cur, chk, &dflags[S]);
        if (r != BTAS_OK) return r;
        std::vector<uint32_t> diag((size_t)n);
        BTAS_CUDA(cudaMemcpy2DAsync(diag.data(), 4, chk, (size_t)(n + 1) * 4, 4, (size_t)n, cudaMemcpyDeviceToHost, st),
                  "diagonal readback");
        BTAS_CUDA(cudaStreamSynchronize(st), "check sync");
        bool cycle = false;
        for (uint32_t v : diag) {
            if (dtype == BTAS_F32) {
                float f;
                memcpy(&f, &v, 4);
                cycle |= semiring == BTAS_MINPLUS ? f < 0.f : f > 0.f;
            } else {
                const int x = static_cast<int>(v);
                cycle |= semiring == BTAS_MINPLUS ? x < 0 : x > 0;
            }
        }
        if (cycle)
            return fail(BTAS_ERR_ARG, semiring == BTAS_MINPLUS ? "btas_closure: negative cycle, A* does not exist"
                                                               : "btas_closure: positive cycle, A* does not exist");
    }
    BTAS_CUDA(cudaMemcpyAsync(Astar, cur, nn * 4, cudaMemcpyDeviceToDevice, st), "copy out");
    if (squarings_done) *squarings_done = done;
    return BTAS_OK;
}

btas_status btas_apsp_paths(int64_t n, const int32_t *W, int32_t *D, int32_t *Next, int flags, int *squarings_done,
                            void *stream) {
    Trace trace_("btas_apsp_paths");
    if (n < 0 || n > 46340) return fail(BTAS_ERR_ARG, "btas_apsp_paths: n out of range");
    if (flags & ~BTAS_APSP_EARLY_EXIT) return fail(BTAS_ERR_ARG, "btas_apsp_paths: unknown flags");
    if (n == 0) {
        if (squarings_done) *squarings_done = 0;
        return BTAS_OK;
    }
    if (!W || !D || !Next) return fail(BTAS_ERR_ARG, "btas_apsp_paths: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int S = btas_apsp_squarings(n);
    const size_t nn = (size_t)n * (size_t)n;
    const long long ldt = (n + 3) & ~3LL;
    // Keyed squarings (one int32 min-plus product carries distance and
    // smallest minimising k, see paths.cu) while the entries allow it;
    // BTAS_PATHS_NO_KEYED=1 keeps every squaring on the argmin kernel.
    const bool keyed_ok = n <= paths_key_max_n() && env_int("BTAS_PATHS_NO_KEYED", 0) == 0;
    Workspace ws(st);
    const size_t flag_bytes = align256((size_t)(2 * S + 4) * 4);
    const size_t ak_bytes = keyed_ok ? align256(nn * 4) : 0;
    BTAS_CUDA(ws.alloc(flag_bytes + 4 * align256(nn * 4) + align256((size_t)n * ldt * 4) + ak_bytes),
              "workspace alloc");
    char *base = static_cast<char *>(ws.p);
    int *dflags = reinterpret_cast<int *>(base);  // [2s] changed, [2s + 1] largest finite entry after squaring s
    int *Db[2], *Nb[2];
    Db[0] = reinterpret_cast<int *>(base + flag_bytes);
    Db[1] = reinterpret_cast<int *>(reinterpret_cast<char *>(Db[0]) + align256(nn * 4));
    Nb[0] = reinterpret_cast<int *>(reinterpret_cast<char *>(Db[1]) + align256(nn * 4));
    Nb[1] = reinterpret_cast<int *>(reinterpret_cast<char *>(Nb[0]) + align256(nn * 4));
    int *T = reinterpret_cast<int *>(reinterpret_cast<char *>(Nb[1]) + align256(nn * 4));
    int *Ak = keyed_ok ? reinterpret_cast<int *>(reinterpret_cast<char *>(T) + align256((size_t)n * ldt * 4)) : nullptr;
    BTAS_CUDA(cudaMemsetAsync(dflags, 0, flag_bytes, st), "memset");
    // domain: zero diagonal, weights in [0, 2^28] or INF
    long long mval = 0;  // bound on the finite entries of the current D
    {
        int host[2] = {0, 0};
        BTAS_CUDA(launch_apsp_scan(W, n, dflags + 2 * S + 1, st), "domain scan");
        BTAS_CUDA(read_back(host, dflags + 2 * S + 1, 8, st), "scan readback");
        if (host[1] != 0) return fail(BTAS_ERR_ARG, "btas_apsp_paths: %d entries outside the domain", host[1]);
        mval = host[0];
    }
    BTAS_CUDA(cudaMemcpyAsync(Db[0], W, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
    BTAS_CUDA(launch_next_init(W, n, Nb[0], st), "next-hop init");
    int cur = 0, done = 0, keyed_count = 0;
    for (int s = 0; s < S; ++s) {
        const bool keyed = keyed_ok && mval <= paths_key_max();
        if (keyed) {
            // keys in Db[cur ^ 1], decoded there in place
            BTAS_CUDA(launch_paths_encode(Db[cur], (int)n, Ak, T, ldt, st), "key encode");
            GemmArgs a{};
            a.m = a.n = a.k = (int)n;
            a.A = Ak; a.lda = n;
            a.Bt = T; a.ldb = ldt;
            a.C = Db[cur ^ 1]; a.ldc = n;
            a.vec_a = aligned16(Ak, n);
            a.vec_b = aligned16(T, ldt);
            btas_status r = run_nt(BTAS_I32, kMin, a, st);
            if (r != BTAS_OK) return r;
            BTAS_CUDA(launch_paths_decode(Db[cur ^ 1], Db[cur], Nb[cur], n, Db[cur ^ 1], Nb[cur ^ 1], &dflags[2 * s],
                                          &dflags[2 * s + 1], st),
                      "key decode");
            ++keyed_count;
        } else {
            BTAS_CUDA(launch_transpose4(Db[cur], n, (int)n, (int)n, T, ldt, 0, nullptr, st), "transpose");
            BTAS_CUDA(launch_paths_square((int)n, Db[cur], n, T, ldt, Nb[cur], Db[cur ^ 1], Nb[cur ^ 1],
                                          &dflags[2 * s], st),
                      "paths squaring");
        }
        cur ^= 1;
        int host[2] = {1, 0};
        BTAS_CUDA(read_back(host, &dflags[2 * s], 8, st), "flag readback");
        // every finite entry of the new D is a sum of two of the old
        mval = keyed ? host[1] : 2 * mval;
        if (host[0]) ++done;
        if (!host[0] && (flags & BTAS_APSP_EARLY_EXIT)) break;
    }
    log_event("apsp paths n=%lld: %d of the squarings keyed (one int32 product each)", (long long)n, keyed_count);
    BTAS_CUDA(cudaMemcpyAsync(D, Db[cur], nn * 4, cudaMemcpyDeviceToDevice, st), "copy D");
    BTAS_CUDA(cudaMemcpyAsync(Next, Nb[cur], nn * 4, cudaMemcpyDeviceToDevice, st), "copy Next");
    if (squarings_done) *squarings_done = done;
    return BTAS_OK;
}

btas_status btas_apsp_paths_f32(int64_t n, const float *W, float *D, int32_t *Next, int flags, int *squarings_done,
                                void *stream) {
    Trace trace_("btas_apsp_paths_f32");
    if (n < 0 || n > 46340) return fail(BTAS_ERR_ARG, "btas_apsp_paths_f32: n out of range");
    if (flags & ~BTAS_APSP_EARLY_EXIT) return fail(BTAS_ERR_ARG, "btas_apsp_paths_f32: unknown flags");
    if (n == 0) {
        if (squarings_done) *squarings_done = 0;
        return BTAS_OK;
    }
    if (!W || !D || !Next) return fail(BTAS_ERR_ARG, "btas_apsp_paths_f32: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int S = btas_apsp_squarings(n);
    const size_t nn = (size_t)n * (size_t)n;
    const long long ldt = (n + 3) & ~3LL;
    Workspace ws(st);
    const size_t flag_bytes = align256((size_t)(S + 4) * 4);
    BTAS_CUDA(ws.alloc(flag_bytes + 4 * align256(nn * 4) + align256((size_t)n * ldt * 4)), "workspace alloc");
    char *base = static_cast<char *>(ws.p);
    int *dflags = reinterpret_cast<int *>(base);  // [s] changed after squaring s, [S] domain count
    float *Db[2];
    int *Nb[2];
    Db[0] = reinterpret_cast<float *>(base + flag_bytes);
    Db[1] = reinterpret_cast<float *>(reinterpret_cast<char *>(Db[0]) + align256(nn * 4));
    Nb[0] = reinterpret_cast<int *>(reinterpret_cast<char *>(Db[1]) + align256(nn * 4));
    Nb[1] = reinterpret_cast<int *>(reinterpret_cast<char *>(Nb[0]) + align256(nn * 4));
    float *T = reinterpret_cast<float *>(reinterpret_cast<char *>(Nb[1]) + align256(nn * 4));
    BTAS_CUDA(cudaMemsetAsync(dflags, 0, flag_bytes, st), "memset");
    {
        int bad = 0;
        BTAS_CUDA(launch_paths_scan_f32(W, n, dflags + S, st), "domain scan");
        BTAS_CUDA(read_back(&bad, dflags + S, 4, st), "scan readback");
        if (bad != 0)
            return fail(BTAS_ERR_ARG,
                        "btas_apsp_paths_f32: %d entries outside the domain (NaN, negative, or non-zero diagonal)",
                        bad);
    }
    BTAS_CUDA(cudaMemcpyAsync(Db[0], W, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
    BTAS_CUDA(launch_next_init_f32(W, n, Nb[0], st), "next-hop init");
    int cur = 0, done = 0;
    for (int s = 0; s < S; ++s) {
        BTAS_CUDA(launch_transpose4(Db[cur], n, (int)n, (int)n, T, ldt, 0, nullptr, st), "transpose");
        BTAS_CUDA(launch_paths_square_f32((int)n, Db[cur], n, T, ldt, Nb[cur], Db[cur ^ 1], Nb[cur ^ 1], &dflags[s],
                                          st),
                  "paths squaring");
        cur ^= 1;
        int changed = 1;
        BTAS_CUDA(read_back(&changed, &dflags[s], 4, st), "flag readback");
        if (changed) ++done;
        if (!changed && (flags & BTAS_APSP_EARLY_EXIT)) break;
    }
    log_event("apsp paths f32 n=%lld: %d changing squarings on the argmin kernel", (long long)n, done);
    BTAS_CUDA(cudaMemcpyAsync(D, Db[cur], nn * 4, cudaMemcpyDeviceToDevice, st), "copy D");
    BTAS_CUDA(cudaMemcpyAsync(Next, Nb[cur], nn * 4, cudaMemcpyDeviceToDevice, st), "copy Next");
    if (squarings_done) *squarings_done = done;
    return BTAS_OK;
}

btas_status btas_apsp_fw(int64_t n, const int32_t *W, int32_t *D, void *stream) {
    Trace trace_("btas_apsp_fw");
    if (n < 0 || n > 46340) return fail(BTAS_ERR_ARG, "btas_apsp_fw: n out of range");
    if (n == 0) return BTAS_OK;
    if (!W || !D) return fail(BTAS_ERR_ARG, "btas_apsp_fw: NULL pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = fw_block();
    const size_t nn = (size_t)n * (size_t)n;
    const int nb = (int)((n + B - 1) / B);
    // Phase 3 runs on the exact packed u16x2 kernel for every pivot block
    // whose row and column panels (after phase 2) have all finite entries
    // below 0x7FFF / 2 -- decided on the device; BTAS_FW_NO_U16=1 keeps it
    // on the int32 kernel.
    const bool allow16 = nb > 1 && env_int("BTAS_FW_NO_U16", 0) == 0;
    const long long ldbu = (n + 7) & ~7LL;
    const size_t s_rpt = align256((size_t)n * B * 4), s_pmax = align256((size_t)nb * 4);
    const size_t s_ad = allow16 ? align256((size_t)n * B * 4) : 0, s_bu = allow16 ? align256((size_t)B * ldbu * 2) : 0;
    Workspace ws(st);
    BTAS_CUDA(ws.alloc(256 + s_rpt + s_pmax + 256 + s_ad + s_bu), "workspace alloc");
    char *wbase = static_cast<char *>(ws.p);
    int *scan = reinterpret_cast<int *>(wbase);
    int *RPT = reinterpret_cast<int *>(wbase + 256);
    int *pmax = reinterpret_cast<int *>(wbase + 256 + s_rpt);
    int *state = reinterpret_cast<int *>(wbase + 256 + s_rpt + s_pmax);
    uint32_t *Ad = reinterpret_cast<uint32_t *>(wbase + 256 + s_rpt + s_pmax + 256);
    uint16_t *Bu = reinterpret_cast<uint16_t *>(wbase + 256 + s_rpt + s_pmax + 256 + s_ad);
    {
        int host[2] = {0, 0};
        BTAS_CUDA(cudaMemsetAsync(scan, 0, 8, st), "memset");
        BTAS_CUDA(launch_apsp_scan(W, n, scan, st), "domain scan");
        BTAS_CUDA(read_back(host, scan, 8, st), "scan readback");
        if (host[1] != 0) return fail(BTAS_ERR_ARG, "btas_apsp_fw: %d entries outside the domain", host[1]);
    }
    if (D != W) BTAS_CUDA(cudaMemcpyAsync(D, W, nn * 4, cudaMemcpyDeviceToDevice, st), "copy");
    BTAS_CUDA(cudaMemsetAsync(pmax, 0xFF, (size_t)nb * 4, st), "memset");  // -1: nothing finite yet
    // Lookahead: phases 1-2 of pivot block kb + 1, preceded by pivot block
    // kb's phase-3 terms on block row and column kb + 1, run on a second
    // stream of higher priority while the rest of phase 3 of kb -- which
    // leaves block row and column kb + 1 alone -- runs on `st`.  The serial
    // phases then hide behind the product.  BTAS_FW_NO_LOOKAHEAD=1 runs the
    // three phases one after another on `st`.
    const bool ahead = nb > 2 && env_int("BTAS_FW_NO_LOOKAHEAD", 0) == 0;
    struct Side {
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        ~Side() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
            if (s) cudaStreamDestroy(s);
        }
    } side;
    if (ahead) {
        int least = 0, greatest = 0;
        BTAS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        BTAS_CUDA(cudaStreamCreateWithPriority(&side.s, cudaStreamNonBlocking, greatest), "side stream");
        BTAS_CUDA(cudaEventCreateWithFlags(&side.a, cudaEventDisableTiming), "event");
        BTAS_CUDA(cudaEventCreateWithFlags(&side.b, cudaEventDisableTiming), "event");
    }
    BTAS_CUDA(launch_fw_phase12(D, n, 0, allow16 ? pmax : nullptr, st), "phases 1-2");
    for (int kb = 0; nb > 1 && kb < nb; ++kb) {
        const long long o = (long long)kb * B, bw = std::min<long long>(B, n - o);
        const bool next = kb + 1 < nb, ahead_now = ahead && next;
        const long long o1 = o + bw;  // next pivot block
        const long long bw1 = ahead_now ? std::min<long long>(B, n - o1) : 0;  // its width, if it runs ahead
        if (allow16) {
            // Ad pitch round4(bw): the pitch the packed kernel reads a pre-duplicated A with
            BTAS_CUDA(launch_fw_pack(D, n, kb, pmax + kb, state, Ad, (bw + 3) & ~3LL, Bu, ldbu, st), "packed panels");
        }
        if (ahead_now) {
            BTAS_CUDA(cudaEventRecord(side.a, st), "event");
            BTAS_CUDA(cudaStreamWaitEvent(side.s, side.a, 0), "event wait");
            BTAS_CUDA(launch_fw_cross(D, n, kb, side.s), "lookahead update");
            BTAS_CUDA(launch_fw_phase12(D, n, kb + 1, allow16 ? pmax + kb + 1 : nullptr, side.s), "phases 1-2");
            BTAS_CUDA(cudaEventRecord(side.b, side.s), "event");
        }
        if (allow16) {
            U16Args a{};
            a.m = (int)n; a.n = (int)n; a.k = (int)bw;
            a.B = Bu; a.ldb = ldbu;
            a.one = 1;
            a.gate = state;
            a.adup_ready = true;
            a.Ci = D; a.ldci = n;
            a.xr0 = a.xc0 = (int)o1;  // block row and column kb + 1 belong to the other stream
            a.xr1 = a.xc1 = (int)(o1 + bw1);
            BTAS_CUDA(launch_tgemm_u16_ws(a, Ad, u16_ns(n, n, bw, st), st), "packed phase 3");
        }
        // row panel D[o:o+bw, :] transposed into RPT (n x B): the k-contiguous B operand
        BTAS_CUDA(launch_transpose4(D + o * n, n, (int)bw, (int)n, RPT, B, 0, allow16 ? state + 1 : nullptr, st),
                  "panel transpose");
        // int32 phase 3 on every tile outside block row and column kb (and
        // kb + 1 when it runs ahead), in one launch
        BTAS_CUDA(launch_fw_phase3_i32(D, n, o, (int)bw, RPT, kb, kb + 1 + (ahead_now ? 1 : 0),
                                       allow16 ? state : nullptr, st),
                  "phase 3");
        if (ahead_now)
            BTAS_CUDA(cudaStreamWaitEvent(st, side.b, 0), "event wait");
        else if (next)
            BTAS_CUDA(launch_fw_phase12(D, n, kb + 1, allow16 ? pmax + kb + 1 : nullptr, st), "phases 1-2");
    }
    return BTAS_OK;
}

btas_status btas_apsp(int64_t n, const int32_t *W, int32_t *D, void *stream) {
    return apsp_impl(n, W, D, BTAS_APSP_EARLY_EXIT, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

btas_status btas_apsp_ex(int64_t n, const int32_t *W, int32_t *D, int flags, int *squarings_done, int64_t *bound,
                         int *path, void *stream) {
    return apsp_impl(n, W, D, flags, squarings_done, bound, path, static_cast<cudaStream_t>(stream));
}

btas_status btas_apsp_u16(int64_t n, const uint16_t *W, uint16_t *D, int max_w, int flags, void *stream) {
    Trace trace_("btas_apsp_u16");
    if (n < 0 || n > 46340) return fail(BTAS_ERR_ARG, "btas_apsp_u16: n out of range");
    if (max_w < 0 || max_w >= BTAS_INF_U16) return fail(BTAS_ERR_ARG, "btas_apsp_u16: max_w out of range");
    if (flags & ~BTAS_APSP_EARLY_EXIT) return fail(BTAS_ERR_ARG, "btas_apsp_u16: unknown flags");
    if (n == 0) return BTAS_OK;
    if (!W || !D) return fail(BTAS_ERR_ARG, "btas_apsp_u16: NULL pointer");
    if ((long long)(n - 1) * max_w >= BTAS_INF_U16)
        return fail(BTAS_ERR_BOUND, "btas_apsp_u16: (n-1)*max_w = %lld >= 0x7FFF", (long long)(n - 1) * max_w);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int S = btas_apsp_squarings(n);
    const size_t nn = (size_t)n * (size_t)n;
    if (S == 0) {
        if (D != W) BTAS_CUDA(cudaMemcpyAsync(D, W, nn * 2, cudaMemcpyDeviceToDevice, st), "copy");
        return BTAS_OK;
    }
    Workspace ws(st);
    const size_t flag_bytes = align256((size_t)(S + 1) * 4);
    const size_t ad_bytes = align256((size_t)n * (size_t)((n + 3) & ~3LL) * 4);
    BTAS_CUDA(ws.alloc(flag_bytes + 2 * align256(nn * 2) + ad_bytes), "workspace alloc");
    int *dflags = static_cast<int *>(ws.p);
    uint16_t *U1 = reinterpret_cast<uint16_t *>(static_cast<char *>(ws.p) + flag_bytes);
    uint16_t *U2 = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(U1) + align256(nn * 2));
    uint32_t *Ad = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(U2) + align256(nn * 2));
    BTAS_CUDA(cudaMemsetAsync(dflags, 0, flag_bytes, st), "memset");
    const bool early = (flags & BTAS_APSP_EARLY_EXIT) != 0;
    const uint16_t *cur = W;
    for (int s = 0; s < S; ++s) {
        uint16_t *out = cur == U1 ? U2 : U1;
        U16Args a{};
        a.m = a.n = a.k = (int)n;
        a.A = cur; a.lda = n;
        a.B = cur; a.ldb = n;
        a.C = out; a.ldc = n;
        a.prev = cur; a.ldp = n;
        a.changed = &dflags[s];
        a.skip = (early && s > 0) ? &dflags[s - 1] : nullptr;
        a.one = 1;
        BTAS_CUDA(launch_tgemm_u16_ws(a, Ad, env_int("BTAS_U16_NS", 5), st), "u16 squaring");
        cur = out;
    }
    if (cur != D) BTAS_CUDA(cudaMemcpyAsync(D, cur, nn * 2, cudaMemcpyDeviceToDevice, st), "copy");
    return BTAS_OK;
}

}  // extern "C"
