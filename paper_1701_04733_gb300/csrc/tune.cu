// Autotuner for the tropical product kernels (btas_tune_* in btas.h).
//
// Every compiled kernel of a (semiring, dtype) computes the same product of
// Eq. 1-4 bit for bit; they differ in tile shape, CTAs per SM, fragment
// width and inner-loop instruction mix, and which is fastest depends on the
// problem shape (waves of tiles over 152 SMs, the k extent) and on the
// device.  The tuner times each candidate on seeded scratch operands, checks
// that all candidates agree bit for bit, then tries the winner with several
// tile-raster group heights, and keeps the fastest in a process-wide table
// keyed by (compute capability, SM count, semiring, dtype, ceil(log2) size
// buckets of m, n, k).  The table can be saved to and loaded from a file of
// JSON lines.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace btas {
namespace {

constexpr int kVarU16 = 16;  // btas_tune_result.variant of the packed u16x2 kernel
constexpr int kU16Ns[] = {0, 4, 5, 6, 8};
constexpr int kGroups[] = {1, 4, 16};  // raster groups tried besides the default 8

struct Key {
    int arch, sms, sr, dtype, mb, nb, kb;
    bool operator<(const Key &o) const {
        const int a[7] = {arch, sms, sr, dtype, mb, nb, kb};
        const int b[7] = {o.arch, o.sms, o.sr, o.dtype, o.mb, o.nb, o.kb};
        return std::lexicographical_compare(a, a + 7, b, b + 7);
    }
};

struct Entry {
    int var, ns, cfg, group_m, candidates, tile_m, tile_n;
    double seconds, tps;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
std::once_flag g_env_once;

int bucket(long long x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

bool device_key(int *arch, int *sms) {
    DeviceInfo d{};
    if (!current_device_info(&d)) return false;
    *arch = d.arch;
    *sms = d.sms;
    return true;
}

bool make_key(int sr, int dtype, long long m, long long n, long long k, Key *key) {
    int arch = 0, sms = 0;
    if (!device_key(&arch, &sms)) return false;
    *key = Key{arch, sms, sr, dtype, bucket(m), bucket(n), bucket(k)};
    return true;
}

// ---------------------------------------------------------------- file I/O

#define BTAS_TUNE_LINE(F)                                                                                     \
    "{\"arch\": %d, \"sms\": %d, \"semiring\": %d, \"dtype\": %d, \"m_bucket\": %d, \"n_bucket\": %d, "         \
    "\"k_bucket\": %d, \"variant\": %d, \"ns\": %d, \"cfg\": %d, \"group_m\": %d, \"candidates\": %d, "         \
    "\"tile_m\": %d, \"tile_n\": %d, \"seconds\": " F ", \"terms_per_second\": " F "}"
const char *kReadFmt = BTAS_TUNE_LINE("%lg");
const char *kWriteFmt = BTAS_TUNE_LINE("%.9g");

bool valid_entry(const Key &k, const Entry &e) {
    if (k.sr != kMin && k.sr != kMax) return false;
    if (e.group_m < 1 || e.group_m > 1024) return false;
    if (k.dtype == BTAS_U16) {
        if (k.sr != kMin || e.var != kVarU16) return false;
        return std::find(std::begin(kU16Ns), std::end(kU16Ns), e.ns) != std::end(kU16Ns);
    }
    if (k.dtype != BTAS_I32 && k.dtype != BTAS_F32) return false;
    const GemmKernel *g = find_gemm_kernel(e.var, k.sr, e.ns, e.cfg);
    if (!g) return false;
    const bool is_f32 = g->var == kF32X2 || g->var == kF32Scalar || g->var == kF32Add2;
    return is_f32 == (k.dtype == BTAS_F32);
}

int load_file(const char *path, std::string *err) {
    FILE *f = fopen(path, "r");
    if (!f) {
        *err = std::string("cannot open ") + path;
        return -1;
    }
    std::vector<std::pair<Key, Entry>> got;
    char line[1024];
    int lineno = 0;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        const char *p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '\n' || *p == '\r' || *p == 0) continue;
        Key k{};
        Entry e{};
        const int got_n = sscanf(p, kReadFmt, &k.arch, &k.sms, &k.sr, &k.dtype, &k.mb, &k.nb, &k.kb, &e.var, &e.ns,
                                 &e.cfg, &e.group_m, &e.candidates, &e.tile_m, &e.tile_n, &e.seconds, &e.tps);
        if (got_n != 16 || !valid_entry(k, e)) {
            fclose(f);
            *err = std::string(path) + ": line " + std::to_string(lineno) +
                   (got_n != 16 ? " is not a tuning entry" : " names a kernel this build does not have");
            return -1;
        }
        got.emplace_back(k, e);
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : got) g_table[kv.first] = kv.second;
    return (int)got.size();
}

int save_file(const char *path, std::string *err) {
    std::vector<std::pair<Key, Entry>> all;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        all.assign(g_table.begin(), g_table.end());
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) {
        *err = std::string("cannot write ") + tmp;
        return -1;
    }
    for (auto &kv : all) {
        const Key &k = kv.first;
        const Entry &e = kv.second;
        fprintf(f, kWriteFmt, k.arch, k.sms, k.sr, k.dtype, k.mb, k.nb, k.kb, e.var, e.ns, e.cfg, e.group_m,
                e.candidates, e.tile_m, e.tile_n, e.seconds, e.tps);
        fputc('\n', f);
    }
    const bool ok = fflush(f) == 0;
    fclose(f);
    if (!ok || rename(tmp.c_str(), path) != 0) {
        *err = std::string("cannot write ") + path;
        return -1;
    }
    return (int)all.size();
}

void load_env_cache() {
    const char *p = getenv("BTAS_TUNE_CACHE");
    if (!p || !*p) return;
    FILE *f = fopen(p, "r");
    if (!f) return;  // nothing saved yet
    fclose(f);
    std::string err;
    if (load_file(p, &err) < 0) record_error(err.c_str());
}

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // SplitMix64 output function (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Seeded operand in the dtype's domain; about 1 in 16 entries is the
// (+)-identity (INF for min-plus, -INF for max-plus).
__global__ void tune_fill_kernel(void *p, long long rows, long long cols, long long ld, int dtype, int sr,
                                 unsigned long long seed) {
    const long long total = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i % cols;
        const unsigned long long h = mix64(seed + (unsigned long long)i * 0x9e3779b97f4a7c15ULL);
        const bool ident = (h & 15) == 0;
        const long long off = r * ld + c;
        if (dtype == BTAS_I32) {
            const int v = (int)((h >> 32) % 1000001u);
            static_cast<int *>(p)[off] = ident ? (sr == kMin ? kInfI32 : kNinfI32) : v;
        } else if (dtype == BTAS_F32) {
            const float v = (float)(h >> 40) * (1.0f / 16777216.0f);
            static_cast<float *>(p)[off] = ident ? __int_as_float(sr == kMin ? 0x7f800000 : 0xff800000) : v;
        } else {
            static_cast<uint16_t *>(p)[off] = ident ? (uint16_t)BTAS_INF_U16 : (uint16_t)((h >> 32) % 0x4000u);
        }
    }
}

// Counts entries of two rows x cols matrices (pitch ld, element size es)
// whose bits differ.
__global__ void tune_diff_kernel(const void *a, const void *b, long long rows, long long cols, long long ld, int es,
                                 unsigned long long *count) {
    unsigned long long local = 0;
    const long long total = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long off = (i / cols) * ld + i % cols;
        if (es == 4) local += static_cast<const uint32_t *>(a)[off] != static_cast<const uint32_t *>(b)[off];
        else local += static_cast<const uint16_t *>(a)[off] != static_cast<const uint16_t *>(b)[off];
    }
    if (local) atomicAdd(count, local);
}

unsigned grid_of(long long total) {
    return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
}

// ---------------------------------------------------------------- tuning run

struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    void *get(size_t bytes) {
        void *p = nullptr;
        if (ws_alloc(&p, bytes ? bytes : 256, st) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return p;
    }
    ~Scratch() {
        for (void *p : ptrs) ws_free(p, st);
    }
};

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Average seconds of one call of f: one warm-up, one probe to size the
// repetition count (about 20 ms of work, at least 2 and at most 50 calls).
template <class F>
cudaError_t time_call(F &&f, cudaStream_t st, Events &ev, double *sec) {
    cudaError_t e = f();
    if (e != cudaSuccess) return e;
    cudaEventRecord(ev.a, st);
    e = f();
    if (e != cudaSuccess) return e;
    cudaEventRecord(ev.b, st);
    if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) return e;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    const int reps = std::max(2, std::min(50, (int)std::ceil(20.0 / std::max(ms, 1e-3f))));
    cudaEventRecord(ev.a, st);
    for (int r = 0; r < reps; ++r)
        if ((e = f()) != cudaSuccess) return e;
    cudaEventRecord(ev.b, st);
    if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) return e;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    *sec = ms * 1e-3 / reps;
    return cudaSuccess;
}

struct Candidate {
    int var, ns, cfg, tile_m, tile_n;
    const GemmKernel *k;  // null for u16
};

}  // namespace

// Tunes (sr, dtype, m, n, k) on stream st and stores the result.  Returns a
// btas_status; *msg describes a failure.
int tune_run(int sr, int dtype, long long m, long long n, long long k, cudaStream_t st, TuneChoice *choice,
             btas_tune_result *res, std::string *msg) {
    Key key{};
    if (!make_key(sr, dtype, m, n, k, &key)) {
        *msg = "btas_tune_gemm: no current CUDA device";
        return BTAS_ERR_CUDA;
    }
    std::vector<Candidate> cands;
    if (dtype == BTAS_U16) {
        for (int ns : kU16Ns) cands.push_back(Candidate{kVarU16, ns, 0, 128, 256, nullptr});
    } else {
        for (int i = 0; i < gemm_kernel_count(); ++i) {
            const GemmKernel *g = gemm_kernel_at(i);
            const bool is_f32 = g->var == kF32X2 || g->var == kF32Scalar || g->var == kF32Add2;
            if (g->sr == sr && is_f32 == (dtype == BTAS_F32))
                cands.push_back(Candidate{g->var, g->ns, g->cfg, g->bm, g->bn, g});
        }
    }
    if (cands.empty()) {
        *msg = "btas_tune_gemm: no compiled kernel for this semiring and dtype";
        return BTAS_ERR_UNSUPPORTED;
    }
    const int es = dtype == BTAS_U16 ? 2 : 4;
    // operands: A m x k, B^T n x k (or B k x n for u16), C and the reference C m x n
    const long long ldk = dtype == BTAS_U16 ? ((k + 7) & ~7LL) : ((k + 3) & ~3LL);
    const long long ldn = dtype == BTAS_U16 ? ((n + 7) & ~7LL) : ((n + 3) & ~3LL);
    Scratch s(st);
    void *A = s.get((size_t)m * ldk * es);
    void *B = dtype == BTAS_U16 ? s.get((size_t)k * ldn * es) : s.get((size_t)n * ldk * es);
    void *C = s.get((size_t)m * ldn * es);
    void *R = s.get((size_t)m * ldn * es);
    void *Ad = dtype == BTAS_U16 ? s.get((size_t)m * ((k + 3) & ~3LL) * 4) : nullptr;
    unsigned long long *cnt = static_cast<unsigned long long *>(s.get(8));
    if (!A || !B || !C || !R || !cnt || (dtype == BTAS_U16 && !Ad)) {
        *msg = "btas_tune_gemm: scratch allocation failed";
        return BTAS_ERR_NOMEM;
    }
    const unsigned long long seed = 0x170104733ULL ^ ((unsigned long long)key.mb << 40) ^
                                    ((unsigned long long)key.nb << 48) ^ ((unsigned long long)key.kb << 56);
    tune_fill_kernel<<<grid_of(m * k), 256, 0, st>>>(A, m, k, ldk, dtype, sr, seed);
    if (dtype == BTAS_U16) tune_fill_kernel<<<grid_of(k * n), 256, 0, st>>>(B, k, n, ldn, dtype, sr, seed + 1);
    else tune_fill_kernel<<<grid_of(n * k), 256, 0, st>>>(B, n, k, ldk, dtype, sr, seed + 1);
    note_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = std::string("btas_tune_gemm: fill: ") + cudaGetErrorString(e);
        return BTAS_ERR_CUDA;
    }
    auto launcher = [&](const Candidate &c, int group_m) {
        return [&, group_m]() -> cudaError_t {
            if (!c.k) {
                U16Args a{};
                a.m = (int)m; a.n = (int)n; a.k = (int)k;
                a.A = static_cast<const uint16_t *>(A); a.lda = ldk;
                a.B = static_cast<const uint16_t *>(B); a.ldb = ldn;
                a.C = static_cast<uint16_t *>(C); a.ldc = ldn;
                a.one = 1;
                return launch_tgemm_u16_ws(a, static_cast<uint32_t *>(Ad), c.ns, st);
            }
            GemmArgs a{};
            a.m = (int)m; a.n = (int)n; a.k = (int)k;
            a.A = A; a.lda = ldk;
            a.Bt = B; a.ldb = ldk;
            a.C = C; a.ldc = ldn;
            a.vec_a = a.vec_b = 1;
            a.group_m = group_m;
            a.one = 1;
            return c.k->launch(a, st);
        };
    };
    Events ev;
    double best = 1e30;
    int bi = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        double t = 0;
        e = time_call(launcher(cands[i], 8), st, ev, &t);
        if (e != cudaSuccess) {
            *msg = std::string("btas_tune_gemm: candidate launch: ") + cudaGetErrorString(e);
            return BTAS_ERR_CUDA;
        }
        if (i == 0) {
            e = cudaMemcpyAsync(R, C, (size_t)m * ldn * es, cudaMemcpyDeviceToDevice, st);
        } else {
            cudaMemsetAsync(cnt, 0, 8, st);
            tune_diff_kernel<<<grid_of(m * n), 256, 0, st>>>(C, R, m, n, ldn, es, cnt);
            note_launch();
            unsigned long long h = 0;
            e = cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && h != 0) {
                char b[256];
                snprintf(b, sizeof b,
                         "btas_tune_gemm: candidate (variant %d, ns %d, cfg %d) differs from (variant %d, ns %d, "
                         "cfg %d) in %llu entries",
                         cands[i].var, cands[i].ns, cands[i].cfg, cands[0].var, cands[0].ns, cands[0].cfg, h);
                *msg = b;
                return BTAS_ERR_INTERNAL;
            }
        }
        if (e != cudaSuccess) {
            *msg = std::string("btas_tune_gemm: ") + cudaGetErrorString(e);
            return BTAS_ERR_CUDA;
        }
        if (t < best) {
            best = t;
            bi = (int)i;
        }
    }
    int best_group = 8;
    if (cands[bi].k) {
        for (int g : kGroups) {
            double t = 0;
            e = time_call(launcher(cands[bi], g), st, ev, &t);
            if (e != cudaSuccess) {
                *msg = std::string("btas_tune_gemm: candidate launch: ") + cudaGetErrorString(e);
                return BTAS_ERR_CUDA;
            }
            if (t < best * 0.98) {  // keep the default unless clearly faster
                best = t;
                best_group = g;
            }
        }
    }
    const Candidate &w = cands[bi];
    Entry ent{w.var, w.ns, w.cfg, best_group, (int)cands.size(), w.tile_m, w.tile_n, best,
              (double)m * n * k / best};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table[key] = ent;
    }
    if (choice) *choice = TuneChoice{ent.var, ent.ns, ent.cfg, ent.group_m};
    if (res) *res = btas_tune_result{ent.var, ent.ns, ent.cfg, ent.tile_m, ent.tile_n, ent.group_m,
                                     ent.candidates, ent.seconds, ent.tps};
    return BTAS_OK;
}

bool tune_choice(int sr, int dtype, long long m, long long n, long long k, cudaStream_t st, TuneChoice *out) {
    std::call_once(g_env_once, load_env_cache);
    Key key{};
    if (!make_key(sr, dtype, m, n, k, &key)) return false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_table.find(key);
        if (it != g_table.end()) {
            *out = TuneChoice{it->second.var, it->second.ns, it->second.cfg, it->second.group_m};
            return true;
        }
    }
    const char *t = getenv("BTAS_TUNE");
    if (!t || atoi(t) != 1) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    std::string msg;
    if (tune_run(sr, dtype, m, n, k, st, out, nullptr, &msg) != BTAS_OK) {
        record_error(msg.c_str());
        return false;
    }
    const char *p = getenv("BTAS_TUNE_CACHE");
    if (p && *p) {
        std::string err;
        if (save_file(p, &err) < 0) record_error(err.c_str());
    }
    return true;
}

}  // namespace btas

using namespace btas;

extern "C" {

btas_status btas_tune_gemm(int semiring, int dtype, int64_t m, int64_t n, int64_t k, btas_tune_result *out,
                           void *stream) {
    if (semiring != BTAS_MINPLUS && semiring != BTAS_MAXPLUS) {
        record_error("btas_tune_gemm: unknown semiring");
        return BTAS_ERR_ARG;
    }
    if (dtype != BTAS_I32 && dtype != BTAS_F32 && dtype != BTAS_U16) {
        record_error("btas_tune_gemm: unknown dtype");
        return BTAS_ERR_ARG;
    }
    if (m < 1 || n < 1 || k < 1 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) {
        record_error("btas_tune_gemm: sizes must be in [1, 2^31-1]");
        return BTAS_ERR_ARG;
    }
    if (dtype == BTAS_U16 && semiring != BTAS_MINPLUS) {
        record_error("btas_tune_gemm: BTAS_U16 is min-plus only");
        return BTAS_ERR_UNSUPPORTED;
    }
    std::call_once(g_env_once, load_env_cache);
    std::string msg;
    const int r = tune_run(semiring, dtype, m, n, k, static_cast<cudaStream_t>(stream), nullptr, out, &msg);
    if (r != BTAS_OK) record_error(msg.c_str());
    return static_cast<btas_status>(r);
}

int btas_tune_lookup(int semiring, int dtype, int64_t m, int64_t n, int64_t k, btas_tune_result *out) {
    std::call_once(g_env_once, load_env_cache);
    Key key{};
    if (!make_key(semiring, dtype, m, n, k, &key)) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(key);
    if (it == g_table.end()) return 0;
    const Entry &e = it->second;
    if (out) *out = btas_tune_result{e.var, e.ns, e.cfg, e.tile_m, e.tile_n, e.group_m, e.candidates, e.seconds, e.tps};
    return 1;
}

btas_status btas_tune_save(const char *path) {
    if (!path || !*path) {
        record_error("btas_tune_save: empty path");
        return BTAS_ERR_ARG;
    }
    std::string err;
    if (save_file(path, &err) < 0) {
        record_error(err.c_str());
        return BTAS_ERR_ARG;
    }
    return BTAS_OK;
}

btas_status btas_tune_load(const char *path, int *loaded) {
    if (!path || !*path) {
        record_error("btas_tune_load: empty path");
        return BTAS_ERR_ARG;
    }
    std::string err;
    const int c = load_file(path, &err);
    if (c < 0) {
        record_error(err.c_str());
        return BTAS_ERR_ARG;
    }
    if (loaded) *loaded = c;
    return BTAS_OK;
}

void btas_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
}

int btas_tune_entries(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return (int)g_table.size();
}

}  // extern "C"
