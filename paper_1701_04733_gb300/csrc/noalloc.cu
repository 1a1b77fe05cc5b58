// btas_apsp_noalloc: APSP by repeated squaring for callers that cannot
// allocate device memory at call time.
//
// btas_apsp takes its scratch (a ping-pong matrix, a transpose buffer and the
// per-squaring change flags) from its stream-ordered pool on every call.  Some callers
// cannot do that: a process whose own memory pool has already reserved the
// device's free memory, or latency-critical code that must not allocate (an
// allocation can block or synchronise) inside its loop.  This entry point
// takes its scratch from one fixed array in device global memory instead,
// declared below.  Every GPU that loads the library holds that array
// (BTAS_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// Host code cannot use the array's name as a device address: in host code it
// names a host-side stand-in.  Every call looks the address up with
// cudaGetSymbolAddress for the current device (a host-side lookup, no
// synchronisation), so a context that was torn down and recreated (for
// example after cudaDeviceReset) gets the array's new address.  The first
// call on a device may load the library's device code there: make it before
// any stream capture.
//
// The smallest graphs run on the one-block kernel and the others on the
// cooperative kernel (the same kernels and size boundary as btas_apsp); the
// tiled int32 squarings below serve where a cooperative launch is refused.
//
// All calls share the one array, and each call leaves its contents behind.
// The change flags, which must start at zero, are cleared on the stream at the
// start of every call.  Calls whose work overlaps on the GPU (different
// streams, or different host threads without ordering) race on the array.
//
// The call reads nothing back.  The kernels leave their outcome (weight
// domain violations, a grid-barrier timeout, squarings that changed D) in the
// status words at the start of the array, and btas_apsp_noalloc_status reads
// them once the call's work has finished.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace btas {

namespace {

constexpr long long kMaxN = BTAS_NOALLOC_MAX_N;
constexpr size_t kFlagBytes = 256;                                  // change flags (<= 64 ints)
constexpr size_t kMatBytes = (size_t)kMaxN * (size_t)kMaxN * 4;     // one n x n int32 matrix
constexpr size_t kMidBytes = BTAS_NOALLOC_SCRATCH_BYTES - kFlagBytes;  // the cooperative kernel's workspace
static_assert(BTAS_NOALLOC_SCRATCH_BYTES ==
                  kFlagBytes + 3 * kMatBytes + 2048 + 4 * (size_t)kMaxN + 8 * 256 * (size_t)kMaxN,
              "scratch layout");

// The scratch: [flags | X (ping-pong output) | T (transpose, row pitch
// round4(n)) | one more matrix, 2 KiB and the edge lists of up to 256 edges
// per row]; the cooperative kernel takes everything after the flags as its
// workspace.
static __device__ __align__(256) unsigned char g_scratch[BTAS_NOALLOC_SCRATCH_BYTES];

// How the most recent call on each device ran, so that the status query
// knows which words hold its outcome.
enum Regime : int { kNone = 0, kTrivial, kOneBlock, kCooperative, kTiled };
struct LastCall {
    int regime;
    int S;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
LastCall g_last[kMaxDevices] = {};

btas_status set_error(btas_status s, const char *msg) {
    record_error(msg);
    return s;
}

cudaError_t current_device(int *dev) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return e;
    return (*dev < 0 || *dev >= kMaxDevices) ? cudaErrorInvalidDevice : cudaSuccess;
}

// Device address of g_scratch in the current context.
cudaError_t scratch_address(void **out) { return cudaGetSymbolAddress(out, g_scratch); }

void note_regime(int dev, int regime, int S) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_last[dev] = LastCall{regime, S};
}

int squarings(long long n) {
    int s = 0;
    long long reach = 1;
    while (reach < n - 1) {
        reach *= 2;
        ++s;
    }
    return s;
}

const GemmKernel *pick_kernel(long long n) {
    const long long tiles = ((n + 127) / 128) * ((n + 127) / 128);
    DeviceInfo di{};
    const int sms = current_device_info(&di) ? di.sms : 152;
    const GemmKernel *k = find_gemm_kernel(kI32Mix, kMin, 5, tiles >= 2LL * sms ? 0 : 2);
    if (!k) k = find_gemm_kernel(kI32Dpx, kMin, 0, 0);
    return k;
}

}  // namespace

}  // namespace btas

using namespace btas;

extern "C" btas_status btas_apsp_noalloc(int64_t n, const int32_t *W, int32_t *D, void *stream) {
    if (n < 0) return set_error(BTAS_ERR_ARG, "btas_apsp_noalloc: negative n");
    if (n > kMaxN) {
        char buf[160];
        snprintf(buf, sizeof buf, "btas_apsp_noalloc: n = %lld exceeds the fixed scratch limit of %lld vertices",
                 (long long)n, kMaxN);
        return set_error(BTAS_ERR_ARG, buf);
    }
    if (n > 0 && (!W || !D)) return set_error(BTAS_ERR_ARG, "btas_apsp_noalloc: NULL pointer");
    int dev = 0;
    cudaError_t e = current_device(&dev);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nn = (size_t)n * (size_t)n;
    const int S = squarings(n);
    if (S == 0) {
        if (n > 0 && D != W) {
            e = cudaMemcpyAsync(D, W, nn * 4, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        }
        note_regime(dev, kTrivial, 0);
        return BTAS_OK;
    }
    void *base = nullptr;
    e = scratch_address(&base);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
    int *flags = static_cast<int *>(base);
    int32_t *X = reinterpret_cast<int32_t *>(static_cast<char *>(base) + kFlagBytes);
    int32_t *T = reinterpret_cast<int32_t *>(static_cast<char *>(base) + kFlagBytes + kMatBytes);
    const long long ldt = (n + 3) & ~3LL;

    e = cudaMemsetAsync(flags, 0, kFlagBytes, st);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));

    // Small and mid-size graphs: the one-block kernel, or the cooperative
    // kernel (its three iterates fit in the scratch for every n); both take
    // their status words from the flag area and need no read-back here.
    if (n <= apsp_small_limit()) {
        e = launch_apsp_small(W, n, (int)n, S, true, D, n, flags, st);
        if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        note_regime(dev, kOneBlock, S);
        return BTAS_OK;
    }
    const char *no_mid = getenv("BTAS_APSP_NO_MID");  // as in btas_apsp: tiled squarings
    if (n <= apsp_mid_max_n() && apsp_mid_workspace_min(n) <= kMidBytes && !(no_mid && *no_mid && atoi(no_mid) != 0)) {
        e = launch_apsp_mid(W, n, (int)n, S, true, true, D, n, X, kMidBytes, flags, st);
        if (e == cudaSuccess) {
            note_regime(dev, kCooperative, S);
            return BTAS_OK;
        }
        if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorNotSupported)
            return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        cudaGetLastError();  // the grid cannot be co-resident here: tiled squarings below
    }

    // Outputs alternate so that the last squaring writes D: squaring s writes
    // bufs[(S-1-s) & 1].  In place (D == W) with S odd the first squaring
    // would write its own input, so the input is first copied to X.
    int32_t *bufs[2] = {D, X};
    const int32_t *cur = W;
    if ((const void *)W == (const void *)D && ((S - 1) & 1) == 0) {
        e = cudaMemcpyAsync(X, W, nn * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        cur = X;
    }
    const GemmKernel *kern = pick_kernel(n);
    if (!kern) return set_error(BTAS_ERR_UNSUPPORTED, "btas_apsp_noalloc: no int32 kernel");
    for (int s = 0; s < S; ++s) {
        int32_t *out = bufs[(S - 1 - s) & 1];
        const int *skip = s > 0 ? &flags[s - 1] : nullptr;
        e = launch_transpose4(cur, n, (int)n, (int)n, T, ldt, 0, skip, st);
        if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        GemmArgs a{};
        a.m = a.n = a.k = (int)n;
        a.A = cur;
        a.lda = n;
        a.Bt = T;
        a.ldb = ldt;
        a.C = out;
        a.ldc = n;
        a.prev = cur;
        a.ldp = n;
        a.changed = &flags[s];
        a.skip = skip;
        a.one = 1;
        a.vec_a = (reinterpret_cast<uintptr_t>(cur) & 15) == 0 && (n & 3) == 0;
        a.vec_b = 1;
        a.group_m = 8;
        e = kern->launch(a, st);
        if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
        cur = out;
    }
    note_regime(dev, kTiled, S);
    return BTAS_OK;
}

extern "C" btas_status btas_apsp_noalloc_status(void *stream, int *squarings_done) {
    int dev = 0;
    cudaError_t e = current_device(&dev);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
    LastCall last;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        last = g_last[dev];
    }
    if (last.regime == kNone)
        return set_error(BTAS_ERR_ARG, "btas_apsp_noalloc_status: no btas_apsp_noalloc call on this device yet");
    if (squarings_done) *squarings_done = 0;
    if (last.regime == kTrivial) return BTAS_OK;
    void *base = nullptr;
    e = scratch_address(&base);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
    // the status words (at most 64 ints), copied into pageable host memory:
    // ordered after the call's work on `stream`, nothing allocated
    int words[64] = {};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(words, base, sizeof words, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(BTAS_ERR_CUDA, cudaGetErrorString(e));
    if (last.regime == kTiled) {
        // one change flag per squaring; the weight domain is not checked here
        int done = 0;
        for (int s = 0; s < last.S && s < 64; ++s) done += words[s] != 0;
        if (squarings_done) *squarings_done = done;
        return BTAS_OK;
    }
    // one-block kernel: [0] entries outside the domain, [1] largest weight,
    // [2] squarings that changed D; the cooperative kernel adds [3] status
    if (last.regime == kCooperative && words[3] != 0) {
        record_error("btas_apsp_noalloc: a bounded grid-barrier wait expired; D was not written");
        return static_cast<btas_status>(words[3]);
    }
    if (words[0] != 0) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "btas_apsp_noalloc: %d entries of W outside the weight domain; D was not written", words[0]);
        return set_error(BTAS_ERR_ARG, buf);
    }
    if (squarings_done) *squarings_done = words[2];
    return BTAS_OK;
}
