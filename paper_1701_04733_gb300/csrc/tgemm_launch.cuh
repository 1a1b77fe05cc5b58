// Launch wrapper and registry-entry helper for the NT tropical GEMM kernel.
#pragma once
#include <atomic>

#include "kernels.h"
#include "tgemm.cuh"

namespace btas {

// Per-translation-unit kernel tables (external linkage; see btas_api.cu).
extern const GemmKernel kGemmI32Dpx[];
extern const int kGemmI32DpxCount;
extern const GemmKernel kGemmI32Mix[];
extern const int kGemmI32MixCount;
extern const GemmKernel kGemmF32[];
extern const int kGemmF32Count;

using Cfg0 = TileCfg<128, 128, 32, 3>;  // 256 threads, 108 KiB smem
using Cfg1 = TileCfg<128, 128, 32, 4>;  // 256 threads, 144 KiB smem
using Cfg2 = TileCfg<64, 64, 32, 4>;    //  64 threads,  72 KiB smem (small problems)
using Cfg3 = TileCfg<128, 64, 32, 4>;   // 128 threads, 108 KiB smem
using Cfg4 = TileCfg<128, 128, 32, 3, 2, 2, 1>;  // 2 CTAs/SM, 64-bit fragments
using Cfg5 = TileCfg<128, 128, 32, 3, 2, 4, 1>;  // 2 CTAs/SM, 128-bit fragments

template <class Cfg, int VAR, int SR, int NS>
cudaError_t launch_nt(const GemmArgs &a, cudaStream_t st) {
    auto kern = tgemm_nt_kernel<Cfg, VAR, SR, NS>;
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load(std::memory_order_relaxed) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit);
    }
    const long long tiles = (long long)((a.m + Cfg::BM - 1) / Cfg::BM) * ((a.n + Cfg::BN - 1) / Cfg::BN);
    if (tiles <= 0) return cudaSuccess;
    GemmArgs args = a;
    args.kwave = a.kwave * Cfg::MINB;  // SMs -> CTAs resident at once
    kern<<<(unsigned)tiles, Cfg::kThreads, Cfg::kSmemBytes, st>>>(args);
    note_launch();
    return cudaGetLastError();
}

template <class Cfg, int VAR, int SR, int NS, int CFGID>
constexpr GemmKernel entry() {
    return GemmKernel{VAR, SR, NS, CFGID, Cfg::BM, Cfg::BN, Cfg::kThreads, Cfg::kSmemBytes,
                      &launch_nt<Cfg, VAR, SR, NS>};
}

}  // namespace btas
