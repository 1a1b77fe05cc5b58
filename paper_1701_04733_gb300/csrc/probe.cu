// Issue-rate probe: how many tropical terms one SM completes per clock for a
// given register-only instruction mix.  It measures the empirical ceiling
// that the tropical GEMM kernels are compared against (their roofline is set
// by ALU issue, not by memory or tensor cores).  CTAs of 256 threads keep 64
// independent accumulators per thread; the 8 + 8 operand registers change
// every iteration, so no two terms share a sum.  The launch reserves enough
// shared memory per CTA that exactly `ctas_per_sm` CTAs run on each SM, and
// the rate of an SM is taken over the span from its first CTA's start to its
// last CTA's end (clock64 is a per-SM counter).
//
// Besides the mixes the kernels use, the probe carries diagnostic mixes that
// separate three candidate limits of 32-bit tropical terms:
//   * pipe throughput (ALU, FMA-heavy, FMA-lite lanes per clock);
//   * register-operand reads per clock (the same instruction with one operand
//     an immediate, so one register read fewer per instruction);
//   * warps available to hide latency (1 or 2 CTAs per SM);
//   * operand reuse between consecutive instructions: the mixes above keep a
//     row's A operand in consecutive instructions (the product kernels'
//     order); mix 15 is DPX with a different A in every consecutive
//     instruction.
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace btas {
namespace {

__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

__device__ __forceinline__ int fi(float v) { return __float_as_int(v); }
__device__ __forceinline__ float if_(int v) { return __int_as_float(v); }

// One (i, j) update of mix MIX: two terms (four for the packed u16x2 mix).
// Operands are bit patterns; only the instruction stream matters here.
template <int MIX, int J>
__device__ __forceinline__ float probe_term(float acc, uint64_t xi, uint64_t yj, int one) {
    float a0, a1, b0, b1;
    unpack2(xi, a0, a1);
    unpack2(yj, b0, b1);
    if constexpr (MIX == 0) {  // int32: two DPX fused add-min
        const int t = __viaddmin_s32(fi(a0), fi(b0), fi(acc));
        return if_(__viaddmin_s32(fi(a1), fi(b1), t));
    } else if constexpr (MIX == 1) {  // fp32: add.f32x2 + 3-input min
        float lo, hi;
        unpack2(fadd2(xi, yj), lo, hi);
        return fsel3<kMin>(acc, lo, hi);
    } else if constexpr (MIX == 2) {  // packed 16-bit: two DPX u16x2 add-min (4 terms)
        const unsigned t = __viaddmin_u16x2(__float_as_uint(a0), __float_as_uint(b0), __float_as_uint(acc));
        return __uint_as_float(__viaddmin_u16x2(__float_as_uint(a1), __float_as_uint(b1), t));
    } else if constexpr (MIX == 3) {  // reference: two FFMA
        return fmaf(a1, b1, fmaf(a0, b0, acc));
    } else if constexpr (MIX == 4) {  // int32: IADD x2 + 3-input min
        return if_(__vimin3_s32(fi(acc), fi(a0) + fi(b0), fi(a1) + fi(b1)));
    } else if constexpr (MIX == 5 || (MIX == 6 && J < 5)) {  // int32: IMAD x2 + 3-input min
        return if_(__vimin3_s32(fi(acc), imad_add(fi(a0), one, fi(b0)), imad_add(fi(a1), one, fi(b1))));
    } else if constexpr (MIX == 6) {
        return probe_term<0, J>(acc, xi, yj, one);
    } else if constexpr (MIX == 7) {  // fp32: two scalar RN adds + 3-input min
        return fsel3<kMin>(acc, __fadd_rn(a0, b0), __fadd_rn(a1, b1));
    } else if constexpr (MIX == 8) {  // FFMA x2, second operand an immediate (2 register reads)
        return fmaf(a1, 1.25f + J, fmaf(a0, 0.75f + J, acc));
    } else if constexpr (MIX == 9) {  // fp32: two scalar adds of an immediate + 3-input min
        return fsel3<kMin>(acc, __fadd_rn(a0, 0.5f + J), __fadd_rn(a1, 0.25f + J));
    } else if constexpr (MIX == 10) {  // int32: IADD of an immediate x2 + 3-input min
        return if_(__vimin3_s32(fi(acc), fi(a0) + (7 + J), fi(a1) + (13 + J)));
    } else if constexpr (MIX == 11) {  // int32: DPX add-min with an immediate addend
        const int t = __viaddmin_s32(fi(a0), 7 + J, fi(acc));
        return if_(__viaddmin_s32(fi(a1), 13 + J, t));
    } else if constexpr (MIX == 12) {  // three pipes: DPX on 3 of 8 columns, IMAD+min3 on 3, FADD+min3 on 2
        if constexpr (J < 3) return probe_term<0, J>(acc, xi, yj, one);
        else if constexpr (J < 6) return probe_term<5, J>(acc, xi, yj, one);
        else return probe_term<7, J>(acc, xi, yj, one);
    } else if constexpr (MIX == 13) {  // DPX on 3 of 8 columns, f32x2 + min3 on 5
        if constexpr (J < 3) return probe_term<0, J>(acc, xi, yj, one);
        else return probe_term<1, J>(acc, xi, yj, one);
    } else {  // 14: IMAD with an immediate addend x2 + 3-input min (x*one + imm)
        return if_(__vimin3_s32(fi(acc), imad_add(fi(a0), one, 7 + J), imad_add(fi(a1), one, 13 + J)));
    }
}

template <int MIX, int J>
__device__ __forceinline__ void probe_row(float (&acc)[8], uint64_t xi, const uint64_t (&y)[8], int one) {
    acc[J] = probe_term<MIX, J>(acc[J], xi, y[J], one);
    if constexpr (J + 1 < 8) probe_row<MIX, J + 1>(acc, xi, y, one);
}

// Mix 15: the DPX terms of mix 0 with output (i, j) taking A operand
// x[(i + j) % 8], so that consecutive instructions (j inner) never share an A
// register.
template <int J>
__device__ __forceinline__ void probe_row_rotated(float (&acc)[8], int i, const uint64_t (&x)[8],
                                                  const uint64_t (&y)[8], int one) {
    acc[J] = probe_term<0, J>(acc[J], x[(i + J) & 7], y[J], one);
    if constexpr (J + 1 < 8) probe_row_rotated<J + 1>(acc, i, x, y, one);
}

template <int MIX, int MINB>
__global__ void __launch_bounds__(256, MINB) probe_kernel(const float *in, float *out, int iters, long long *cyc,
                                                        int one) {
    uint64_t x[8], y[8];
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[i] = pk(in[(threadIdx.x + i) & 63], in[(threadIdx.x + i + 5) & 63]);
        y[i] = pk(in[64 + ((threadIdx.x * 3 + i) & 63)], in[64 + ((threadIdx.x + 7 * i) & 63)]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = in[128 + ((8 * i + j + threadIdx.x) & 63)];
    const uint64_t inc = pk(in[200], in[201]);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fadd2(x[i], inc);
#pragma unroll
        for (int j = 0; j < 8; ++j) y[j] = fadd2(y[j], inc);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if constexpr (MIX == 15) probe_row_rotated<0>(acc[i], i, x, y, one);
            else probe_row<MIX, 0>(acc[i], x[i], y, one);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) s += acc[i][j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cyc[3 * blockIdx.x] = t0;
        cyc[3 * blockIdx.x + 1] = t1;
        cyc[3 * blockIdx.x + 2] = smid;
    }
}

constexpr int kMaxMix = 15;

// Dynamic shared memory that lets exactly MINB probe CTAs share an SM.
template <int MINB>
constexpr int probe_smem() { return MINB == 1 ? 120 * 1024 : 100 * 1024; }

template <int MIX, int MINB>
cudaError_t run_probe_t(int blocks, const float *in, float *out, long long *cyc, int iters) {
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(probe_kernel<MIX, MINB>), probe_smem<MINB>());
    if (e != cudaSuccess) return e;
    probe_kernel<MIX, MINB><<<blocks, 256, probe_smem<MINB>()>>>(in, out, iters, cyc, 1);
    note_launch();
    return cudaGetLastError();
}

template <int MINB, int MIX = 0>
cudaError_t run_probe(int mix, int blocks, const float *in, float *out, long long *cyc, int iters) {
    if (mix == MIX) return run_probe_t<MIX, MINB>(blocks, in, out, cyc, iters);
    if constexpr (MIX < kMaxMix) return run_probe<MINB, MIX + 1>(mix, blocks, in, out, cyc, iters);
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace btas

using namespace btas;

extern "C" btas_status btas_measure_issue_rate_ex(int mix, int ctas_per_sm, double *terms_per_clock_per_sm) {
    if (mix < 0 || mix > kMaxMix || (ctas_per_sm != 1 && ctas_per_sm != 2) || !terms_per_clock_per_sm) {
        record_error("btas_measure_issue_rate_ex: mix must be 0..15 and ctas_per_sm 1 or 2");
        return BTAS_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * ctas_per_sm;
    float *in = nullptr, *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&in, 1024 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&cyc, (size_t)blocks * 3 * sizeof(long long)) != cudaSuccess) {
        cudaFree(in);
        cudaFree(out);
        record_error("btas_measure_issue_rate_ex: allocation failed");
        return BTAS_ERR_NOMEM;
    }
    std::vector<float> h(1024);
    for (int i = 0; i < 1024; ++i) h[i] = (float)((i * 37) % 101) * 0.01f;
    cudaError_t e = cudaMemcpy(in, h.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice);
    const int iters = 4000;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
        const int it = rep ? iters : 16;
        e = ctas_per_sm == 1 ? run_probe<1>(mix, blocks, in, out, cyc, it) : run_probe<2>(mix, blocks, in, out, cyc, it);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    std::vector<long long> hc((size_t)blocks * 3);
    if (e == cudaSuccess)
        e = cudaMemcpy(hc.data(), cyc, hc.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    cudaFree(in);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) {
        record_error(cudaGetErrorString(e));
        return BTAS_ERR_CUDA;
    }
    // per SM: span from its first CTA's start to its last CTA's end; the
    // slowest SM sets the rate
    std::vector<long long> lo(sms, -1), hi(sms, -1);
    std::vector<int> cnt(sms, 0);
    for (int b = 0; b < blocks; ++b) {
        const long long s = hc[3 * b + 2];
        if (s < 0 || s >= sms) continue;
        if (lo[s] < 0 || hc[3 * b] < lo[s]) lo[s] = hc[3 * b];
        if (hc[3 * b + 1] > hi[s]) hi[s] = hc[3 * b + 1];
        ++cnt[s];
    }
    const double terms_per_thread = (double)iters * 64 * (mix == 2 ? 4 : 2);
    double worst = 0.0;
    bool any = false;
    for (int s = 0; s < sms; ++s) {
        if (cnt[s] == 0 || hi[s] <= lo[s]) continue;
        const double r = terms_per_thread * 256.0 * cnt[s] / (double)(hi[s] - lo[s]);
        if (!any || r < worst) worst = r;
        any = true;
    }
    if (!any) {
        record_error("btas_measure_issue_rate_ex: no timing recorded");
        return (btas_status)BTAS_ERR_INTERNAL;
    }
    *terms_per_clock_per_sm = worst;
    return BTAS_OK;
}

extern "C" btas_status btas_measure_issue_rate(int mix, double *terms_per_clock_per_sm) {
    if (mix < 0 || mix > 7) {
        record_error("btas_measure_issue_rate: mix must be 0..7");
        return BTAS_ERR_ARG;
    }
    return btas_measure_issue_rate_ex(mix, 1, terms_per_clock_per_sm);
}
