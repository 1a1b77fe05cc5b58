// Issue-rate probe: how many tropical terms one SM completes per clock for a
// given register-only instruction mix.  It measures the empirical ceiling
// that the tropical GEMM kernels are compared against (their roofline is set
// by ALU issue, not by memory or tensor cores).  One CTA of 256 threads per
// SM keeps 64 independent accumulators per thread; the 8 + 8 operand
// registers change every iteration, so no two terms share a sum.  The
// launch reserves 120 KiB of shared memory per CTA so that exactly one CTA
// runs on each SM.
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

template <int MIX>
__global__ void __launch_bounds__(256, 1) probe_kernel(const float *in, float *out, int iters, long long *cyc, int one) {
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
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float a0, a1, b0, b1;
                unpack2(x[i], a0, a1);
                unpack2(y[j], b0, b1);
                if (MIX == 0) {  // int32: two DPX fused add-min (2 terms)
                    const int t = __viaddmin_s32(__float_as_int(a0), __float_as_int(b0), __float_as_int(acc[i][j]));
                    acc[i][j] = __int_as_float(__viaddmin_s32(__float_as_int(a1), __float_as_int(b1), t));
                } else if (MIX == 1) {  // fp32: add.f32x2 + 3-input min (2 terms)
                    float lo, hi;
                    unpack2(fadd2(x[i], y[j]), lo, hi);
                    acc[i][j] = fsel3<kMin>(acc[i][j], lo, hi);
                } else if (MIX == 2) {  // packed 16-bit: two DPX u16x2 add-min (4 terms)
                    const unsigned t = __viaddmin_u16x2(__float_as_uint(a0), __float_as_uint(b0), __float_as_uint(acc[i][j]));
                    acc[i][j] = __uint_as_float(__viaddmin_u16x2(__float_as_uint(a1), __float_as_uint(b1), t));
                } else if (MIX == 4 || MIX == 5 || (MIX == 6 && j < 5)) {
                    // int32: two adds (4: IADD on the ALU pipe; 5, 6: IMAD x*1+y on
                    // the FMA pipe) + one 3-input min (2 terms); 6 uses this on 5
                    // of 8 columns and DPX on the other 3
                    const int s0 = MIX == 4 ? __float_as_int(a0) + __float_as_int(b0)
                                            : imad_add(__float_as_int(a0), one, __float_as_int(b0));
                    const int s1 = MIX == 4 ? __float_as_int(a1) + __float_as_int(b1)
                                            : imad_add(__float_as_int(a1), one, __float_as_int(b1));
                    acc[i][j] = __int_as_float(__vimin3_s32(__float_as_int(acc[i][j]), s0, s1));
                } else if (MIX == 6) {
                    const int t = __viaddmin_s32(__float_as_int(a0), __float_as_int(b0), __float_as_int(acc[i][j]));
                    acc[i][j] = __int_as_float(__viaddmin_s32(__float_as_int(a1), __float_as_int(b1), t));
                } else if (MIX == 7) {  // fp32: two scalar RN adds + 3-input min (2 terms)
                    acc[i][j] = fsel3<kMin>(acc[i][j], __fadd_rn(a0, b0), __fadd_rn(a1, b1));
                } else {  // reference: two FFMA (2 multiply-adds)
                    acc[i][j] = fmaf(a1, b1, fmaf(a0, b0, acc[i][j]));
                }
            }
    }
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) s += acc[i][j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// Dynamic shared memory large enough that only one probe CTA fits per SM.
constexpr int kProbeSmem = 120 * 1024;

template <int MIX>
cudaError_t run_probe(int sms, const float *in, float *out, long long *cyc, int iters) {
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(probe_kernel<MIX>), kProbeSmem);
    if (e != cudaSuccess) return e;
    probe_kernel<MIX><<<sms, 256, kProbeSmem>>>(in, out, iters, cyc, 1);
    note_launch();
    return cudaGetLastError();
}

}  // namespace
}  // namespace btas

using namespace btas;

extern "C" btas_status btas_measure_issue_rate(int mix, double *terms_per_clock_per_sm) {
    if (mix < 0 || mix > 7 || !terms_per_clock_per_sm) {
        record_error("btas_measure_issue_rate: mix must be 0..7");
        return BTAS_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *in = nullptr, *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&in, 1024 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&out, (size_t)sms * 256 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&cyc, (size_t)sms * sizeof(long long)) != cudaSuccess) {
        cudaFree(in);
        cudaFree(out);
        record_error("btas_measure_issue_rate: allocation failed");
        return BTAS_ERR_NOMEM;
    }
    std::vector<float> h(1024);
    for (int i = 0; i < 1024; ++i) h[i] = (float)((i * 37) % 101) * 0.01f;
    cudaMemcpy(in, h.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice);
    const int iters = 4000;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
        switch (mix) {
            case 0: e = run_probe<0>(sms, in, out, cyc, rep ? iters : 16); break;
            case 1: e = run_probe<1>(sms, in, out, cyc, rep ? iters : 16); break;
            case 2: e = run_probe<2>(sms, in, out, cyc, rep ? iters : 16); break;
            case 3: e = run_probe<3>(sms, in, out, cyc, rep ? iters : 16); break;
            case 4: e = run_probe<4>(sms, in, out, cyc, rep ? iters : 16); break;
            case 5: e = run_probe<5>(sms, in, out, cyc, rep ? iters : 16); break;
            case 6: e = run_probe<6>(sms, in, out, cyc, rep ? iters : 16); break;
            default: e = run_probe<7>(sms, in, out, cyc, rep ? iters : 16); break;
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    std::vector<long long> hc(sms);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, (size_t)sms * sizeof(long long), cudaMemcpyDeviceToHost);
    cudaFree(in);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) {
        record_error(cudaGetErrorString(e));
        return BTAS_ERR_CUDA;
    }
    long long mx = 1;
    for (long long c : hc) mx = c > mx ? c : mx;
    const double terms_per_thread = (double)iters * 64 * (mix == 2 ? 4 : 2);
    *terms_per_clock_per_sm = terms_per_thread * 256.0 / (double)mx;
    return BTAS_OK;
}
