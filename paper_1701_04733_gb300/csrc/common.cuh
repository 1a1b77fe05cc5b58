// Shared device/host helpers of the CUDA path: semiring constants, cp.async
// and register-level semiring primitives.  Nothing here is used by the CPU
// oracle.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/btas.h"

namespace btas {

constexpr int kInfI32 = BTAS_INF_I32;
constexpr int kNinfI32 = BTAS_NINF_I32;
// Any min-plus result >= kInfI32 - 2^28 contains an INF term (finite operands
// are bounded by 2^28, so finite sums stay <= 2^29 < this threshold).
constexpr int kClampI32 = BTAS_INF_I32 - BTAS_I32_FINITE_MAX;
constexpr unsigned kInfU16x2 = 0x7FFF7FFFu;

enum Semiring : int { kMin = 0, kMax = 1 };

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
// 4-byte asynchronous copy through L1 (.ca): only for data that no CTA of the
// running launch writes, since L1 is not coherent within a launch.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ------------------------------------------------- semiring primitives
// 3-input min/max of fp32 (sm_100+ PTX form).
template <int SR>
__device__ __forceinline__ float fsel3(float a, float b, float c) {
    float d;
    if (SR == kMin)
        asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    else
        asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
template <int SR>
__device__ __forceinline__ float fsel2(float a, float b) {
    return SR == kMin ? fminf(a, b) : fmaxf(a, b);
}
// Two IEEE round-to-nearest fp32 adds in one instruction (sm_100+).
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// Fused add then min/max (DPX).
template <int SR>
__device__ __forceinline__ int iaddsel(int a, int b, int c) {
    return SR == kMin ? __viaddmin_s32(a, b, c) : __viaddmax_s32(a, b, c);
}
template <int SR>
__device__ __forceinline__ int isel3(int a, int b, int c) {
    return SR == kMin ? __vimin3_s32(a, b, c) : __vimax3_s32(a, b, c);
}
// a*one + b with a runtime `one`: an integer add the compiler has to issue as
// a multiply-add, i.e. on the FMA pipe rather than the ALU pipe.
__device__ __forceinline__ int imad_add(int a, int one, int b) {
    int d;
    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(one), "r"(b));
    return d;
}
__device__ __forceinline__ unsigned u16x2_addmin(unsigned a, unsigned b, unsigned c) {
    return __viaddmin_u16x2(a, b, c);
}
__device__ __forceinline__ unsigned u16x2_min3(unsigned a, unsigned b, unsigned c) {
    return __vimin3_u16x2(a, b, c);
}

// Clamp an int32 accumulator back to the INF encoding.
template <int SR>
__device__ __forceinline__ int clamp_i32(int v) {
    if (SR == kMin) return v >= kClampI32 ? kInfI32 : v;
    return v <= -kClampI32 ? kNinfI32 : v;
}

template <typename T, int SR>
struct Ident;
template <>
struct Ident<int, kMin> { static __device__ __host__ int v() { return kInfI32; } };
template <>
struct Ident<int, kMax> { static __device__ __host__ int v() { return kNinfI32; } };
template <>
struct Ident<float, kMin> { static __device__ __host__ float v() { return __builtin_huge_valf(); } };
template <>
struct Ident<float, kMax> { static __device__ __host__ float v() { return -__builtin_huge_valf(); } };

}  // namespace btas
