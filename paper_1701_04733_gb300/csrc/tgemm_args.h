// Arguments of the tropical GEMM kernels (host and device visible).
#pragma once

namespace btas {

enum Variant : int { kI32Dpx = 0, kI32Mix = 1, kF32X2 = 2, kF32Scalar = 3, kF32Add2 = 4 };

struct GemmArgs {
    int m, n, k;
    const void *A;
    long long lda;
    const void *Bt;  // B transposed: n x k
    long long ldb;
    void *C;
    long long ldc;
    int accumulate;     // C <- C (+) A (x) B
    const void *prev;   // optional: output (i,j) is compared with prev[i*ldp+j]
    long long ldp;
    int *changed;       // set to 1 if any output differs from prev
    const int *skip;    // optional: *skip == 0 => C = prev (converged squaring)
    int one;            // the constant 1, opaque to the compiler
    int vec_a, vec_b;   // operand rows are 16-byte aligned (cp.async usable)
    int ro_a, ro_b;     // operand not written by any CTA of this launch: unaligned and edge
                        // elements may then be staged with 4-byte cp.async through L1
    int group_m;        // CTA rasterisation: tile rows per group
    int *maxfin;        // optional: atomicMax of the largest finite output (as int)
    const int *bypass;  // optional: *bypass != 0 => do nothing (another path computes C)
    int kwave;          // > 0: rasterise by groups of group_m tile COLUMNS (consecutive
                        // waves share their B^T panels) and run k backwards in every other
                        // wave of kwave CTAs, so that a wave starts on the k-slices the
                        // previous one left in L2 (the launcher scales it by CTAs per SM)
};

}  // namespace btas
