// Instantiations: fp32, add.f32x2 + 3-input min/max, and the scalar form.
#include "tgemm_launch.cuh"

namespace btas {
const GemmKernel kGemmF32[] = {
    entry<Cfg0, kF32X2, kMin, 0, 0>(), entry<Cfg0, kF32X2, kMax, 0, 0>(),
    entry<Cfg1, kF32X2, kMin, 0, 1>(), entry<Cfg1, kF32X2, kMax, 0, 1>(),
    entry<Cfg2, kF32X2, kMin, 0, 2>(), entry<Cfg2, kF32X2, kMax, 0, 2>(),
    entry<Cfg0, kF32Scalar, kMin, 0, 0>(), entry<Cfg0, kF32Scalar, kMax, 0, 0>(),
    entry<Cfg4, kF32X2, kMin, 0, 4>(), entry<Cfg4, kF32X2, kMax, 0, 4>(), entry<Cfg5, kF32X2, kMin, 0, 5>(),
    entry<Cfg0, kF32Add2, kMin, 0, 0>(), entry<Cfg4, kF32Add2, kMin, 0, 4>(),
};
const int kGemmF32Count = sizeof(kGemmF32) / sizeof(kGemmF32[0]);
}  // namespace btas
