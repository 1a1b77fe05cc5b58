// Instantiations: int32, IMAD adds + 3-input min/max mixed with DPX.
#include "tgemm_launch.cuh"

namespace btas {
const GemmKernel kGemmI32Mix[] = {
    entry<Cfg0, kI32Mix, kMin, 4, 0>(), entry<Cfg0, kI32Mix, kMax, 4, 0>(),
    entry<Cfg0, kI32Mix, kMin, 5, 0>(), entry<Cfg0, kI32Mix, kMax, 5, 0>(),
    entry<Cfg0, kI32Mix, kMin, 6, 0>(), entry<Cfg0, kI32Mix, kMax, 6, 0>(),
    entry<Cfg0, kI32Mix, kMin, 8, 0>(),
    entry<Cfg2, kI32Mix, kMin, 5, 2>(), entry<Cfg2, kI32Mix, kMax, 5, 2>(),
    entry<Cfg4, kI32Mix, kMin, 4, 4>(), entry<Cfg4, kI32Mix, kMax, 4, 4>(),
    entry<Cfg4, kI32Mix, kMin, 5, 4>(), entry<Cfg4, kI32Mix, kMin, 6, 4>(),
    entry<Cfg5, kI32Mix, kMin, 5, 5>(),
};
const int kGemmI32MixCount = sizeof(kGemmI32Mix) / sizeof(kGemmI32Mix[0]);
}  // namespace btas
