// Instantiations: int32, one fused DPX add-min/max per term.
#include "tgemm_launch.cuh"

namespace btas {
const GemmKernel kGemmI32Dpx[] = {
    entry<Cfg0, kI32Dpx, kMin, 0, 0>(), entry<Cfg0, kI32Dpx, kMax, 0, 0>(),
    entry<Cfg2, kI32Dpx, kMin, 0, 2>(), entry<Cfg2, kI32Dpx, kMax, 0, 2>(),
    entry<Cfg4, kI32Dpx, kMin, 0, 4>(), entry<Cfg4, kI32Dpx, kMax, 0, 4>(), entry<Cfg5, kI32Dpx, kMin, 0, 5>(),
};
const int kGemmI32DpxCount = sizeof(kGemmI32Dpx) / sizeof(kGemmI32Dpx[0]);
}  // namespace btas
