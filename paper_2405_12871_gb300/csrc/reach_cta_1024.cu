// reach_cta_1024.cu -- instantiations of the CTA-per-world reach kernel for 1024-thread
// CTAs (compiled apart so that the variants build in parallel).
#include "reach_cta.cuh"

namespace reach_cta {
IMIN_REACH_CTA_INSTANTIATE(1024, 1)
IMIN_REACH_CTA_INSTANTIATE(1024, 2)
}  // namespace reach_cta
