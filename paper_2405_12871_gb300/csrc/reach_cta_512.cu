// reach_cta_512.cu -- instantiations of the CTA-per-world reach kernel for 512-thread
// CTAs (compiled apart so that the variants build in parallel).
#include "reach_cta.cuh"

namespace reach_cta {
IMIN_REACH_CTA_INSTANTIATE(512, 2)
IMIN_REACH_CTA_INSTANTIATE(512, 4)
}  // namespace reach_cta
