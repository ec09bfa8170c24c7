// reach_cta_256.cu -- instantiations of the CTA-per-world reach kernel for 256-thread
// CTAs (compiled apart so that the variants build in parallel).
#include "reach_cta.cuh"

namespace reach_cta {
IMIN_REACH_CTA_INSTANTIATE(256, 4)
IMIN_REACH_CTA_INSTANTIATE(256, 8)
}  // namespace reach_cta
