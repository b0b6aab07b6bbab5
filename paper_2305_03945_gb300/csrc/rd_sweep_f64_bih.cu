// The sweep kernels k_res and k_upd in double for the fourth-order equations (13-point biharmonic:
// Cahn-Hilliard implicit and convex-concave split, no reaction).
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_KIND(double, KK_CH_IMPL)
RD_SWEEP_KIND(double, KK_CH_SPLIT)
RD_SWEEP_KIND(double, KK_NONE_BIH)
}  // namespace rd
