// The fused update + residual kernel k_updres (FP32 inner solve) for the second-order equations.
#include "rd_sweep.cuh"

namespace rd {
RD_FUSED_KIND(KK_NONE_LAP)
RD_FUSED_KIND(KK_AC)
RD_FUSED_KIND(KK_GS)
RD_FUSED_KIND(KK_SCHNAK)
}  // namespace rd
