// The fused update + residual kernel k_updres (FP32 inner solve) for the fourth-order equations.
#include "rd_sweep.cuh"

namespace rd {
RD_FUSED_KIND(KK_CH_IMPL)
RD_FUSED_KIND(KK_CH_SPLIT)
RD_FUSED_KIND(KK_NONE_BIH)
}  // namespace rd
