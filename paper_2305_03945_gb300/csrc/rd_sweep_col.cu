// The column-transform kernel k_col in float and double, and the per-equation dispatch of one
// PDHG iteration (the equation kernels themselves are in rd_sweep_{f32,f64}_{lap,bih}.cu and
// rd_fused_{lap,bih}.cu).
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_COMMON(float)
RD_SWEEP_COMMON(double)
}  // namespace rd
