// The sweep kernels k_res and k_upd in float for the second-order equations (five-point
// Laplacian: no reaction, Allen-Cahn, Gray-Scott, Schnakenberg) and the preconditioner-only form.
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_KIND(float, KK_NONE_LAP)
RD_SWEEP_KIND(float, KK_AC)
RD_SWEEP_KIND(float, KK_GS)
RD_SWEEP_KIND(float, KK_SCHNAK)
RD_SWEEP_KIND(float, KK_PCONLY)
}  // namespace rd
