// The sweep kernels k_res and k_upd in double for the second-order equations (five-point
// Laplacian: no reaction, Allen-Cahn, Gray-Scott, Schnakenberg) and the preconditioner-only form.
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_KIND(double, KK_NONE_LAP)
RD_SWEEP_KIND(double, KK_AC)
RD_SWEEP_KIND(double, KK_GS)
RD_SWEEP_KIND(double, KK_SCHNAK)
RD_SWEEP_KIND(double, KK_PCONLY)
}  // namespace rd
