// Instantiation of the PDHG sweep kernels for double arithmetic (plain FP64 method and the preconditioner entry point).
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_INSTANTIATE(double)
}  // namespace rd
