// Instantiation of the PDHG sweep kernels for float arithmetic (inner solve of FP64 defect correction).
#include "rd_sweep.cuh"

namespace rd {
RD_SWEEP_INSTANTIATE(float)
}  // namespace rd
