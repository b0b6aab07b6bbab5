// Host-side launchers of the 3-D PDHG kernels (rd_3d.cu) and their launch plan.
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

// One PDHG iteration on a 3-D grid (k3_res, the five transform passes, k3_upd) of the solve
// described by d; with ev != NULL, events ev[0..3] are recorded around the residual, the
// transform passes and the update.
template <class T>
cudaError_t launch_iteration3(const Desc& d, State* st, cudaStream_t s, cudaEvent_t* ev);
// Y = G^{-1} W on a 3-D grid: W in d.WY, Y into d.X (d.mode = MODE_PRECOND_ONLY).
template <class T>
cudaError_t launch_precond3(const Desc& d, State* st, cudaStream_t s);
// Raise the dynamic shared-memory limit of the 3-D transform passes.
template <class T>
cudaError_t allow3(int optin);

// Step set-up and FP64 residual of defect correction on 3-D grids (hd: host copy of *d64).
cudaError_t launch_begin3(const Desc& hd, const Desc* d64, State* st, const double* uk, double* rhs, double tol,
                          int tol_kind, cudaStream_t s);
cudaError_t launch_resid64_3(const Desc& hd, const Desc* d64, State* outer, State* inner, const double* u,
                             const double* rhs, double* w64, float* r32, float* u32, float* z0, float* z1, int decide,
                             double rtol, int max_outer, cudaStream_t s);

// Launch plan of the 3-D kernels: blocks per instance (about eight points per thread, at most
// 1024: one transform tile per block at 128^3, which measured 22% faster than one wave of two
// blocks per SM) and, per axis, the lines per tile of the transform passes (even,
// dividing the lines available: up to 16 FP32 / 8 FP64 lines, i.e. 64-byte row segments for the
// y and z passes) and the threads of their blocks (enough for one pass over all the tile's
// lines, at least one line's n / 8 and 32, at most 256).  Returns false (with *why) when a line
// is longer than a 256-thread block transforms or a tile does not fit in shared memory.
bool plan3(int nx, int ny, int nz, int nc, int elem_bytes, bool neumann, int smem_limit, Desc& d, const char** why);

}  // namespace rd
