// Host-side launchers of the small-grid inner solve (rd_small.cu).
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

// How the whole FP32 inner solve of an nx x ny grid with nc components (equation key `key`) runs
// within `usable` bytes of shared memory per block: 2 = on a cluster of 8 blocks (sides >= 16,
// at most 16 K points), 1 = in one block (at most 4 K points), 0 = not at all (the multi-kernel
// sweeps).
int small_mode(int nx, int ny, int nc, int key, bool neumann, int usable);
int small_smem_of(int mode, int nx, int ny, int nc, int key, bool neumann);
// The inner solve of the FP32 descriptor d on the solve state st, to its end, in one launch.
cudaError_t launch_small(const Desc& d, State* st, int mode, cudaStream_t s);
// One block (mode 1) or one cluster (mode 2) per batch slot of equation key `key` in items
// (slot, 0); smem = the largest slot's bytes.
cudaError_t launch_small_batch(int key, int mode, const Desc* descs, Slot* slots, const int2* items, int nitems,
                               int smem, cudaStream_t s);
// Raise the dynamic shared-memory limit of the small-solve kernels.
cudaError_t allow_small(int optin);

}  // namespace rd
