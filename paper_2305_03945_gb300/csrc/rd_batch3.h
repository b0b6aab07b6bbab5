// Launch interface of the batched 3-D kernels (rd_batch3.cu).
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

// One iteration of the 3-D slots of one equation key (axpy, step phases, residual, the five
// transform passes, update) over the work list items[0..nitems) of (slot, block) pairs; thr[a]
// and smem[a] are the block size and dynamic shared memory of the transform passes of axis a,
// the largest any slot in the list needs.
struct Batch3Launch {
  const Desc* d32s;
  const Desc* d64s;
  Slot* slots;
  const int2* items;
  int nitems;
  int thr[3];
  int smem[3];
};

cudaError_t batch3_launch_group(int key, const Batch3Launch& L, cudaStream_t s);
// Raise the dynamic shared-memory limit of the batched 3-D transform passes.
cudaError_t batch3_allow(int optin);

}  // namespace rd
