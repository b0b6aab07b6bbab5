// The small-grid inner solve (rd_small.cuh) for single solves and batch slots, and its launchers.
#include "rd_small.cuh"
#include "rd_launch_small.h"

namespace rd {

template <int K>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  small_solve_body<K>(d, st, nullptr, smem_raw);
}

// one block per small slot of a batch: items[b] = (slot, 0)
template <int K>
__global__ void __launch_bounds__(kSmallThreads, 1)
    k_small_b(const Desc* __restrict__ descs, Slot* __restrict__ slots, const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (*((volatile const int*)&slots[w.x].phase) != PH_INNER) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  small_solve_body<K>(sd, &slots[w.x].inner, slots + w.x, smem_raw);
}

// the cluster form: kClusterCtas blocks per solve
template <int K>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kSmallThreads, 1)
    k_small_cl(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  small_cluster_body<K>(d, st, nullptr, smem_raw);
}

// one cluster per small slot of a batch: items[b] = (slot, 0), blocks 8 b .. 8 b + 7
template <int K>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kSmallThreads, 1)
    k_small_cl_b(const Desc* __restrict__ descs, Slot* __restrict__ slots, const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x / kClusterCtas];
  // every block of the cluster sees the same phase (it changes only inside the body, after the
  // body's first cluster barrier)
  if (*((volatile const int*)&slots[w.x].phase) != PH_INNER) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  small_cluster_body<K>(sd, &slots[w.x].inner, slots + w.x, smem_raw);
}

namespace {

template <class K_>
cudaError_t allow_k(K_ kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

int halo_of(int key) { return key == KK_CH_IMPL || key == KK_CH_SPLIT || key == KK_NONE_BIH ? 2 : 1; }

}  // namespace

int small_mode(int nx, int ny, int nc, int key, bool neumann, int usable) {
  if (nx >= 2 * kClusterCtas && ny >= 2 * kClusterCtas && nc * nx * ny <= 16384 &&
      cluster_smem_bytes(nx, ny, nc, halo_of(key), neumann) <= usable)
    return 2;
  if (nx >= 2 && ny >= 2 && nc * nx * ny <= 4096 && small_smem_bytes(nx, ny, nc, neumann) <= usable) return 1;
  return 0;
}

int small_smem_of(int mode, int nx, int ny, int nc, int key, bool neumann) {
  return mode == 2 ? cluster_smem_bytes(nx, ny, nc, halo_of(key), neumann) : small_smem_bytes(nx, ny, nc, neumann);
}

cudaError_t launch_small(const Desc& d, State* st, int mode, cudaStream_t s) {
  const int key = kind_key(d);
  const int sm = small_smem_of(mode, d.nx, d.ny, d.ncomp, key, d.bc == BC_NEUMANN);
  if (mode == 2) {
    switch (key) {
      case KK_NONE_LAP: k_small_cl<KK_NONE_LAP><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_AC: k_small_cl<KK_AC><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_CH_IMPL: k_small_cl<KK_CH_IMPL><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_CH_SPLIT: k_small_cl<KK_CH_SPLIT><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_GS: k_small_cl<KK_GS><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_SCHNAK: k_small_cl<KK_SCHNAK><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      case KK_NONE_BIH: k_small_cl<KK_NONE_BIH><<<kClusterCtas, kSmallThreads, sm, s>>>(d, st); break;
      default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
  }
  switch (key) {
    case KK_NONE_LAP: k_small<KK_NONE_LAP><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_AC: k_small<KK_AC><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_CH_IMPL: k_small<KK_CH_IMPL><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_CH_SPLIT: k_small<KK_CH_SPLIT><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_GS: k_small<KK_GS><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_SCHNAK: k_small<KK_SCHNAK><<<1, kSmallThreads, sm, s>>>(d, st); break;
    case KK_NONE_BIH: k_small<KK_NONE_BIH><<<1, kSmallThreads, sm, s>>>(d, st); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

cudaError_t launch_small_batch(int key, int mode, const Desc* descs, Slot* slots, const int2* items, int nitems,
                               int smem, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  if (mode == 2) {
    const int g = nitems * kClusterCtas;
    switch (key) {
      case KK_NONE_LAP: k_small_cl_b<KK_NONE_LAP><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_AC: k_small_cl_b<KK_AC><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_CH_IMPL: k_small_cl_b<KK_CH_IMPL><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_CH_SPLIT: k_small_cl_b<KK_CH_SPLIT><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_NONE_BIH: k_small_cl_b<KK_NONE_BIH><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_GS: k_small_cl_b<KK_GS><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      case KK_SCHNAK: k_small_cl_b<KK_SCHNAK><<<g, kSmallThreads, smem, s>>>(descs, slots, items); break;
      default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
  }
  switch (key) {
    case KK_NONE_LAP: k_small_b<KK_NONE_LAP><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_AC: k_small_b<KK_AC><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_CH_IMPL: k_small_b<KK_CH_IMPL><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_CH_SPLIT: k_small_b<KK_CH_SPLIT><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_NONE_BIH: k_small_b<KK_NONE_BIH><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_GS: k_small_b<KK_GS><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    case KK_SCHNAK: k_small_b<KK_SCHNAK><<<nitems, kSmallThreads, smem, s>>>(descs, slots, items); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

cudaError_t allow_small(int optin) {
  cudaError_t e;
  if ((e = allow_k(k_small<KK_NONE_LAP>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_AC>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_CH_IMPL>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_CH_SPLIT>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_GS>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_SCHNAK>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small<KK_NONE_BIH>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_NONE_LAP>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_AC>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_CH_IMPL>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_CH_SPLIT>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_NONE_BIH>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_NONE_LAP>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_AC>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_CH_IMPL>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_CH_SPLIT>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_GS>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_SCHNAK>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl<KK_NONE_BIH>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_NONE_LAP>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_AC>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_CH_IMPL>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_CH_SPLIT>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_NONE_BIH>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_GS>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_b<KK_SCHNAK>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k_small_cl_b<KK_GS>, optin)) != cudaSuccess) return e;
  return allow_k(k_small_cl_b<KK_SCHNAK>, optin);
}

}  // namespace rd
