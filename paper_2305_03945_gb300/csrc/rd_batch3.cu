// Batched kernels of 3-D requests (rd_batch_*): the 3-D PDHG iteration of rd_3d.cuh and the
// device-side phase machine of a batch slot (step set-up, FP64 residual and outer decision of
// defect correction, u += d), over work lists of (slot, block) pairs.  Every 3-D slot runs its
// descriptor's blk3 blocks in every kernel, whatever else shares the launch.
#include "rd_3d.cuh"
#include "rd_batch3.h"

namespace rd {

namespace {

__device__ __forceinline__ bool slot_in(const Slot* sl, int ph) { return *((volatile const int*)&sl->phase) == ph; }

template <int K>
__global__ void __launch_bounds__(256) k3_res_b(const Desc* __restrict__ descs, Slot* __restrict__ slots,
                                                const int2* __restrict__ items) {
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (!slot_in(slots + w.x, PH_INNER)) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  res3_body<float, K>(sd, &slots[w.x].inner, slots + w.x, w.y);
}

template <int K>
__global__ void __launch_bounds__(256) k3_upd_b(const Desc* __restrict__ descs, Slot* __restrict__ slots,
                                                const int2* __restrict__ items) {
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (!slot_in(slots + w.x, PH_INNER)) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  upd3_body<float, K>(sd, &slots[w.x].inner, slots + w.x, w.y);
}

template <int AX, int MODE>
__global__ void __launch_bounds__(256) k3_lines_b(const Desc* __restrict__ descs, Slot* __restrict__ slots,
                                                  const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (!slot_in(slots + w.x, PH_INNER)) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  lines3_body<float, AX, MODE>(sd, &slots[w.x].inner, slots + w.x, w.y, smem_raw);
}

// PH_BEGIN: rhs of the step from U^k (the explicit part of the convex split), ||U^k||, the outer
//           threshold -> PH_RESID.
// PH_RESID: r = F(u) in FP64; r and u rounded to FP32; d = 0, P_0 = 0; outer stopping rule ->
//           next step / DONE / FAILED, or arm the inner FP32 solve -> PH_INNER.
template <int K>
__global__ void __launch_bounds__(256) k3_step_b(const Desc* __restrict__ d64s, Slot* __restrict__ slots,
                                                 const int2* __restrict__ items) {
  __shared__ Desc sd;
  __shared__ double red[32];
  const int2 w = items[blockIdx.x];
  Slot* sl = slots + w.x;
  const int ph = *((volatile const int*)&sl->phase);
  if (ph != PH_BEGIN && ph != PH_RESID) return;
  load_desc(sd, d64s + w.x);
  __syncthreads();
  const Desc& d = sd;
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const int b = w.y, nb = d.blk3;
  double* u = static_cast<double*>(d.X);
  double* rhs = static_cast<double*>(const_cast<void*>(d.rhs));
  const G3<double> f{u, d.nx, d.ny, d.nz, d.bc};
  State* outer = &sl->outer;
  double acc = 0.0;
  if (ph == PH_BEGIN) {
    for (size_t q = (size_t)b * blockDim.x + threadIdx.x; q < N; q += (size_t)nb * blockDim.x) {
      const double uv = u[q];
      double v = uv;
      if constexpr (K == KK_CH_SPLIT) {
        int l, i, j;
        point3(d, q, l, i, j);
        v = uv - d.dt * d.b * lap7(f, l, i, j, uv, d.hx2, d.hy2, d.hz2);
      }
      rhs[q] = v;
      acc += uv * uv;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) d.partials[b] = s;
    if (last_block(outer, nb)) {
      __threadfence();
      const double tot = sum_partials(d.partials, nb, red);
      if (threadIdx.x == 0) {
        outer->ticket = 0u;
        outer->aux = sqrt(tot);
        outer->thresh = sl->tol_kind == 1 ? sl->tol * sqrt(tot) : sl->tol;
        outer->n = 0;
        outer->r = 0.0;
        outer->r0 = 0.0;
        outer->status = ST_ACTIVE;
        sl->phase = PH_RESID;
      }
    }
    return;
  }
  for (size_t q = (size_t)b * blockDim.x + threadIdx.x; q < N; q += (size_t)nb * blockDim.x) {
    int l, i, j;
    point3(d, q, l, i, j);
    const double wv = residual3_pt<double, K, false>(d, f, f, l, i, j, rhs[q]);
    d.f32_r[q] = (float)wv;
    d.f32_u[q] = (float)u[q];
    d.f32_d[q] = 0.f;
    d.f32_p0[q] = 0.f;
    acc += wv * wv;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[b] = s;
  if (last_block(outer, nb)) {
    __threadfence();
    const double tot = sqrt(sum_partials(d.partials, nb, red));
    if (threadIdx.x == 0) {
      const double meas = d.meas_div_dt ? tot / d.dt : tot;
      const double prev = outer->r;
      outer->ticket = 0u;
      outer->r = meas;
      const int n = outer->n;
      if (n == 0) outer->r0 = meas;
      const double r0 = n == 0 ? meas : outer->r0;
      outer->n = n + 1;
      sl->outer_total += 1;
      if (meas <= outer->thresh) {
        outer->status = ST_CONVERGED;
        sl->steps_done += 1;
        sl->phase = sl->steps_done >= sl->nsteps ? PH_DONE : PH_BEGIN;
      } else if (!isfinite(meas) || meas > kDivergeFactor * r0 || outer->n > sl->max_outer) {
        outer->status = isfinite(meas) && meas <= kDivergeFactor * r0 ? ST_NOT_CONVERGED : ST_DIVERGED;
        sl->phase = PH_FAILED;
      } else {
        State* in = &sl->inner;
        in->stall_mul = next_stall_mul(n, meas, prev, in->stall_mul);
        in->n = 0;
        in->r = 0.0;
        in->r0 = 0.0;
        in->thresh = fmax(sl->rtol * tot, 0.5 * outer->thresh * (d.meas_div_dt ? d.dt : 1.0));
        in->status = ST_ACTIVE;
        in->ticket = 0u;
        sl->phase = PH_INNER;
      }
    }
  }
}

// PH_AXPY: u += d (FP64 += FP32) -> PH_RESID.
__global__ void __launch_bounds__(256) k3_axpy_b(const Desc* __restrict__ d64s, Slot* __restrict__ slots,
                                                 const int2* __restrict__ items) {
  const int2 w = items[blockIdx.x];
  Slot* sl = slots + w.x;
  if (!slot_in(sl, PH_AXPY)) return;
  const Desc& d = d64s[w.x];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const int nb = d.blk3;
  double* u = static_cast<double*>(d.X);
  const float* dl = d.f32_d;
  for (size_t q = (size_t)w.y * blockDim.x + threadIdx.x; q < N; q += (size_t)nb * blockDim.x) u[q] += (double)dl[q];
  if (last_block(&sl->outer, nb) && threadIdx.x == 0) {
    sl->outer.ticket = 0u;
    sl->phase = PH_RESID;
  }
}

template <class K_>
cudaError_t allow_k(K_ kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <int K>
void group3(const Batch3Launch& L, cudaStream_t s) {
  const int n = L.nitems;
  k3_axpy_b<<<n, 256, 0, s>>>(L.d64s, L.slots, L.items);
  k3_step_b<K><<<n, 256, 0, s>>>(L.d64s, L.slots, L.items);
  k3_res_b<K><<<n, 256, 0, s>>>(L.d32s, L.slots, L.items);
  k3_lines_b<0, L3_FWD><<<n, L.thr[0], L.smem[0], s>>>(L.d32s, L.slots, L.items);
  k3_lines_b<1, L3_FWD><<<n, L.thr[1], L.smem[1], s>>>(L.d32s, L.slots, L.items);
  k3_lines_b<2, L3_FSI><<<n, L.thr[2], L.smem[2], s>>>(L.d32s, L.slots, L.items);
  k3_lines_b<1, L3_INV><<<n, L.thr[1], L.smem[1], s>>>(L.d32s, L.slots, L.items);
  k3_lines_b<0, L3_INVP><<<n, L.thr[0], L.smem[0], s>>>(L.d32s, L.slots, L.items);
  k3_upd_b<K><<<n, 256, 0, s>>>(L.d32s, L.slots, L.items);
}

}  // namespace

cudaError_t batch3_launch_group(int key, const Batch3Launch& L, cudaStream_t s) {
  if (L.nitems == 0) return cudaSuccess;
  switch (key) {
    case KK_NONE_LAP: group3<KK_NONE_LAP>(L, s); break;
    case KK_AC: group3<KK_AC>(L, s); break;
    case KK_CH_IMPL: group3<KK_CH_IMPL>(L, s); break;
    case KK_CH_SPLIT: group3<KK_CH_SPLIT>(L, s); break;
    case KK_NONE_BIH: group3<KK_NONE_BIH>(L, s); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

cudaError_t batch3_allow(int optin) {
  cudaError_t e;
  if ((e = allow_k(k3_lines_b<0, L3_FWD>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k3_lines_b<1, L3_FWD>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k3_lines_b<2, L3_FSI>, optin)) != cudaSuccess) return e;
  if ((e = allow_k(k3_lines_b<1, L3_INV>, optin)) != cudaSuccess) return e;
  return allow_k(k3_lines_b<0, L3_INVP>, optin);
}

}  // namespace rd
