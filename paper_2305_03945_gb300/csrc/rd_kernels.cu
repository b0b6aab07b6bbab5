// Step-level sm_103a kernels of the PDHG solver (arxiv 2305.03945, Section 2.1, Algorithm 1):
// the step set-up, the FP64 residual of defect correction, the FP64 update and the mass sum.
// The per-iteration sweeps live in rd_sweep.cuh (instantiated per equation group in rd_sweep_{f32,f64}_{lap,bih}.cu,
// rd_fused_{lap,bih}.cu and rd_sweep_col.cu).
//
// One PDHG iteration is three launches:
//   k_res  (row bands)      W = F(U_n) (eq. F(U) rd equation / F(U) CH / Section 3.4.1), the
//                           per-band partial sums of ||W_c||^2, the forward row transform of W
//                           along x, and (last block of the instance) the stopping decision
//                           ||Res(U_n)||_2 <= delta of Section 2.1;
//   k_col  (column blocks)  forward column transform along y, multiplication by 1/g_hat (the
//                           spectral inverse of G = A_lin^2), inverse column transform;
//   k_upd  (row bands)      inverse row transform of Y = G^{-1} W, the dual update
//                           P_{n+1} = P_n + tau_p Y, the extrapolation P~ = P_n + (1+omega) tau_p Y
//                           (eqs. G-prox ... dynamic 1-2) and the primal update
//                           U_{n+1} = U_n - tau_u dF(U_n)^T P~ (eq. G-prox ... dynamic 3).
// The transforms are the separable Hartley transform (periodic) and Makhoul's DCT-II (Neumann),
// both of which diagonalise the five-point Laplacian with its boundary rule.
#include <algorithm>
#include <cstdio>

#include "rd_sweep.cuh"

namespace rd {

// ---------------------------------------------------------------------------------------
// step set-up, FP64 residual (defect correction and the residual entry point), axpy, mass
// ---------------------------------------------------------------------------------------

// The step-level kernels below work on pairs of horizontally adjacent points (j even) of one row,
// in a grid-stride loop over a grid of one wave (resident blocks per SM x SMs, 256 threads):
// on this GPU every extra block costs scheduling time, so the grid is not sized by the data.
// Block partial sums go to d.partials[c * gridDim.x + block] and the last block reduces them in
// a fixed order.

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }

// rhs of the step from U^k, ||U^k||^2, and the solve state (n = 0, ACTIVE, threshold).
__global__ void __launch_bounds__(256) k_begin(const Desc* __restrict__ d64, State* __restrict__ st,
                                               const double* __restrict__ uk, double* __restrict__ rhs, double tol,
                                               int tol_kind) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const int lh = d.lognx - 1;
  double acc = 0.0;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (plane >> 1); g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g >> lh), j = 2 * (int)(g & (size_t)((nx >> 1) - 1));
    for (int c = 0; c < nc; ++c) {
      const size_t o = c * plane + (size_t)i * nx + j;
      const double2 u = ld2(uk + o);
      double2 v = u;
      switch (d.kind) {
        case RX_CH_SPLIT: {  // explicit part of the split: - (-b dt Lap U^k)
          const GField<double> f{uk + c * plane, nx, ny, bc};
          v.x = u.x - d.dt * d.b * lap5(f, i, j, u.x, d.hx2, d.hy2);
          v.y = u.y - d.dt * d.b * lap5(f, i, j + 1, u.y, d.hx2, d.hy2);
          break;
        }
        case RX_GS:
          if (c == 0) {
            v.x = u.x + d.dt * d.p[2];
            v.y = u.y + d.dt * d.p[2];
          }
          break;
        case RX_SCHNAK: {
          const double add = d.dt * d.p[2] * (c == 0 ? d.p[3] : d.p[4]);
          v.x = u.x + add;
          v.y = u.y + add;
          break;
        }
        default:
          break;
      }
      *reinterpret_cast<double2*>(rhs + o) = v;
      acc += u.x * u.x + u.y * u.y;
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[blockIdx.x] = s;
  if (last_block(st, gridDim.x)) {
    __threadfence();
    const double tot = sum_partials(d.partials, gridDim.x, red);
    if (threadIdx.x == 0) begin_state(st, tot, tol, tol_kind);
  }
}

// W = F(u) in FP64.  Optional outputs: w64 (FP64), r32 = (float)W and u32 = (float)u.  With
// `decide`, the kernel does nothing unless `outer` is active; its last block applies the outer
// stopping rule of defect correction to `outer` (evaluation number max_outer, counting from 0,
// ends the step as not converged) and otherwise arms the inner FP32 solve `inner` (threshold
// max(rtol * sum_c ||W_c||, half the outer threshold in the same units)).  zero32 (optional,
// two FP32 arrays) are cleared: the inner unknown d and the dual P_0.
template <int K>
__global__ void __launch_bounds__(256)
    k_resid64(const Desc* __restrict__ d64, State* __restrict__ outer, State* __restrict__ inner,
              const double* __restrict__ u, const double* __restrict__ rhs, double* __restrict__ w64,
              float* __restrict__ r32, float* __restrict__ u32, float* __restrict__ z0, float* __restrict__ z1,
              int decide, double rtol, int max_outer) {
  if (decide && *((volatile const int*)&outer->status) != ST_ACTIVE) return;
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const int lh = d.lognx - 1;
  const GField<double> f0{u, nx, ny, bc}, f1{u + plane, nx, ny, bc};
  double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 2
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (plane >> 1); g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g >> lh), j = 2 * (int)(g & (size_t)((nx >> 1) - 1));
    const size_t o = (size_t)i * nx + j;
    const double2 ra = ld2(rhs + o);
    const double2 rb = nc > 1 ? ld2(rhs + plane + o) : make_double2(0.0, 0.0);
    double wa[2] = {0.0, 0.0}, wb[2] = {0.0, 0.0};
    residual_pt<double, K, false>(d, f0, f1, f0, f1, i, j, ra.x, rb.x, wa);
    residual_pt<double, K, false>(d, f0, f1, f0, f1, i, j + 1, ra.y, rb.y, wb);
    for (int c = 0; c < nc; ++c) {
      const size_t oc = c * plane + o;
      if (w64) *reinterpret_cast<double2*>(w64 + oc) = make_double2(wa[c], wb[c]);
      if (r32) *reinterpret_cast<float2*>(r32 + oc) = make_float2((float)wa[c], (float)wb[c]);
      if (u32) {
        const double2 uu = ld2(u + oc);
        *reinterpret_cast<float2*>(u32 + oc) = make_float2((float)uu.x, (float)uu.y);
      }
      if (z0) *reinterpret_cast<float2*>(z0 + oc) = make_float2(0.f, 0.f);
      if (z1) *reinterpret_cast<float2*>(z1 + oc) = make_float2(0.f, 0.f);
    }
    acc0 += wa[0] * wa[0] + wb[0] * wb[0];
    acc1 += wa[1] * wa[1] + wb[1] * wb[1];
  }
  if (!decide) return;
  const int nb = gridDim.x;
  const double s0 = block_sum(acc0, red);
  const double s1 = nc > 1 ? block_sum(acc1, red) : 0.0;
  if (threadIdx.x == 0) {
    d.partials[blockIdx.x] = s0;
    if (nc > 1) d.partials[nb + blockIdx.x] = s1;
  }
  if (last_block(outer, nb)) {
    __threadfence();
    double tot = 0.0;
    for (int c = 0; c < nc; ++c) tot += sqrt(sum_partials(d.partials + c * nb, nb, red));
    if (threadIdx.x == 0) outer_decide(d, outer, inner, tot, rtol, max_outer);
  }
}

// Extra k_res launches a device-side loop may take beyond max_iter before it is stopped: covers
// the launches that find the solve already finished inside the last loop trip (<= 256 per trip).
constexpr unsigned kLoopSlack = 1024;

// Decision of a device-side loop (a WHILE node of the step's CUDA graph: the PDHG loop, or the
// outer rounds of defect correction), taken by one thread after the loop's first pass and at the
// end of every trip: adds `sweeps` (k_res launches, or 1 per round) to st->trips, and sets the
// loop condition to 0 when the solve is no longer active or, as a hard bound that holds
// whatever the stopping logic does, when the count exceeds max_iter + kLoopSlack, else to 1.
// Kept out of the sweep kernels, which thereby use no device-side graph API.
__global__ void k_loop_cond(State* __restrict__ st, cudaGraphConditionalHandle cond, unsigned sweeps) {
  volatile State* vs = st;
  const unsigned t = vs->trips + sweeps;
  vs->trips = t;
  // set on every call (not only cleared): a loop nested in another loop's body starts each trip of
  // the outer loop with the condition this call leaves
  cudaGraphSetConditional(cond, (vs->status != ST_ACTIVE || t > (unsigned)vs->max_iter + kLoopSlack) ? 0u : 1u);
}

// u += d after an inner solve of defect correction, when `outer` is active and the inner solve
// ended converged (or stalled at its rounding floor) or at its iteration limit; an inner solve
// that diverged, or that is still active, ends the step as diverged.  Adds the inner solve's
// updates and k_res launches to the outer state's totals.  n is a multiple of 4.
__global__ void k_axpy_dc(double* __restrict__ u, const float* __restrict__ dlt, size_t n, State* __restrict__ outer,
                          const State* __restrict__ inner) {
  if (*((volatile const int*)&outer->status) != ST_ACTIVE) return;
  const int is = *((volatile const int*)&inner->status);
  const bool ok = is == ST_CONVERGED || is == ST_NOT_CONVERGED;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    outer->total += inner->n;
    outer->launches += (int)inner->trips;
    if (!ok) outer->status = ST_DIVERGED;
  }
  if (!ok) return;
  const size_t n4 = n >> 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 dv = reinterpret_cast<const float4*>(dlt)[i];
    double2 a = reinterpret_cast<double2*>(u)[2 * i];
    double2 b = reinterpret_cast<double2*>(u)[2 * i + 1];
    a.x += (double)dv.x;
    a.y += (double)dv.y;
    b.x += (double)dv.z;
    b.y += (double)dv.w;
    reinterpret_cast<double2*>(u)[2 * i] = a;
    reinterpret_cast<double2*>(u)[2 * i + 1] = b;
  }
}

// h_x h_y (h_z) sum of u into st->mass; with `gate`, only once `gate` is no longer active.
__global__ void __launch_bounds__(256) k_mass(const Desc* __restrict__ d64, State* __restrict__ st,
                                              const double* __restrict__ u, const State* __restrict__ gate) {
  if (gate && *((volatile const int*)&gate->status) == ST_ACTIVE) return;
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nc = d.ncomp;
  const size_t plane = (size_t)d.nx * d.ny * (d.nz > 1 ? d.nz : 1);  // points per component
  double acc = 0.0;
#pragma unroll 4
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (plane >> 1); g += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) {
      const double2 v = ld2(u + c * plane + 2 * g);
      acc += v.x + v.y;
    }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[blockIdx.x] = s;
  if (last_block(st, gridDim.x)) {
    __threadfence();
    const double tot = sum_partials(d.partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->ticket = 0u;
      st->mass = tot / (sqrt(d.hx2) * sqrt(d.hy2) * (d.nz > 1 ? sqrt(d.hz2) : 1.0));
    }
  }
}

// ---------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------

// One wave of `kernel` at 256 threads (resident blocks per SM x SMs), at most `nblocks`.
template <class F>
static int wave_blocks(F kernel, int nblocks) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess)
    return nblocks;
  const int wave = std::max(1, occ) * std::max(1, sms);
  return std::max(1, std::min(nblocks, wave));
}

cudaError_t launch_begin(const Desc* d64, State* st, const double* uk, double* rhs, double tol, int tol_kind,
                         int nblocks, cudaStream_t s) {
  k_begin<<<wave_blocks(k_begin, nblocks), 256, 0, s>>>(d64, st, uk, rhs, tol, tol_kind);
  return cudaGetLastError();
}

cudaError_t launch_resid64(const Desc& hd, const Desc* d64, State* outer, State* inner, const double* u,
                           const double* rhs, double* w64, float* r32, float* u32, float* z0, float* z1, int decide,
                           double rtol, int max_outer, int nblocks, cudaStream_t s) {
  switch (kind_key(hd)) {
    case KK_AC: k_resid64<KK_AC><<<wave_blocks(k_resid64<KK_AC>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_CH_IMPL: k_resid64<KK_CH_IMPL><<<wave_blocks(k_resid64<KK_CH_IMPL>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_CH_SPLIT: k_resid64<KK_CH_SPLIT><<<wave_blocks(k_resid64<KK_CH_SPLIT>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_GS: k_resid64<KK_GS><<<wave_blocks(k_resid64<KK_GS>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_SCHNAK: k_resid64<KK_SCHNAK><<<wave_blocks(k_resid64<KK_SCHNAK>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_NONE_BIH: k_resid64<KK_NONE_BIH><<<wave_blocks(k_resid64<KK_NONE_BIH>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    default: k_resid64<KK_NONE_LAP><<<wave_blocks(k_resid64<KK_NONE_LAP>, nblocks), 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_axpy_dc(double* u, const float* dlt, size_t n, State* outer, const State* inner, cudaStream_t s) {
  k_axpy_dc<<<wave_blocks(k_axpy_dc, (int)((n / 4 + 255) / 256)), 256, 0, s>>>(u, dlt, n, outer, inner);
  return cudaGetLastError();
}

cudaError_t launch_loop_cond(State* st, unsigned long long cond, unsigned sweeps, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(st, (cudaGraphConditionalHandle)cond, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_mass(const Desc* d64, State* st, const double* u, const State* gate, int nblocks, cudaStream_t s) {
  k_mass<<<wave_blocks(k_mass, nblocks), 256, 0, s>>>(d64, st, u, gate);
  return cudaGetLastError();
}

}  // namespace rd
