// Step-level sm_103a kernels of the PDHG solver (arxiv 2305.03945, Section 2.1, Algorithm 1):
// the step set-up, the FP64 residual of defect correction, the FP64 update and the mass sum.
// The per-iteration sweeps live in rd_sweep.cuh (instantiated in rd_sweep_f32.cu / _f64.cu).
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
#include <cstdio>

#include "rd_sweep.cuh"

namespace rd {

// ---------------------------------------------------------------------------------------
// step set-up, FP64 residual (defect correction and the residual entry point), axpy, mass
// ---------------------------------------------------------------------------------------

// rhs of the step from U^k, ||U^k||^2, and the solve state (n = 0, ACTIVE, threshold).
__global__ void k_begin(const Desc* __restrict__ d64, State* __restrict__ st, const double* __restrict__ uk,
                        double* __restrict__ rhs, double tol, int tol_kind) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const int band = blockIdx.x;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < nc * rows * nx; idx += blockDim.x) {
    const int c = idx / (rows * nx);
    const int rem = idx - c * rows * nx;
    const int r = rem / nx, j = rem - r * nx;
    const int i = y0 + r;
    const size_t o = c * plane + (size_t)i * nx + j;
    const double u = uk[o];
    double v = u;
    switch (d.kind) {
      case RX_CH_SPLIT: {  // explicit part of the split: - (-b dt Lap U^k)
        const GField<double> f{uk, nx, ny, bc};
        v = u - d.dt * d.b * lap5(f, i, j, u, d.hx2, d.hy2);
        break;
      }
      case RX_GS:
        if (c == 0) v = u + d.dt * d.p[2];
        break;
      case RX_SCHNAK:
        v = u + d.dt * d.p[2] * (c == 0 ? d.p[3] : d.p[4]);
        break;
      default:
        break;
    }
    rhs[o] = v;
    acc += u * u;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[band] = s;
  if (last_block(st, d.nbands)) {
    __threadfence();
    const double tot = sum_partials(d.partials, d.nbands, red);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(tot);
      st->ticket = 0u;
      st->aux = nrm;
      st->thresh = tol_kind == 1 ? tol * nrm : tol;
      st->n = 0;
      st->r = 0.0;
      st->r0 = 0.0;
      st->status = ST_ACTIVE;
    }
  }
}

// W = F(u) in FP64.  Optional outputs: w64 (FP64), r32 = (float)W and u32 = (float)u.  With
// `decide`, the last block applies the outer stopping rule of defect correction to `outer` and
// arms the inner FP32 solve `inner` (threshold rtol * sum_c ||W_c||).  zero32 (optional, two
// FP32 arrays) are cleared: the inner unknown d and the dual P_0.
template <int K>
__global__ void k_resid64(const Desc* __restrict__ d64, State* __restrict__ outer, State* __restrict__ inner,
                          const double* __restrict__ u, const double* __restrict__ rhs,
                          double* __restrict__ w64, float* __restrict__ r32, float* __restrict__ u32,
                          float* __restrict__ z0, float* __restrict__ z1, int decide, double rtol) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const int band = blockIdx.x;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  const GField<double> f0{u, nx, ny, bc}, f1{u + plane, nx, ny, bc};
  double acc0 = 0.0, acc1 = 0.0;
  for (int idx = threadIdx.x; idx < rows * nx; idx += blockDim.x) {
    const int r = idx / nx, j = idx - r * nx;
    const int i = y0 + r;
    const size_t o = (size_t)i * nx + j;
    double w[2] = {0.0, 0.0};
    residual_pt<double, K, false>(d, f0, f1, f0, f1, i, j, rhs[o], nc > 1 ? rhs[plane + o] : 0.0, w);
    for (int c = 0; c < nc; ++c) {
      const size_t oc = c * plane + o;
      if (w64) w64[oc] = w[c];
      if (r32) r32[oc] = (float)w[c];
      if (u32) u32[oc] = (float)u[oc];
      if (z0) z0[oc] = 0.f;
      if (z1) z1[oc] = 0.f;
    }
    acc0 += w[0] * w[0];
    acc1 += w[1] * w[1];
  }
  if (!decide) return;
  const double s0 = block_sum(acc0, red);
  const double s1 = nc > 1 ? block_sum(acc1, red) : 0.0;
  if (threadIdx.x == 0) {
    d.partials[band] = s0;
    if (nc > 1) d.partials[d.nbands + band] = s1;
  }
  if (last_block(outer, d.nbands)) {
    __threadfence();
    double tot = 0.0;
    for (int c = 0; c < nc; ++c) tot += sqrt(sum_partials(d.partials + c * d.nbands, d.nbands, red));
    if (threadIdx.x == 0) {
      const double meas = d.meas_div_dt ? tot / d.dt : tot;
      outer->ticket = 0u;
      outer->r = meas;
      const int n = outer->n;
      if (n == 0) outer->r0 = meas;
      const double r0 = n == 0 ? meas : outer->r0;
      outer->n = n + 1;
      if (meas <= outer->thresh) {
        outer->status = ST_CONVERGED;
      } else if (!isfinite(meas) || meas > kDivergeFactor * r0) {
        outer->status = ST_DIVERGED;
      } else {
        inner->n = 0;
        inner->r = 0.0;
        inner->r0 = 0.0;
        inner->thresh = rtol * tot;
        inner->status = ST_ACTIVE;
        inner->ticket = 0u;
      }
    }
  }
}

__global__ void k_axpy_dc(double* __restrict__ u, const float* __restrict__ dlt, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    u[i] += (double)dlt[i];
}

__global__ void k_mass(const Desc* __restrict__ d64, State* __restrict__ st, const double* __restrict__ u) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp;
  const size_t plane = (size_t)nx * ny;
  const int band = blockIdx.x;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < nc * rows * nx; idx += blockDim.x) {
    const int c = idx / (rows * nx);
    const int rem = idx - c * rows * nx;
    acc += u[c * plane + (size_t)y0 * nx + rem];
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[band] = s;
  if (last_block(st, d.nbands)) {
    __threadfence();
    const double tot = sum_partials(d.partials, d.nbands, red);
    if (threadIdx.x == 0) {
      st->ticket = 0u;
      st->mass = tot / (sqrt(d.hx2) * sqrt(d.hy2));
    }
  }
}

// ---------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------

cudaError_t launch_begin(const Desc* d64, State* st, const double* uk, double* rhs, double tol, int tol_kind,
                         int nbands, cudaStream_t s) {
  k_begin<<<nbands, 256, 0, s>>>(d64, st, uk, rhs, tol, tol_kind);
  return cudaGetLastError();
}

cudaError_t launch_resid64(const Desc& hd, const Desc* d64, State* outer, State* inner, const double* u,
                           const double* rhs, double* w64, float* r32, float* u32, float* z0, float* z1, int decide,
                           double rtol, int nbands, cudaStream_t s) {
  switch (kind_key(hd)) {
    case KK_AC: k_resid64<KK_AC><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    case KK_CH_IMPL: k_resid64<KK_CH_IMPL><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    case KK_CH_SPLIT: k_resid64<KK_CH_SPLIT><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    case KK_GS: k_resid64<KK_GS><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    case KK_SCHNAK: k_resid64<KK_SCHNAK><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    case KK_NONE_BIH: k_resid64<KK_NONE_BIH><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
    default: k_resid64<KK_NONE_LAP><<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_axpy_dc(double* u, const float* dlt, size_t n, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_axpy_dc<<<blocks, 256, 0, s>>>(u, dlt, n);
  return cudaGetLastError();
}

cudaError_t launch_mass(const Desc* d64, State* st, const double* u, int nbands, cudaStream_t s) {
  k_mass<<<nbands, 256, 0, s>>>(d64, st, u);
  return cudaGetLastError();
}

}  // namespace rd
