// The sixth-order functionalized Cahn-Hilliard step (arxiv 2305.03945, Section 3.3) in FP64:
//
//   mu(U) = a Lap U - b W'(U),   A(U) = a Lap - b diag(W''(U)) + a I,   B(U) = a Lap - b diag(W''(U))
//   F(U)  = U - U^k - dt Lap A(U) mu(U)
//   dF(U)^T P = P - dt B(U) A(U) Lap P + dt b mu(U) W'''(U) Lap P
//
// with W(u) = (u^2 - 1)^2 / 4 (W' = u^3 - u, W'' = 3u^2 - 1, W''' = 6u).  F nests three
// five-point Laplacians and the adjoint three more, each with pointwise nonlinear factors in
// between, so one PDHG iteration is a chain of simple stencil passes over whole grids (which
// at the paper's 128^2 stay in L2), with the preconditioner solve of the other equations in the
// middle (the preconditioner-only k_res / k_col / k_upd with the symbol
// g = (1 + dt a mu^2 (a mu + 2b - a))^2 of G = (I - dt Lap (a Lap - (2b - a) I) a Lap)^2):
//
//   k_fch_mu    M = mu(U)                           (skips once the solve has stopped)
//   k_fch_nu    N = A(U) M
//   k_fch_w     W = U - U^k - dt Lap N, ||W||^2 partials; last block: the stopping decision
//   [k_res, k_col, k_upd in preconditioner-only mode: W <- G^{-1} W]
//   k_fch_dual  P~ = P + (1 + omega) tau_p Y,  P += tau_p Y      (pointwise, in place on P)
//   k_fch_q     Q = Lap P~
//   k_fch_r     N = A(U) Q
//   k_fch_upd   U -= tau_u (P~ - dt B(U) N + dt b M W'''(U) Q)   (pointwise in U: in place)
//
// Every kernel runs one wave of 256-thread blocks over a grid-stride loop, one point per step.
#include <algorithm>

#include "rd_sweep.cuh"

namespace rd {

namespace {

__device__ __forceinline__ bool fch_active(const State* st) {
  return st == nullptr || *((volatile const int*)&st->status) == ST_ACTIVE;
}

struct FchPt {
  int i, j;
  size_t o;
};

template <class Body>
__device__ __forceinline__ void fch_points(const Desc& d, Body body) {
  const size_t np = (size_t)d.nx * d.ny;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < np; g += (size_t)gridDim.x * blockDim.x)
    body(FchPt{(int)(g >> d.lognx), (int)(g & (size_t)(d.nx - 1)), g});
}

__global__ void __launch_bounds__(256) k_fch_mu(const __grid_constant__ Desc d, const State* st,
                                                const double* __restrict__ U, double* __restrict__ M) {
  if (!fch_active(st)) return;
  const GField<double> u{U, d.nx, d.ny, d.bc};
  fch_points(d, [&](FchPt p) {
    const double c = U[p.o];
    M[p.o] = d.a * lap5(u, p.i, p.j, c, d.hx2, d.hy2) - d.b * (c * c * c - c);
  });
}

// N = A(U) X = a Lap X - b W''(U) X + a X
__global__ void __launch_bounds__(256) k_fch_apply_a(const __grid_constant__ Desc d, const State* st,
                                                     const double* __restrict__ U, const double* __restrict__ X,
                                                     double* __restrict__ N) {
  if (!fch_active(st)) return;
  const GField<double> x{X, d.nx, d.ny, d.bc};
  fch_points(d, [&](FchPt p) {
    const double c = X[p.o], u = U[p.o];
    N[p.o] = d.a * lap5(x, p.i, p.j, c, d.hx2, d.hy2) - d.b * (3.0 * u * u - 1.0) * c + d.a * c;
  });
}

// W = U - U^k - dt Lap N; with st, the block partials of ||W||^2 and the stopping decision.
__global__ void __launch_bounds__(256) k_fch_w(const __grid_constant__ Desc d, State* st, const double* __restrict__ U,
                                               const double* __restrict__ Uk, const double* __restrict__ N,
                                               double* __restrict__ W) {
  __shared__ double red[32];
  if (!fch_active(st)) return;
  const GField<double> n{N, d.nx, d.ny, d.bc};
  double acc = 0.0;
  fch_points(d, [&](FchPt p) {
    const double w = U[p.o] - Uk[p.o] - d.dt * lap5(n, p.i, p.j, N[p.o], d.hx2, d.hy2);
    W[p.o] = w;
    acc += w * w;
  });
  if (st == nullptr) return;
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[blockIdx.x] = s;
  if (last_block(st, gridDim.x)) finalize_measure(d, st, red, nullptr, gridDim.x);
}

// P~ = P + (1 + omega) tau_p Y, P <- P + tau_p Y
__global__ void __launch_bounds__(256) k_fch_dual(const __grid_constant__ Desc d, const State* st,
                                                  const double* __restrict__ Y, double* __restrict__ P,
                                                  double* __restrict__ Pt) {
  if (!fch_active(st)) return;
  const double tp = d.tau_p, tpe = (1.0 + d.omega) * d.tau_p;
  fch_points(d, [&](FchPt p) {
    const double y = Y[p.o], pn = P[p.o];
    Pt[p.o] = pn + tpe * y;
    P[p.o] = pn + tp * y;
  });
}

__global__ void __launch_bounds__(256) k_fch_lap(const __grid_constant__ Desc d, const State* st,
                                                 const double* __restrict__ X, double* __restrict__ Q) {
  if (!fch_active(st)) return;
  const GField<double> x{X, d.nx, d.ny, d.bc};
  fch_points(d, [&](FchPt p) { Q[p.o] = lap5(x, p.i, p.j, X[p.o], d.hx2, d.hy2); });
}

// U -= tau_u (P~ - dt B(U) R + dt b mu W'''(U) Q), B(U) R = a Lap R - b W''(U) R
__global__ void __launch_bounds__(256) k_fch_upd(const __grid_constant__ Desc d, const State* st,
                                                 double* __restrict__ U, const double* __restrict__ M,
                                                 const double* __restrict__ Q, const double* __restrict__ R,
                                                 const double* __restrict__ Pt) {
  if (!fch_active(st)) return;
  const GField<double> r{R, d.nx, d.ny, d.bc};
  fch_points(d, [&](FchPt p) {
    const double u = U[p.o], rc = R[p.o];
    const double s = d.a * lap5(r, p.i, p.j, rc, d.hx2, d.hy2) - d.b * (3.0 * u * u - 1.0) * rc;
    const double g = Pt[p.o] - d.dt * s + d.dt * d.b * M[p.o] * (6.0 * u) * Q[p.o];
    U[p.o] = u - d.tau_u * g;
  });
}

template <class F>
int fch_grid(F kernel, size_t npts) {
  int dev = 0, sms = 0, occ = 0;
  const int want = (int)std::min<size_t>((npts + 255) / 256, (size_t)1 << 20);
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess)
    return std::max(1, want);
  return std::max(1, std::min(want, std::max(1, occ) * std::max(1, sms)));
}

}  // namespace

cudaError_t launch_fch_residual(const Desc& d, State* st, const FchBuffers& b, const double* U, const double* Uk,
                                double* W, int max_blocks, cudaStream_t s) {
  const size_t np = (size_t)d.nx * d.ny;
  k_fch_mu<<<fch_grid(k_fch_mu, np), 256, 0, s>>>(d, st, U, b.M);
  k_fch_apply_a<<<fch_grid(k_fch_apply_a, np), 256, 0, s>>>(d, st, U, b.M, b.N);
  k_fch_w<<<std::min(max_blocks, fch_grid(k_fch_w, np)), 256, 0, s>>>(d, st, U, Uk, b.N, W);
  return cudaGetLastError();
}

cudaError_t launch_fch_iteration(const Desc& d, const Desc& dpc, State* st, State* st_pc, const LaunchCfg& cpc,
                                 const FchBuffers& b, int max_blocks, cudaStream_t s, cudaEvent_t* ev) {
  unsigned flags;
  cudaError_t e = record_flags(s, ev, &flags);
  if (e != cudaSuccess) return e;
  auto mark = [&](int i) {
    if (ev && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[i], s, flags);
  };
  const size_t np = (size_t)d.nx * d.ny;
  double* U = static_cast<double*>(d.X);
  const double* Uk = static_cast<const double*>(d.rhs);
  double* P = static_cast<double*>(d.P[0]);
  double* W = static_cast<double*>(dpc.X);  // F(U), then G^{-1} F(U) in place
  mark(0);
  if (e == cudaSuccess) e = launch_fch_residual(d, st, b, U, Uk, W, max_blocks, s);
  mark(1);
  if (e == cudaSuccess && d.precond != 0) e = launch_iteration<double>(dpc, st_pc, cpc, s, nullptr);
  mark(2);
  k_fch_dual<<<fch_grid(k_fch_dual, np), 256, 0, s>>>(d, st, W, P, b.Pt);
  k_fch_lap<<<fch_grid(k_fch_lap, np), 256, 0, s>>>(d, st, b.Pt, b.Q);
  k_fch_apply_a<<<fch_grid(k_fch_apply_a, np), 256, 0, s>>>(d, st, U, b.Q, b.N);
  k_fch_upd<<<fch_grid(k_fch_upd, np), 256, 0, s>>>(d, st, U, b.M, b.Q, b.N, b.Pt);
  mark(3);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace rd
