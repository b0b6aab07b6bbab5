// sm_103a kernels of the G-prox PDHG iteration (arxiv 2305.03945, Section 2.1, Algorithm 1).
//
// One PDHG iteration is three launches over every active instance:
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

#include "rd_device.cuh"
#include "rd_launch.h"

namespace rd {

// ---------------------------------------------------------------------------------------
// pointwise physics
// ---------------------------------------------------------------------------------------

// W_c = F_c(X) at (i, j) for every component.
//   plain (dc = 0): X = U, R = rhs of the step (U^k plus the explicit / constant terms)
//   dc    (dc = 1): X = d, B = u, R = F(u); returns F(u + d) = F(u) + A_lin d + N(u + d) - N(u)
//                   with the nonlinear increment expanded so no large terms cancel.
template <class T>
__device__ __forceinline__ void residual_at(const Desc& d, const T* __restrict__ X,
                                            const T* __restrict__ B, const T* __restrict__ R,
                                            int i, int j, T* w) {
  const int nx = d.nx, ny = d.ny, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const size_t o = (size_t)i * nx + j;
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const GField<T> f0{X, nx, ny, bc};
  const T c0 = X[o];
  const T r0 = R[o];
  switch (d.kind) {
    case RX_NONE: {
      const T lin = d.op == OP_LAP ? c0 - dt * a * lap5(f0, i, j, c0, hx2, hy2)
                                   : c0 + dt * a * lap13(f0, i, j, c0, hx2, hy2);
      w[0] = d.dc ? r0 + lin : lin - r0;
      break;
    }
    case RX_AC: {
      const T lin = c0 - dt * a * lap5(f0, i, j, c0, hx2, hy2);
      if (!d.dc) {
        w[0] = lin - r0 + dt * b * (c0 * c0 * c0 - c0);
      } else {
        const T u = B[o];
        w[0] = r0 + lin + dt * b * (c0 * (T(3) * u * u - T(1)) + c0 * c0 * (T(3) * u + c0));
      }
      break;
    }
    case RX_CH_IMPL:
    case RX_CH_SPLIT: {
      const T lin = c0 + dt * a * lap13(f0, i, j, c0, hx2, hy2);
      const T sh = d.kind == RX_CH_IMPL ? T(1) : T(0);
      const int dcm = d.dc;
      auto q = [&](int ii, int jj) -> T {
        const size_t oo = (size_t)bcmap(ii, ny, bc) * nx + bcmap(jj, nx, bc);
        const T xv = X[oo];
        if (!dcm) return xv * xv * xv - sh * xv;
        const T u = B[oo];
        return xv * (T(3) * u * u - sh) + xv * xv * (T(3) * u + xv);
      };
      const T qc = q(i, j);
      const T lq = (q(i, j + 1) + q(i, j - 1) - T(2) * qc) * hx2 + (q(i + 1, j) + q(i - 1, j) - T(2) * qc) * hy2;
      w[0] = d.dc ? r0 + lin - dt * b * lq : lin - r0 - dt * b * lq;
      break;
    }
    case RX_GS: {
      const T Du = T(d.p[0]), Dv = T(d.p[1]), Ff = T(d.p[2]), kk = T(d.p[3]);
      const GField<T> f1{X + plane, nx, ny, bc};
      const T u0 = c0, v0 = X[plane + o];
      const T lu = lap5(f0, i, j, u0, hx2, hy2), lv = lap5(f1, i, j, v0, hx2, hy2);
      const T ru = r0, rv = R[plane + o];
      if (!d.dc) {
        const T uvv = u0 * v0 * v0;
        w[0] = u0 - ru - dt * Du * lu + dt * uvv + dt * Ff * u0;
        w[1] = v0 - rv - dt * Dv * lv - dt * uvv + dt * (Ff + kk) * v0;
      } else {
        const T U = B[o], V = B[plane + o];
        const T inc = u0 * V * V + T(2) * U * V * v0 + T(2) * u0 * V * v0 + U * v0 * v0 + u0 * v0 * v0;
        w[0] = ru + u0 - dt * Du * lu + dt * inc + dt * Ff * u0;
        w[1] = rv + v0 - dt * Dv * lv - dt * inc + dt * (Ff + kk) * v0;
      }
      break;
    }
    default: {  // RX_SCHNAK
      const T D1 = T(d.p[0]), D2 = T(d.p[1]), kap = T(d.p[2]);
      const GField<T> f1{X + plane, nx, ny, bc};
      const T u0 = c0, v0 = X[plane + o];
      const T lu = lap5(f0, i, j, u0, hx2, hy2), lv = lap5(f1, i, j, v0, hx2, hy2);
      const T ru = r0, rv = R[plane + o];
      if (!d.dc) {
        const T u2v = u0 * u0 * v0;
        w[0] = u0 - ru - dt * D1 * lu + dt * kap * u0 - dt * kap * u2v;
        w[1] = v0 - rv - dt * D2 * lv + dt * kap * u2v;
      } else {
        const T U = B[o], V = B[plane + o];
        const T inc = T(2) * U * u0 * V + u0 * u0 * V + U * U * v0 + T(2) * U * u0 * v0 + u0 * u0 * v0;
        w[0] = ru + u0 - dt * D1 * lu + dt * kap * u0 - dt * kap * inc;
        w[1] = rv + v0 - dt * D2 * lv + dt * kap * inc;
      }
      break;
    }
  }
}

// P~ in shared memory: component line block `line0`, local row lr (two rows per line).
template <class T>
struct SField {
  const cx<T>* buf;
  int ls, nx, bc, line0;
  __device__ __forceinline__ T operator()(int lr, int j) const {
    const cx<T> v = buf[(line0 + (lr >> 1)) * ls + pidx(bcmap(j, nx, bc))];
    return (lr & 1) ? v.y : v.x;
  }
};

// g = dF(x)^T P~ at local row lr, column j; x0, x1 are the components of the current state.
template <class T>
__device__ __forceinline__ void gradT_at(const Desc& d, const SField<T>& p0, const SField<T>& p1,
                                         T x0, T x1, int lr, int j, T* g) {
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const T P = p0(lr, j);
  switch (d.kind) {
    case RX_NONE:
      g[0] = d.op == OP_LAP ? P - dt * a * lap5(p0, lr, j, P, hx2, hy2) : P + dt * a * lap13(p0, lr, j, P, hx2, hy2);
      break;
    case RX_AC:
      g[0] = P - dt * a * lap5(p0, lr, j, P, hx2, hy2) + dt * b * (T(3) * x0 * x0 - T(1)) * P;
      break;
    case RX_CH_IMPL:
    case RX_CH_SPLIT: {
      const T sh = d.kind == RX_CH_IMPL ? T(1) : T(0);
      g[0] = P + dt * a * lap13(p0, lr, j, P, hx2, hy2) - dt * b * (T(3) * x0 * x0 - sh) * lap5(p0, lr, j, P, hx2, hy2);
      break;
    }
    case RX_GS: {
      const T Du = T(d.p[0]), Dv = T(d.p[1]), Ff = T(d.p[2]), kk = T(d.p[3]);
      const T Q = p1(lr, j);
      const T u = x0, v = x1;
      g[0] = P - dt * Du * lap5(p0, lr, j, P, hx2, hy2) + dt * (v * v + Ff) * P - dt * v * v * Q;
      g[1] = Q - dt * Dv * lap5(p1, lr, j, Q, hx2, hy2) + T(2) * dt * u * v * P - dt * (T(2) * u * v - (Ff + kk)) * Q;
      break;
    }
    default: {  // RX_SCHNAK
      const T D1 = T(d.p[0]), D2 = T(d.p[1]), kap = T(d.p[2]);
      const T Q = p1(lr, j);
      const T u = x0, v = x1;
      g[0] = P - dt * (D1 * lap5(p0, lr, j, P, hx2, hy2) + kap * (-P + T(2) * u * v * (P - Q)));
      g[1] = Q - dt * (D2 * lap5(p1, lr, j, Q, hx2, hy2) + kap * (u * u * (P - Q)));
      break;
    }
  }
}

__device__ __forceinline__ bool instance_active(const Desc& d, const State* st) {
  if (d.mode != MODE_PDHG) return true;
  return *((volatile const int*)&st->status) == ST_ACTIVE;
}

// Stopping decision of one PDHG solve from the per-band partial sums (last block only).
__device__ void finalize_measure(const Desc& d, State* st) {
  __threadfence();
  double tot = 0.0;
  for (int c = 0; c < d.ncomp; ++c) {
    double s = 0.0;
    for (int bnd = 0; bnd < d.nbands; ++bnd) s += __ldcg(d.partials + c * d.nbands + bnd);
    tot += sqrt(s);
  }
  const double meas = d.meas_div_dt ? tot / d.dt : tot;
  st->ticket = 0u;
  st->r = meas;
  const int n = st->n;
  if (n == 0) st->r0 = meas;
  const double r0 = n == 0 ? meas : st->r0;
  if (meas <= st->thresh) {
    st->status = ST_CONVERGED;
  } else if (!isfinite(meas) || meas > kDivergeFactor * r0) {
    st->status = ST_DIVERGED;
  } else if (n >= st->max_iter) {
    st->status = ST_NOT_CONVERGED;
  } else {
    st->n = n + 1;
  }
}

// Ticket: returns true in every thread of the last block of the instance to arrive.
__device__ __forceinline__ bool last_block(State* st, int nblocks) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket, 1u);
    s_last = (t == (unsigned)nblocks - 1u);
  }
  __syncthreads();
  return s_last != 0;
}

// ---------------------------------------------------------------------------------------
// k_res: W = F(U_n), ||W||^2 partials, forward row transform, stopping decision
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(512) k_res(const Desc* __restrict__ descs, State* __restrict__ states) {
  const Desc& d = descs[blockIdx.y];
  State* st = states + blockIdx.y;
  const int band = blockIdx.x;
  if (band >= d.nbands) return;
  if (!instance_active(d, st)) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  __shared__ double red[32];

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, nc = d.ncomp;
  const size_t plane = (size_t)nx * ny;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  const int lpc = rows >> 1;
  const int ls = padded_len(nx);
  const T* X = static_cast<const T*>(d.X);
  const T* B = static_cast<const T*>(d.base);
  const T* R = static_cast<const T*>(d.rhs);
  T* WY = static_cast<T*>(d.WY);
  const bool transform = d.precond != 0;

  T acc0 = T(0), acc1 = T(0);
  for (int idx = tid; idx < rows * nx; idx += nt) {
    const int r = idx / nx, j = idx - r * nx;
    const int i = y0 + r;
    T w[2] = {T(0), T(0)};
    if (d.mode == MODE_PRECOND_ONLY) {
      for (int c = 0; c < nc; ++c) w[c] = X[c * plane + (size_t)i * nx + j];
    } else {
      residual_at<T>(d, X, B, R, i, j, w);
    }
    acc0 += w[0] * w[0];
    acc1 += w[1] * w[1];
    if (transform) {
      const int slot = d.bc == BC_PERIODIC ? j : mk_slot(j, nx);
      for (int c = 0; c < nc; ++c) {
        T* e = reinterpret_cast<T*>(buf + (c * lpc + (r >> 1)) * ls + pidx(slot));
        e[r & 1] = w[c];
      }
    } else {
      for (int c = 0; c < nc; ++c) WY[c * plane + (size_t)i * nx + j] = w[c];
    }
  }

  if (transform) {
    __syncthreads();
    block_fft<T, -1>(buf, nc * lpc, d.lognx, ls, static_cast<const cx<T>*>(d.twx), tid, nt);
    const int half = (nx >> 1) + 1;
    const cx<T>* dcx = static_cast<const cx<T>*>(d.dcx);
    for (int g = tid; g < nc * lpc * half; g += nt) {
      const int line = g / half, k = g - line * half;
      const int c = line / lpc, m = line - c * lpc;
      cx<T> ok, okp;
      fwd_post(buf + line * ls, nx, d.bc, dcx, k, ok, okp);
      T* Wa = WY + c * plane + (size_t)(y0 + 2 * m) * nx;
      T* Wb = Wa + nx;
      Wa[k] = ok.x;
      Wb[k] = ok.y;
      if (k != 0) {
        Wa[nx - k] = okp.x;
        Wb[nx - k] = okp.y;
      }
    }
  }

  if (d.mode != MODE_PDHG) return;
  const double s0 = block_sum((double)acc0, red);
  const double s1 = block_sum((double)acc1, red);
  if (tid == 0) {
    d.partials[band] = s0;
    if (nc > 1) d.partials[d.nbands + band] = s1;
  }
  if (last_block(st, d.nbands) && tid == 0) finalize_measure(d, st);
}

// ---------------------------------------------------------------------------------------
// k_col: forward column transform, multiply by 1/(g_hat nx ny), inverse column transform
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(512) k_col(const Desc* __restrict__ descs, State* __restrict__ states) {
  const Desc& d = descs[blockIdx.y];
  State* st = states + blockIdx.y;
  if (d.precond == 0) return;
  if ((int)blockIdx.x >= d.ncomp * d.ncolblk) return;
  if (!instance_active(d, st)) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny;
  const size_t plane = (size_t)nx * ny;
  const int c = blockIdx.x / d.ncolblk, cb = blockIdx.x - c * d.ncolblk;
  const int x0 = cb * d.col_width;
  const int nl = d.col_width >> 1;
  const int ls = padded_len(ny);
  T* WY = static_cast<T*>(d.WY) + c * plane;
  const T* S = static_cast<const T*>(d.scale) + c * plane;
  const cx<T>* twy = static_cast<const cx<T>*>(d.twy);
  const cx<T>* dcy = static_cast<const cx<T>*>(d.dcy);
  const bool per = d.bc == BC_PERIODIC;

  for (int g = tid; g < ny * nl; g += nt) {
    const int row = g / nl, m = g - row * nl;
    const T* src = WY + (size_t)row * nx + x0 + 2 * m;
    const int slot = per ? row : mk_slot(row, ny);
    buf[m * ls + pidx(slot)] = cx<T>{src[0], src[1]};
  }
  __syncthreads();
  block_fft<T, -1>(buf, nl, d.logny, ls, twy, tid, nt);
  const int half = (ny >> 1) + 1;
  for (int g = tid; g < nl * half; g += nt) {
    const int m = g / half, k = g - m * half;
    cx<T>* L = buf + m * ls;
    cx<T> ok, okp;
    fwd_post(L, ny, d.bc, dcy, k, ok, okp);
    const int col = x0 + 2 * m;
    ok.x *= S[(size_t)k * nx + col];
    ok.y *= S[(size_t)k * nx + col + 1];
    L[pidx(k)] = ok;
    if (k != 0) {
      okp.x *= S[(size_t)(ny - k) * nx + col];
      okp.y *= S[(size_t)(ny - k) * nx + col + 1];
      L[pidx(ny - k)] = okp;
    }
  }
  __syncthreads();
  if (per) {
    block_fft<T, -1>(buf, nl, d.logny, ls, twy, tid, nt);
    fwd_post_inplace(buf, nl, ny, ls, d.bc, dcy, tid, nt);
    __syncthreads();
    for (int g = tid; g < ny * nl; g += nt) {
      const int row = g / nl, m = g - row * nl;
      const cx<T> v = buf[m * ls + pidx(row)];
      T* dst = WY + (size_t)row * nx + x0 + 2 * m;
      dst[0] = v.x;
      dst[1] = v.y;
    }
  } else {
    for (int g = tid; g < nl * half; g += nt) {
      const int m = g / half, k = g - m * half;
      cx<T>* L = buf + m * ls;
      const cx<T> Xk = L[pidx(k)];
      const cx<T> Xkp = k != 0 ? L[pidx(ny - k)] : cx<T>{T(0), T(0)};
      const cx<T> w = ldg(dcy + k);
      cx<T> zk, zkp;
      dct_inv_pre(Xk, Xkp, w.x, w.y, zk, zkp);
      L[pidx(k)] = zk;
      if (k != 0) L[pidx(ny - k)] = zkp;
    }
    __syncthreads();
    block_fft<T, 1>(buf, nl, d.logny, ls, twy, tid, nt);
    for (int g = tid; g < ny * nl; g += nt) {
      const int n = g / nl, m = g - n * nl;
      const cx<T> v = buf[m * ls + pidx(n)];
      T* dst = WY + (size_t)mk_perm(n, ny) * nx + x0 + 2 * m;
      dst[0] = v.x;
      dst[1] = v.y;
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_upd: inverse row transform of Y, dual update, extrapolation, primal update
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(512) k_upd(const Desc* __restrict__ descs, State* __restrict__ states) {
  const Desc& d = descs[blockIdx.y];
  State* st = states + blockIdx.y;
  const int band = blockIdx.x;
  if (band >= d.nbands) return;
  if (!instance_active(d, st)) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, nc = d.ncomp, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const bool pconly = d.mode == MODE_PRECOND_ONLY;
  const int H = pconly ? 0 : (d.op == OP_BIHARM ? 2 : 1);
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  const int lrows = rows + 2 * H;
  const int lpc = lrows >> 1;
  const int nl = nc * lpc;
  const int ls = padded_len(nx);
  const T* WY = static_cast<const T*>(d.WY);
  const cx<T>* twx = static_cast<const cx<T>*>(d.twx);
  const cx<T>* dcx = static_cast<const cx<T>*>(d.dcx);

  // 1. Y on rows y0-H .. y0+rows+H-1 (boundary-mapped) into buf, two rows per line
  if (d.precond == 0) {
    for (int g = tid; g < nl * nx; g += nt) {
      const int line = g / nx, j = g - line * nx;
      const int c = line / lpc, m = line - c * lpc;
      const int ga = bcmap(y0 - H + 2 * m, ny, bc), gb = bcmap(y0 - H + 2 * m + 1, ny, bc);
      const T* Wc = WY + c * plane;
      buf[line * ls + pidx(j)] = cx<T>{Wc[(size_t)ga * nx + j], Wc[(size_t)gb * nx + j]};
    }
    __syncthreads();
  } else if (bc == BC_PERIODIC) {
    for (int g = tid; g < nl * nx; g += nt) {
      const int line = g / nx, j = g - line * nx;
      const int c = line / lpc, m = line - c * lpc;
      const int ga = bcmap(y0 - H + 2 * m, ny, bc), gb = bcmap(y0 - H + 2 * m + 1, ny, bc);
      const T* Wc = WY + c * plane;
      buf[line * ls + pidx(j)] = cx<T>{Wc[(size_t)ga * nx + j], Wc[(size_t)gb * nx + j]};
    }
    __syncthreads();
    block_fft<T, -1>(buf, nl, d.lognx, ls, twx, tid, nt);
    fwd_post_inplace(buf, nl, nx, ls, bc, dcx, tid, nt);
    __syncthreads();
  } else {
    const int half = (nx >> 1) + 1;
    for (int g = tid; g < nl * half; g += nt) {
      const int line = g / half, k = g - line * half;
      const int c = line / lpc, m = line - c * lpc;
      const int ga = bcmap(y0 - H + 2 * m, ny, bc), gb = bcmap(y0 - H + 2 * m + 1, ny, bc);
      const T* Wa = WY + c * plane + (size_t)ga * nx;
      const T* Wb = WY + c * plane + (size_t)gb * nx;
      const cx<T> Xk{Wa[k], Wb[k]};
      const cx<T> Xkp = k != 0 ? cx<T>{Wa[nx - k], Wb[nx - k]} : cx<T>{T(0), T(0)};
      const cx<T> w = ldg(dcx + k);
      cx<T> zk, zkp;
      dct_inv_pre(Xk, Xkp, w.x, w.y, zk, zkp);
      cx<T>* L = buf + line * ls;
      L[pidx(k)] = zk;
      if (k != 0) L[pidx(nx - k)] = zkp;
    }
    __syncthreads();
    block_fft<T, 1>(buf, nl, d.lognx, ls, twx, tid, nt);
    // undo the Makhoul reordering in place: slot n holds column mk_perm(n); lines are done in
    // chunks so that each thread holds at most 16 values between the two barriers
    {
      constexpr int MAXV = 16;
      int chunk = (nt * MAXV) / nx;
      if (chunk < 1) chunk = 1;
      for (int l0 = 0; l0 < nl; l0 += chunk) {
        const int cl = nl - l0 < chunk ? nl - l0 : chunk;
        const int total = cl * nx;
        const int nthr = (total + MAXV - 1) / MAXV;
        cx<T> v[MAXV];
#pragma unroll
        for (int s = 0; s < MAXV; ++s) {
          const int g = tid + s * nthr;
          if (tid < nthr && g < total) {
            const int line = l0 + g / nx, n = g % nx;
            v[s] = buf[line * ls + pidx(n)];
          }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < MAXV; ++s) {
          const int g = tid + s * nthr;
          if (tid < nthr && g < total) {
            const int line = l0 + g / nx, n = g % nx;
            buf[line * ls + pidx(mk_perm(n, nx))] = v[s];
          }
        }
        __syncthreads();
      }
    }
  }

  T* X = static_cast<T*>(d.X);
  if (pconly) {
    for (int idx = tid; idx < nc * rows * nx; idx += nt) {
      const int c = idx / (rows * nx);
      const int rem = idx - c * rows * nx;
      const int r = rem / nx, j = rem - r * nx;
      const cx<T> e = buf[(c * lpc + (r >> 1)) * ls + pidx(j)];
      X[c * plane + (size_t)(y0 + r) * nx + j] = (r & 1) ? e.y : e.x;
    }
    return;
  }

  // 2. P~ = P_n + (1 + omega) tau_p Y on all local rows; P_{n+1} = P_n + tau_p Y on band rows
  const int n = st->n;  // already counts this update
  const T* Pin = static_cast<const T*>(d.P[(n - 1) & 1]);
  T* Pout = static_cast<T*>(d.P[n & 1]);
  const T tp = T(d.tau_p), tpe = T((1.0 + d.omega) * d.tau_p), tu = T(d.tau_u);
  for (int g = tid; g < nl * nx; g += nt) {
    const int line = g / nx, j = g - line * nx;
    const int c = line / lpc, m = line - c * lpc;
    cx<T>& e = buf[line * ls + pidx(j)];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int lr = 2 * m + h;
      const int gr = bcmap(y0 - H + lr, ny, bc);
      const size_t o = c * plane + (size_t)gr * nx + j;
      const T pold = Pin[o];
      T& yv = h ? e.y : e.x;
      const T y = yv;
      yv = pold + tpe * y;
      if (lr >= H && lr < H + rows) Pout[o] = pold + tp * y;
    }
  }
  __syncthreads();

  // 3. U_{n+1} = U_n - tau_u dF(U_n)^T P~ on band rows
  const T* Bs = static_cast<const T*>(d.base);
  const SField<T> p0{buf, ls, nx, bc, 0};
  const SField<T> p1{buf, ls, nx, bc, lpc};
  for (int idx = tid; idx < rows * nx; idx += nt) {
    const int r = idx / nx, j = idx - r * nx;
    const size_t o = (size_t)(y0 + r) * nx + j;
    const T xa = X[o];
    const T xb = nc > 1 ? X[plane + o] : T(0);
    T s0 = xa, s1 = xb;
    if (d.dc) {
      s0 += Bs[o];
      if (nc > 1) s1 += Bs[plane + o];
    }
    T g[2] = {T(0), T(0)};
    gradT_at<T>(d, p0, p1, s0, s1, H + r, j, g);
    X[o] = xa - tu * g[0];
    if (nc > 1) X[plane + o] = xb - tu * g[1];
  }
}

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
  if (last_block(st, d.nbands) && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (int b2 = 0; b2 < d.nbands; ++b2) tot += __ldcg(d.partials + b2);
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

// W = F(u) in FP64.  Optional outputs: w64 (FP64), r32 = (float)W and u32 = (float)u.  With
// `decide`, the last block applies the outer stopping rule of defect correction to `outer` and
// arms the inner FP32 solve `inner` (threshold rtol * sum_c ||W_c||).
__global__ void k_resid64(const Desc* __restrict__ d64, State* __restrict__ outer, State* __restrict__ inner,
                          const double* __restrict__ u, const double* __restrict__ rhs,
                          double* __restrict__ w64, float* __restrict__ r32, float* __restrict__ u32,
                          int decide, double rtol) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp;
  const size_t plane = (size_t)nx * ny;
  const int band = blockIdx.x;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  double acc0 = 0.0, acc1 = 0.0;
  for (int idx = threadIdx.x; idx < rows * nx; idx += blockDim.x) {
    const int r = idx / nx, j = idx - r * nx;
    const int i = y0 + r;
    double w[2] = {0.0, 0.0};
    residual_at<double>(d, u, nullptr, rhs, i, j, w);
    for (int c = 0; c < nc; ++c) {
      const size_t o = c * plane + (size_t)i * nx + j;
      if (w64) w64[o] = w[c];
      if (r32) r32[o] = (float)w[c];
      if (u32) u32[o] = (float)u[o];
    }
    acc0 += w[0] * w[0];
    acc1 += w[1] * w[1];
  }
  if (!decide) return;
  const double s0 = block_sum(acc0, red);
  const double s1 = block_sum(acc1, red);
  if (threadIdx.x == 0) {
    d.partials[band] = s0;
    if (nc > 1) d.partials[d.nbands + band] = s1;
  }
  if (last_block(outer, d.nbands) && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (int c = 0; c < nc; ++c) {
      double s = 0.0;
      for (int b2 = 0; b2 < d.nbands; ++b2) s += __ldcg(d.partials + c * d.nbands + b2);
      tot += sqrt(s);
    }
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
  if (last_block(st, d.nbands) && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (int b2 = 0; b2 < d.nbands; ++b2) tot += __ldcg(d.partials + b2);
    st->ticket = 0u;
    st->mass = tot / (sqrt(d.hx2) * sqrt(d.hy2));
  }
}

// ---------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------

// Allow each kernel the opt-in shared memory of the device minus its static shared memory.
template <class K>
static cudaError_t allow_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <class T>
cudaError_t set_kernel_smem_limits(int* usable) {
  int dev = 0, optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  if ((e = allow_smem(k_res<T>, optin)) != cudaSuccess) return e;
  if ((e = allow_smem(k_col<T>, optin)) != cudaSuccess) return e;
  if ((e = allow_smem(k_upd<T>, optin)) != cudaSuccess) return e;
  if (usable) *usable = optin - 1024;  // headroom for the kernels' static shared memory
  return cudaSuccess;
}

template <class T>
cudaError_t launch_iteration(const Desc* d, State* st, int ninst, const LaunchCfg& c, cudaStream_t s) {
  k_res<T><<<dim3(c.grid_bands, ninst), c.thr_res, c.smem_res, s>>>(d, st);
  if (c.transform) k_col<T><<<dim3(c.grid_cols, ninst), c.thr_col, c.smem_col, s>>>(d, st);
  k_upd<T><<<dim3(c.grid_bands, ninst), c.thr_upd, c.smem_upd, s>>>(d, st);
  return cudaGetLastError();
}

// As launch_iteration, with events recorded before k_res and after each kernel.
template <class T>
cudaError_t launch_iteration_timed(const Desc* d, State* st, int ninst, const LaunchCfg& c, cudaStream_t s,
                                   cudaEvent_t* ev) {
  cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
  k_res<T><<<dim3(c.grid_bands, ninst), c.thr_res, c.smem_res, s>>>(d, st);
  cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
  if (c.transform) k_col<T><<<dim3(c.grid_cols, ninst), c.thr_col, c.smem_col, s>>>(d, st);
  cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
  k_upd<T><<<dim3(c.grid_bands, ninst), c.thr_upd, c.smem_upd, s>>>(d, st);
  cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal);
  return cudaGetLastError();
}

template cudaError_t launch_iteration_timed<float>(const Desc*, State*, int, const LaunchCfg&, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_iteration_timed<double>(const Desc*, State*, int, const LaunchCfg&, cudaStream_t, cudaEvent_t*);
template cudaError_t set_kernel_smem_limits<float>(int*);
template cudaError_t set_kernel_smem_limits<double>(int*);
template cudaError_t launch_iteration<float>(const Desc*, State*, int, const LaunchCfg&, cudaStream_t);
template cudaError_t launch_iteration<double>(const Desc*, State*, int, const LaunchCfg&, cudaStream_t);

cudaError_t launch_begin(const Desc* d64, State* st, const double* uk, double* rhs, double tol, int tol_kind,
                         int nbands, cudaStream_t s) {
  k_begin<<<nbands, 256, 0, s>>>(d64, st, uk, rhs, tol, tol_kind);
  return cudaGetLastError();
}

cudaError_t launch_resid64(const Desc* d64, State* outer, State* inner, const double* u, const double* rhs,
                           double* w64, float* r32, float* u32, int decide, double rtol, int nbands,
                           cudaStream_t s) {
  k_resid64<<<nbands, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, decide, rtol);
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
