// The three kernels of one G-prox PDHG iteration (arxiv 2305.03945, Section 2.1, Algorithm 1),
// templated on the arithmetic type T and on the equation K so that each instantiation holds only
// its own physics.  T = float is the inner solve of FP64 defect correction (the unknown is the
// correction d of u + d); T = double is the plain FP64 method.
//
//   k_res  (row bands)      W = F(U_n) (eq. F(U) rd equation / F(U) CH / Section 3.4.1), the
//                           per-band partial sums of ||W_c||^2, the forward row transform of W
//                           along x, and (last block to finish) the stopping decision
//                           ||Res(U_n)||_2 <= delta of Section 2.1;
//   k_col  (column blocks)  forward column transform along y, multiplication by 1/g_hat (the
//                           spectral inverse of G = A_lin^2), inverse column transform;
//   k_upd  (row bands)      inverse row transform of Y = G^{-1} W, the dual update
//                           P_{n+1} = P_n + tau_p Y, the extrapolation P~ = P_n + (1+omega) tau_p Y
//                           (eqs. G-prox ... dynamic 1-2) and the primal update
//                           U_{n+1} = U_n - tau_u dF(U_n)^T P~ (eq. G-prox ... dynamic 3).
// The transforms are the separable Hartley transform (periodic) and Makhoul's DCT-II (Neumann),
// both of which diagonalise the five-point Laplacian with its boundary rule.
#pragma once

#include "rd_device.cuh"
#include "rd_launch.h"

namespace rd {

__host__ __device__ inline int kind_key(const Desc& d) {
  if (d.mode == MODE_PRECOND_ONLY) return KK_PCONLY;
  if (d.kind == RX_NONE) return d.op == OP_BIHARM ? KK_NONE_BIH : KK_NONE_LAP;
  return d.kind;
}

template <int K>
struct KT {
  static constexpr bool biharm = K == KK_CH_IMPL || K == KK_CH_SPLIT || K == KK_NONE_BIH;
  static constexpr bool two = K == KK_GS || K == KK_SCHNAK;
  static constexpr int H = K == KK_PCONLY ? 0 : (biharm ? 2 : 1);
  static constexpr bool nonlinear = K != KK_NONE_LAP && K != KK_NONE_BIH && K != KK_PCONLY;
};

__host__ __device__ inline int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// staged rows in shared memory, row stride nx; columns boundary-mapped only when EDGE
template <class T, bool EDGE>
struct Rows {
  const T* p;
  int nx, bc;
  __device__ __forceinline__ T operator()(int lr, int j) const {
    if constexpr (EDGE) return p[lr * nx + bcmap(j, nx, bc)];
    else return p[lr * nx + j];
  }
};

// Base values of the points of one vector group, held in registers (kinds whose residual reads
// the defect-correction base state only at the point itself)
template <class T>
struct PtVals {
  const T* v;
  int j0;
  __device__ __forceinline__ T operator()(int, int j) const { return v[j - j0]; }
};

// Does the defect-correction residual of kind K read the base state at neighbouring points
// (Cahn-Hilliard: the Laplacian of the linearised chemical potential)?  Otherwise only at the
// point itself, and the base rows are not staged in shared memory.
template <int K>
__host__ __device__ constexpr bool base_stencil() { return K == KK_CH_IMPL || K == KK_CH_SPLIT; }

// P~ in the complex transform buffer: two rows per line (row a in .x, row b in .y)
template <class T, bool EDGE>
struct Pairs {
  const cx<T>* buf;
  int ls, nx, bc, line0;
  __device__ __forceinline__ T operator()(int lr, int j) const {
    const int jj = EDGE ? bcmap(j, nx, bc) : j;
    const cx<T> v = buf[(line0 + (lr >> 1)) * ls + pidx(jj)];
    return (lr & 1) ? v.y : v.x;
  }
};

// W_c = F_c(X) at one point for every component (see residual map definitions in rd_pdhg.h).
//   plain (DC = false): X = U, r = rhs of the step (U^k plus the explicit / constant terms)
//   DC    (DC = true) : X = d, B = u, r = F(u); returns F(u + d) = F(u) + A_lin d + N(u + d) - N(u)
//                       with the nonlinear increment expanded so that no large terms cancel.
template <class T, int K, bool DC, class A, class B = A>
__device__ __forceinline__ void residual_pt(const Desc& d, const A& x0, const A& x1, const B& b0, const B& b1,
                                            int i, int j, T r0, T r1, T* w) {
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const T c0 = x0(i, j);
  if constexpr (K == KK_NONE_LAP || K == KK_NONE_BIH) {
    const T lin = K == KK_NONE_LAP ? c0 - dt * a * lap5(x0, i, j, c0, hx2, hy2)
                                   : c0 + dt * a * lap13(x0, i, j, c0, hx2, hy2);
    w[0] = DC ? r0 + lin : lin - r0;
  } else if constexpr (K == KK_AC) {
    const T lin = c0 - dt * a * lap5(x0, i, j, c0, hx2, hy2);
    if constexpr (!DC) {
      w[0] = lin - r0 + dt * b * (c0 * c0 * c0 - c0);
    } else {
      const T u = b0(i, j);
      w[0] = r0 + lin + dt * b * (c0 * (T(3) * u * u - T(1)) + c0 * c0 * (T(3) * u + c0));
    }
  } else if constexpr (K == KK_CH_IMPL || K == KK_CH_SPLIT) {
    const T lin = c0 + dt * a * lap13(x0, i, j, c0, hx2, hy2);
    constexpr T sh = K == KK_CH_IMPL ? T(1) : T(0);
    auto q = [&](int ii, int jj) -> T {
      const T xv = x0(ii, jj);
      if constexpr (!DC) {
        return xv * xv * xv - sh * xv;
      } else {
        const T u = b0(ii, jj);
        return xv * (T(3) * u * u - sh) + xv * xv * (T(3) * u + xv);
      }
    };
    const T qc = q(i, j);
    const T lq = (q(i, j + 1) + q(i, j - 1) - T(2) * qc) * hx2 + (q(i + 1, j) + q(i - 1, j) - T(2) * qc) * hy2;
    w[0] = DC ? r0 + lin - dt * b * lq : lin - r0 - dt * b * lq;
  } else if constexpr (K == KK_GS) {
    const T Du = T(d.p[0]), Dv = T(d.p[1]), Ff = T(d.p[2]), kk = T(d.p[3]);
    const T u0 = c0, v0 = x1(i, j);
    const T lu = lap5(x0, i, j, u0, hx2, hy2), lv = lap5(x1, i, j, v0, hx2, hy2);
    if constexpr (!DC) {
      const T uvv = u0 * v0 * v0;
      w[0] = u0 - r0 - dt * Du * lu + dt * uvv + dt * Ff * u0;
      w[1] = v0 - r1 - dt * Dv * lv - dt * uvv + dt * (Ff + kk) * v0;
    } else {
      const T U = b0(i, j), V = b1(i, j);
      const T inc = u0 * V * V + T(2) * U * V * v0 + T(2) * u0 * V * v0 + U * v0 * v0 + u0 * v0 * v0;
      w[0] = r0 + u0 - dt * Du * lu + dt * inc + dt * Ff * u0;
      w[1] = r1 + v0 - dt * Dv * lv - dt * inc + dt * (Ff + kk) * v0;
    }
  } else if constexpr (K == KK_SCHNAK) {
    const T D1 = T(d.p[0]), D2 = T(d.p[1]), kap = T(d.p[2]);
    const T u0 = c0, v0 = x1(i, j);
    const T lu = lap5(x0, i, j, u0, hx2, hy2), lv = lap5(x1, i, j, v0, hx2, hy2);
    if constexpr (!DC) {
      const T u2v = u0 * u0 * v0;
      w[0] = u0 - r0 - dt * D1 * lu + dt * kap * u0 - dt * kap * u2v;
      w[1] = v0 - r1 - dt * D2 * lv + dt * kap * u2v;
    } else {
      const T U = b0(i, j), V = b1(i, j);
      const T inc = T(2) * U * u0 * V + u0 * u0 * V + U * U * v0 + T(2) * U * u0 * v0 + u0 * u0 * v0;
      w[0] = r0 + u0 - dt * D1 * lu + dt * kap * u0 - dt * kap * inc;
      w[1] = r1 + v0 - dt * D2 * lv + dt * kap * inc;
    }
  }
}

// g = dF(x)^T P~ at local row lr, column j; x0, x1 are the components of the current state.
template <class T, int K, class SF>
__device__ __forceinline__ void gradT_pt(const Desc& d, const SF& p0, const SF& p1, T x0, T x1, int lr, int j,
                                         T* g) {
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const T P = p0(lr, j);
  if constexpr (K == KK_NONE_LAP) {
    g[0] = P - dt * a * lap5(p0, lr, j, P, hx2, hy2);
  } else if constexpr (K == KK_NONE_BIH) {
    g[0] = P + dt * a * lap13(p0, lr, j, P, hx2, hy2);
  } else if constexpr (K == KK_AC) {
    g[0] = P - dt * a * lap5(p0, lr, j, P, hx2, hy2) + dt * b * (T(3) * x0 * x0 - T(1)) * P;
  } else if constexpr (K == KK_CH_IMPL || K == KK_CH_SPLIT) {
    constexpr T sh = K == KK_CH_IMPL ? T(1) : T(0);
    g[0] = P + dt * a * lap13(p0, lr, j, P, hx2, hy2) - dt * b * (T(3) * x0 * x0 - sh) * lap5(p0, lr, j, P, hx2, hy2);
  } else if constexpr (K == KK_GS) {
    const T Du = T(d.p[0]), Dv = T(d.p[1]), Ff = T(d.p[2]), kk = T(d.p[3]);
    const T Q = p1(lr, j);
    const T u = x0, v = x1;
    g[0] = P - dt * Du * lap5(p0, lr, j, P, hx2, hy2) + dt * (v * v + Ff) * P - dt * v * v * Q;
    g[1] = Q - dt * Dv * lap5(p1, lr, j, Q, hx2, hy2) + T(2) * dt * u * v * P - dt * (T(2) * u * v - (Ff + kk)) * Q;
  } else if constexpr (K == KK_SCHNAK) {
    const T D1 = T(d.p[0]), D2 = T(d.p[1]), kap = T(d.p[2]);
    const T Q = p1(lr, j);
    const T u = x0, v = x1;
    g[0] = P - dt * (D1 * lap5(p0, lr, j, P, hx2, hy2) + kap * (-P + T(2) * u * v * (P - Q)));
    g[1] = Q - dt * (D2 * lap5(p1, lr, j, Q, hx2, hy2) + kap * (u * u * (P - Q)));
  }
}

// Ticket: returns true in every thread of the last block of the launch to arrive.
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

// Sum of n partials with a fixed thread partition and a fixed tree (the result depends only on
// n and blockDim).  Called by every thread of the block; valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* p, int n, double* red) {
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += __ldcg(p + k);
  return block_sum(s, red);
}

// Is the solve this sweep belongs to running?  Single solves look at their status; batch
// members (slot != nullptr) at the slot's phase.
__device__ __forceinline__ bool sweep_active(const State* st, const Slot* slot) {
  if (slot) return *((volatile const int*)&slot->phase) == PH_INNER;
  return *((volatile const int*)&st->status) == ST_ACTIVE;
}

// Cooperative copy of a descriptor into shared memory (batched kernels).
__device__ __forceinline__ void load_desc(Desc& dst, const Desc* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* t = reinterpret_cast<int*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Desc) / sizeof(int)); k += blockDim.x) t[k] = s[k];
}

// Stopping decision of one PDHG solve from the per-band partial sums (all threads of the last
// block call it): r <= threshold -> converged; non-finite or 1e8-fold growth -> diverged;
// max_iter updates done -> not converged; otherwise count the coming update.  A batch member
// hands control back to its slot's defect-correction loop when the solve stops.
// The stopping rule itself, from tot = sum_c ||F_c(U_n)|| (one thread; st may be a copy in shared
// memory).
__device__ inline void measure_decide(const Desc& d, State* st, double tot, Slot* slot) {
  const double meas = d.meas_div_dt ? tot / d.dt : tot;
  st->ticket = 0u;
  st->r = meas;
  const int n = st->n;
  if (n == 0) {
    st->r0 = meas;
    st->best = meas;
    st->best_n = 0;
  } else if (meas < 0.5 * st->best) {
    st->best = meas;
    st->best_n = n;
  }
  const double r0 = n == 0 ? meas : st->r0;
  if (meas <= st->thresh) {
    st->status = ST_CONVERGED;
  } else if (!isfinite(meas) || meas > kDivergeFactor * r0) {
    st->status = ST_DIVERGED;
  } else if (d.stall_window > 0 && n - st->best_n >= d.stall_window * (st->stall_mul > 1 ? st->stall_mul : 1)) {
    st->status = ST_CONVERGED;  // stalled at the rounding floor of this precision
  } else if (n >= st->max_iter) {
    st->status = ST_NOT_CONVERGED;
  } else {
    st->n = n + 1;
  }
  if (slot && st->status != ST_ACTIVE) {
    slot->inner_total += st->n;
    slot->phase = st->status == ST_DIVERGED ? PH_FAILED : PH_AXPY;
  }
}

__device__ inline void finalize_measure(const Desc& d, State* st, double* red, Slot* slot = nullptr, int nblk = 0) {
  __threadfence();
  const int nb = nblk > 0 ? nblk : d.nbands;
  double tot = 0.0;
  for (int c = 0; c < d.ncomp; ++c) tot += sqrt(sum_partials(d.partials + c * nb, nb, red));
  if (threadIdx.x != 0) return;
  measure_decide(d, st, tot, slot);
}

// Step set-up decision (thread 0 of the last block of a begin kernel): ||U^k|| = sqrt(tot), the
// stopping threshold of the step (tol, or tol ||U^k||), and a fresh solve state.
__device__ inline void begin_state(State* st, double tot, double tol, int tol_kind) {
  const double nrm = sqrt(tot);
  st->ticket = 0u;
  st->aux = nrm;
  st->thresh = tol_kind == 1 ? tol * nrm : tol;
  st->n = 0;
  st->r = 0.0;
  st->r0 = 0.0;
  st->trips = 0u;
  st->total = 0;
  st->launches = 0;
  st->status = ST_ACTIVE;
}

// Outer stopping rule of defect correction (thread 0 of the last block of an FP64 residual
// kernel), from tot = sum_c ||W_c|| of W = F(u): evaluation number max_outer (counting from 0)
// ends the step as not converged; otherwise the inner FP32 solve is armed with the threshold
// max(rtol tot, half the outer threshold in the same units).
__device__ inline void outer_decide(const Desc& d, State* outer, State* inner, double tot, double rtol,
                                    int max_outer) {
  const double meas = d.meas_div_dt ? tot / d.dt : tot;
  const double prev = outer->r;
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
  } else if (n >= max_outer) {
    outer->status = ST_NOT_CONVERGED;
  } else {
    inner->stall_mul = next_stall_mul(n, meas, prev, inner->stall_mul);
    inner->n = 0;
    inner->trips = 0u;
    inner->r = 0.0;
    inner->r0 = 0.0;
    // rtol of the current FP64 residual, but no tighter than half of what the outer stopping
    // rule still needs: the last round solves no further than the step requires
    inner->thresh = fmax(rtol * tot, 0.5 * outer->thresh * (d.meas_div_dt ? d.dt : 1.0));
    inner->status = ST_ACTIVE;
    inner->ticket = 0u;
  }
}

// 16-byte vectors
template <class T> struct V16;
template <> struct V16<float> { using t = float4; static constexpr int n = 4; };
template <> struct V16<double> { using t = double2; static constexpr int n = 2; };

template <class T, int W>
__device__ __forceinline__ void vld(const T* __restrict__ p, T* v) {
  if constexpr (W == V16<T>::n) {
    const typename V16<T>::t q = *reinterpret_cast<const typename V16<T>::t*>(p);
    const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = e[k];
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = p[k];
  }
}
template <class T, int W>
__device__ __forceinline__ void vst(T* __restrict__ p, const T* v) {
  if constexpr (W == V16<T>::n) {
    typename V16<T>::t q;
    T* e = reinterpret_cast<T*>(&q);
#pragma unroll
    for (int k = 0; k < W; ++k) e[k] = v[k];
    *reinterpret_cast<typename V16<T>::t*>(p) = q;
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) p[k] = v[k];
  }
}

// two adjacent entries of an array as one 8- or 16-byte load
template <class T>
__device__ __forceinline__ cx<T> ld_pair(const T* p) {
  return *reinterpret_cast<const cx<T>*>(p);
}

// Copy rows g0 .. g0+nrows-1 (boundary-mapped) of a plane into shared memory (row stride nx).
// Each thread first gathers up to 8 vectors into registers and only then stores them, so that
// all of its global loads are in flight together.
template <class T, int W>
__device__ __forceinline__ void stage_rows_w(T* dst, const T* __restrict__ src, int nx, int lognx, int ny, int bc,
                                             int g0, int nrows) {
  constexpr int MAXV = 8;
  const int lw = W == 4 ? 2 : (W == 2 ? 1 : 0);
  const int lv = lognx - lw;  // log2 vectors per row
  const int total = nrows << lv;
  const int nt = blockDim.x;
  for (int base = 0; base < total; base += MAXV * nt) {
    T e[MAXV][W];
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int v = base + threadIdx.x + q * nt;
      if (v < total) {
        const int r = v >> lv, c = v & ((1 << lv) - 1);
        vld<T, W>(src + (size_t)bcmap(g0 + r, ny, bc) * nx + c * W, e[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int v = base + threadIdx.x + q * nt;
      if (v < total) {
        const int r = v >> lv, c = v & ((1 << lv) - 1);
        vst<T, W>(dst + r * nx + c * W, e[q]);
      }
    }
  }
}
template <class T>
__device__ __forceinline__ void stage_rows(T* dst, const T* __restrict__ src, int nx, int lognx, int ny, int bc,
                                           int g0, int nrows) {
  constexpr int W = V16<T>::n;
  if (nx >= W) stage_rows_w<T, W>(dst, src, nx, lognx, ny, bc, g0, nrows);
  else stage_rows_w<T, 1>(dst, src, nx, lognx, ny, bc, g0, nrows);
}

// In-place forward epilogue over all lines (slot k <- real coefficients of both lines).
template <class T>
__device__ __forceinline__ void post_inplace(cx<T>* buf, int nlines, int logN, int ls, int bc,
                                             const cx<T>* __restrict__ dc) {
  const int N = 1 << logN, hn = N >> 1, lh = logN - 1;
  for (int g = threadIdx.x; g < (nlines << lh); g += blockDim.x) {
    const int line = g >> lh, k = g & (hn - 1);
    cx<T>* L = buf + line * ls;
    cx<T> ok, okp;
    fwd_post(L, N, bc, dc, k, ok, okp);
    if (k == 0) {
      cx<T> mk, mkp;
      fwd_post(L, N, bc, dc, hn, mk, mkp);
      L[pidx(0)] = ok;
      L[pidx(hn)] = mk;
    } else {
      L[pidx(k)] = ok;
      L[pidx(N - k)] = okp;
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_res
// ---------------------------------------------------------------------------------------
template <class T, int K, bool EDGE, int W>
__device__ __forceinline__ void res_group(const Desc& d, cx<T>* buf, const T* xs, const T* bs, int srows, int r,
                                          int j0, const T* rr0, const T* rr1, const T* pb0, const T* pb1, int lpc,
                                          int ls, T* w0, T* w1) {
  constexpr bool PC = K == KK_PCONLY;
  constexpr bool DC = !PC && sizeof(T) == 4;
  constexpr int H = KT<K>::H;
  const Rows<T, EDGE> x0{xs, d.nx, d.bc}, x1{xs + srows * d.nx, d.nx, d.bc};
  const Rows<T, EDGE> b0{bs, d.nx, d.bc}, b1{bs + srows * d.nx, d.nx, d.bc};
  const PtVals<T> v0{pb0, j0}, v1{pb1, j0};
#pragma unroll
  for (int q = 0; q < W; ++q) {
    T w[2] = {T(0), T(0)};
    if constexpr (PC) {
      w[0] = x0(r, j0 + q);
      if (d.ncomp > 1) w[1] = x1(r, j0 + q);
    } else if constexpr (DC && !base_stencil<K>()) {
      residual_pt<T, K, DC>(d, x0, x1, v0, v1, H + r, j0 + q, rr0[q], KT<K>::two ? rr1[q] : T(0), w);
    } else {
      residual_pt<T, K, DC>(d, x0, x1, b0, b1, H + r, j0 + q, rr0[q], KT<K>::two ? rr1[q] : T(0), w);
    }
    w0[q] = w[0];
    w1[q] = w[1];
  }
}

template <class T, int K, int W>
__device__ __forceinline__ void res_points(const Desc& d, cx<T>* buf, const T* xs, const T* bs, int y0, int rows,
                                           int ls, T& acc0, T& acc1) {
  constexpr bool PC = K == KK_PCONLY;
  constexpr int H = KT<K>::H;
  const int nx = d.nx, bc = d.bc;
  const int nc = PC ? d.ncomp : (KT<K>::two ? 2 : 1);
  const size_t plane = (size_t)nx * d.ny;
  const int srows = rows + 2 * H;
  const int lpc = rows >> 1;
  const T* R = static_cast<const T*>(d.rhs);
  T* WY = static_cast<T*>(d.WY);
  const bool transform = d.precond != 0;
  const int lw = W == 4 ? 2 : (W == 2 ? 1 : 0);
  const int lv = d.lognx - lw;
  // defect-correction base values read at the point only (not staged in shared memory)
  constexpr bool PTB = !PC && sizeof(T) == 4 && KT<K>::nonlinear && !base_stencil<K>();
  const T* Bg = static_cast<const T*>(d.base);
  constexpr int G = PTB ? 2 : 4;  // vector groups whose right-hand sides are loaded together
  const int total = rows << lv;
  for (int base = 0; base < total; base += G * blockDim.x) {
   T rrg0[G][W], rrg1[G][W], pbg0[G][W], pbg1[G][W];
   if constexpr (!PC) {
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int v = base + threadIdx.x + q * blockDim.x;
      if (v < total) {
        const size_t o = (size_t)(y0 + (v >> lv)) * nx + (v & ((1 << lv) - 1)) * W;
        vld<T, W>(R + o, rrg0[q]);
        if constexpr (KT<K>::two) vld<T, W>(R + plane + o, rrg1[q]);
        if constexpr (PTB) {
          vld<T, W>(Bg + o, pbg0[q]);
          if constexpr (KT<K>::two) vld<T, W>(Bg + plane + o, pbg1[q]);
        }
      }
    }
   }
#pragma unroll
   for (int q = 0; q < G; ++q) {
    const int v = base + threadIdx.x + q * blockDim.x;
    if (v >= total) break;
    const int r = v >> lv, j0 = (v & ((1 << lv) - 1)) * W;
    const size_t o = (size_t)(y0 + r) * nx + j0;
    const T* rr0 = rrg0[q];
    const T* rr1 = rrg1[q];
    T w0[W], w1[W];
    // five-point kinds: boundary-mapped columns everywhere (one copy of the residual code, see
    // upd_points); the 13-point biharmonic stencil keeps an interior copy without the mapping
    // (its 13 mapped reads per point cost more than the extra code)
    if (KT<K>::biharm && j0 >= 2 && j0 + W + 2 <= nx)
      res_group<T, K, false, W>(d, buf, xs, bs, srows, r, j0, rr0, rr1, pbg0[q], pbg1[q], lpc, ls, w0, w1);
    else
      res_group<T, K, true, W>(d, buf, xs, bs, srows, r, j0, rr0, rr1, pbg0[q], pbg1[q], lpc, ls, w0, w1);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      acc0 += w0[q] * w0[q];
      acc1 += w1[q] * w1[q];
    }
    if (transform) {
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int j = j0 + q;
        const int slot = bc == BC_PERIODIC ? j : mk_slot(j, nx);
        T* e0 = reinterpret_cast<T*>(buf + (r >> 1) * ls + pidx(slot));
        e0[r & 1] = w0[q];
        if (nc > 1) {
          T* e1 = reinterpret_cast<T*>(buf + (lpc + (r >> 1)) * ls + pidx(slot));
          e1[r & 1] = w1[q];
        }
      }
    } else {
      vst<T, W>(WY + o, w0);
      if (nc > 1) vst<T, W>(WY + plane + o, w1);
    }
   }
  }
}

template <class T, int K>
__device__ __forceinline__ void res_body(const Desc& d, State* __restrict__ st, Slot* slot, int band,
                                         unsigned char* smem_raw) {
  constexpr bool PC = K == KK_PCONLY;
  constexpr bool DC = !PC && sizeof(T) == 4;
  constexpr int H = KT<K>::H;
  if (band >= d.nbands) return;
  if (!PC && !sweep_active(st, slot)) return;

  __shared__ double red[32];

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, bc = d.bc, lognx = d.lognx;
  const int nc = PC ? d.ncomp : (KT<K>::two ? 2 : 1);
  const size_t plane = (size_t)nx * ny;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  const int lpc = rows >> 1;
  const int ls = padded_len(nx);
  const int srows = rows + 2 * H;
  T* WY = static_cast<T*>(d.WY);

  // 1. stage the unknown (and the defect-correction base state) rows with halo, and the
  //    transform tables
  const cx<T>* tws;
  const cx<T>* dcs;
  cx<T>* buf = reinterpret_cast<cx<T>*>(place_tables<T>(smem_raw, d.twx, d.dcx, nx, d.precond != 0,
                                                        d.precond != 0 && bc == BC_NEUMANN, tws, dcs));
  const bool pp = (d.fft_pp & 1) != 0;
  cx<T>* scr = pp ? buf + nc * lpc * ls : buf;
  T* xs = reinterpret_cast<T*>(buf + (pp ? 2 : 1) * nc * lpc * ls);
  T* bs = xs + nc * srows * nx;
  const T* X = static_cast<const T*>(d.X);
  for (int c = 0; c < nc; ++c) stage_rows<T>(xs + c * srows * nx, X + c * plane, nx, lognx, ny, bc, y0 - H, srows);
  if constexpr (DC && base_stencil<K>()) {
    const T* Bg = static_cast<const T*>(d.base);
    for (int c = 0; c < nc; ++c) stage_rows<T>(bs + c * srows * nx, Bg + c * plane, nx, lognx, ny, bc, y0 - H, srows);
  }
  __syncthreads();

  // 2. W = F(U_n) on the band rows, written packed into the transform buffer
  T acc0 = T(0), acc1 = T(0);
  if (nx >= V16<T>::n) res_points<T, K, V16<T>::n>(d, buf, xs, bs, y0, rows, ls, acc0, acc1);
  else res_points<T, K, 1>(d, buf, xs, bs, y0, rows, ls, acc0, acc1);

  // 3. forward row transform and its epilogue straight to global memory
  if (d.precond != 0) {
    __syncthreads();
    const cx<T>* res = block_fft<T, -1>(buf, scr, nc * lpc, lognx, ls, tws, tid, nt, (d.fft_pp & 8) != 0);
    const int hn = nx >> 1, lh = lognx - 1;
    const cx<T>* dcx = dcs;
    for (int g = tid; g < ((nc * lpc) << lh); g += nt) {
      const int line = g >> lh, k = g & (hn - 1);
      const int c = (PC ? nc > 1 : KT<K>::two) ? line / lpc : 0, m = line - c * lpc;
      const cx<T>* L = res + line * ls;
      T* Wa = WY + c * plane + (size_t)(y0 + 2 * m) * nx;
      T* Wb = Wa + nx;
      cx<T> ok, okp;
      fwd_post(L, nx, bc, dcx, k, ok, okp);
      Wa[k] = ok.x;
      Wb[k] = ok.y;
      if (k != 0) {
        Wa[nx - k] = okp.x;
        Wb[nx - k] = okp.y;
      } else {
        fwd_post(L, nx, bc, dcx, hn, ok, okp);
        Wa[hn] = ok.x;
        Wb[hn] = ok.y;
      }
    }
  }

  if constexpr (PC) return;
  // 4. partial norms, ticket, stopping decision in the last block
  const double s0 = block_sum((double)acc0, red);
  const double s1 = KT<K>::two ? block_sum((double)acc1, red) : 0.0;
  if (tid == 0) {
    d.partials[band] = s0;
    if (KT<K>::two) d.partials[d.nbands + band] = s1;
  }
  if (last_block(st, d.nbands)) finalize_measure(d, st, red, slot);
}

template <class T, int K>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value) k_res(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  res_body<T, K>(d, st, nullptr, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// k_col
// ---------------------------------------------------------------------------------------
template <class T, bool PC>
__device__ __forceinline__ void col_body(const Desc& d, State* __restrict__ st, Slot* slot, int blk,
                                         unsigned char* smem_raw) {
  if (blk >= d.ncomp * d.ncolblk) return;
  if (!PC && !sweep_active(st, slot)) return;

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, logny = d.logny;
  const size_t plane = (size_t)nx * ny;
  const int c = blk / d.ncolblk, cb = blk - c * d.ncolblk;
  const int x0 = cb * d.col_width;
  const int nl = d.col_width >> 1;
  const int lnl = ilog2i(nl);
  const int ls = padded_len(ny);
  T* WY = static_cast<T*>(d.fused ? d.WYb[(*((volatile const int*)&st->n) - 1) & 1] : d.WY) + c * plane;
  const bool per = d.bc == BC_PERIODIC;
  const int hn = ny >> 1, lh = logny - 1;
  const cx<T>* twy;
  const cx<T>* dcy;
  cx<T>* buf = reinterpret_cast<cx<T>*>(place_tables<T>(smem_raw, d.twy, d.dcy, ny, true, !per, twy, dcy));
  cx<T>* scr = (d.fft_pp & 2) ? buf + nl * ls : buf;
  // spectral symbol 1 / (g_hat nx ny), g_hat = (1 + c1 mu + c2 mu^2 + c3 mu^3)^2, mu = mu_x(kx) + mu_y(ky)
  const T* mux = static_cast<const T*>(d.mux);
  const T* muy = static_cast<const T*>(d.muy);
  const T c1 = T(d.gc1[c]), c2 = T(d.gc2[c]), c3 = T(d.gc3[c]), inn = T(d.inv_nn);
  auto sym = [&](T mu) -> T {
    const T g = T(1) + mu * (c1 + mu * (c2 + c3 * mu));
    if constexpr (sizeof(T) == 4) return inn * __frcp_rn(g * g);
    else return inn / (g * g);
  };

  {
    // gather all of this thread's column pairs first, then store them (loads in flight together)
    constexpr int MAXV = 16;
    const int total = ny << lnl;
    for (int base = 0; base < total; base += MAXV * nt) {
      cx<T> v[MAXV];
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int g = base + tid + q * nt;
        if (g < total) v[q] = *reinterpret_cast<const cx<T>*>(WY + (size_t)(g >> lnl) * nx + x0 + 2 * (g & (nl - 1)));
      }
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int g = base + tid + q * nt;
        if (g < total) {
          const int row = g >> lnl, m = g & (nl - 1);
          buf[m * ls + pidx(per ? row : mk_slot(row, ny))] = v[q];
        }
      }
    }
  }
  __syncthreads();
  cx<T>* cur = block_fft<T, -1>(buf, scr, nl, logny, ls, twy, tid, nt, (d.fft_pp & 8) != 0);
  cx<T>* oth = cur == buf ? scr : buf;
  // forward epilogue and the spectral scaling 1 / (g_hat nx ny), in place
  for (int g = tid; g < (nl << lh); g += nt) {
    const int m = g >> lh, k = g & (hn - 1);
    cx<T>* L = cur + m * ls;
    const int col = x0 + 2 * m;
    cx<T> ok, okp;
    fwd_post(L, ny, d.bc, dcy, k, ok, okp);
    const int k2 = k == 0 ? hn : ny - k;
    if (k == 0) {
      cx<T> t;
      fwd_post(L, ny, d.bc, dcy, hn, okp, t);
    }
    const T ma = __ldg(mux + col), mb = __ldg(mux + col + 1);
    const T m1 = __ldg(muy + k), m2 = __ldg(muy + k2);
    L[pidx(k)] = cx<T>{ok.x * sym(ma + m1), ok.y * sym(mb + m1)};
    L[pidx(k2)] = cx<T>{okp.x * sym(ma + m2), okp.y * sym(mb + m2)};
  }
  __syncthreads();
  // The second transform is one forward call for both boundary kinds: the Neumann inverse is
  // the conjugate of the forward transform of the conjugated DCT-III preparation.
  if (!per) {
    for (int g = tid; g < (nl << lh); g += nt) {
      const int m = g >> lh, k = g & (hn - 1);
      cx<T>* L = cur + m * ls;
      const cx<T> w = dcy[k];
      cx<T> zk, zkp;
      if (k == 0) {
        // k = 0 (partner X_N = 0) and the self-paired middle frequency N/2
        dct_inv_pre(L[pidx(0)], cx<T>{T(0), T(0)}, w.x, w.y, zk, zkp);
        const cx<T> Xm = L[pidx(hn)];
        const cx<T> wm = dcy[hn];
        cx<T> zm, zmp;
        dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
        L[pidx(0)] = cx<T>{zk.x, -zk.y};
        L[pidx(hn)] = cx<T>{zm.x, -zm.y};
      } else {
        dct_inv_pre(L[pidx(k)], L[pidx(ny - k)], w.x, w.y, zk, zkp);
        L[pidx(k)] = cx<T>{zk.x, -zk.y};
        L[pidx(ny - k)] = cx<T>{zkp.x, -zkp.y};
      }
    }
    __syncthreads();
  }
  cx<T>* y2 = block_fft<T, -1>(cur, oth, nl, logny, ls, twy, tid, nt, (d.fft_pp & 8) != 0);
  if (per) {
    post_inplace(y2, nl, logny, ls, d.bc, dcy);
    __syncthreads();
#pragma unroll 4
    for (int g = tid; g < (ny << lnl); g += nt) {
      const int row = g >> lnl, m = g & (nl - 1);
      *reinterpret_cast<cx<T>*>(WY + (size_t)row * nx + x0 + 2 * m) = y2[m * ls + pidx(row)];
    }
  } else {
#pragma unroll 4
    for (int g = tid; g < (ny << lnl); g += nt) {
      const int n = g >> lnl, m = g & (nl - 1);
      const cx<T> v = y2[m * ls + pidx(n)];
      *reinterpret_cast<cx<T>*>(WY + (size_t)mk_perm(n, ny) * nx + x0 + 2 * m) = cx<T>{v.x, -v.y};
    }
  }
}

template <class T, bool PC>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value) k_col(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  col_body<T, PC>(d, st, nullptr, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// k_upd
// ---------------------------------------------------------------------------------------
template <class T, int K, bool EDGE, int W>
__device__ __forceinline__ void upd_group(const Desc& d, const cx<T>* buf, int ls, int lpc, int lr, int j0,
                                          T* xa, T* xb, const T* sa, const T* sb) {
  constexpr bool DC = sizeof(T) == 4;
  const T tu = T(d.tau_u);
  const Pairs<T, EDGE> p0{buf, ls, d.nx, d.bc, 0};
  const Pairs<T, EDGE> p1{buf, ls, d.nx, d.bc, lpc};
#pragma unroll
  for (int q = 0; q < W; ++q) {
    T s0 = xa[q], s1 = KT<K>::two ? xb[q] : T(0);
    if constexpr (DC && KT<K>::nonlinear) {
      s0 += sa[q];
      if constexpr (KT<K>::two) s1 += sb[q];
    }
    T g[2] = {T(0), T(0)};
    gradT_pt<T, K>(d, p0, p1, s0, s1, lr, j0 + q, g);
    xa[q] -= tu * g[0];
    if constexpr (KT<K>::two) xb[q] -= tu * g[1];
  }
}

template <class T, int K, int W>
__device__ __forceinline__ void upd_points(const Desc& d, const cx<T>* buf, int y0, int rows, int ls, int lpc) {
  constexpr bool DC = sizeof(T) == 4;
  constexpr int H = KT<K>::H;
  const int nx = d.nx;
  const size_t plane = (size_t)nx * d.ny;
  T* X = static_cast<T*>(d.X);
  const T* Bs = static_cast<const T*>(d.base);
  const int lw = W == 4 ? 2 : (W == 2 ? 1 : 0);
  const int lv = d.lognx - lw;
  constexpr int G = 1;  // one vector group per trip: more unrolled groups cost more in
                        // instruction fetch than they gained in loads in flight (measured)
  const int total = rows << lv;
  for (int base = 0; base < total; base += G * blockDim.x) {
    T xa[G][W], xb[G][W], sa[G][W], sb[G][W];
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int v = base + threadIdx.x + q * blockDim.x;
      if (v < total) {
        const size_t o = (size_t)(y0 + (v >> lv)) * nx + (v & ((1 << lv) - 1)) * W;
        vld<T, W>(X + o, xa[q]);
        if constexpr (KT<K>::two) vld<T, W>(X + plane + o, xb[q]);
        if constexpr (DC && KT<K>::nonlinear) {
          vld<T, W>(Bs + o, sa[q]);
          if constexpr (KT<K>::two) vld<T, W>(Bs + plane + o, sb[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const int v = base + threadIdx.x + q * blockDim.x;
      if (v >= total) break;
      const int r = v >> lv, j0 = (v & ((1 << lv) - 1)) * W;
      const size_t o = (size_t)(y0 + r) * nx + j0;
      // boundary-mapped columns everywhere: one copy of the gradient code, not an interior and
      // an edge copy (the smaller kernel is faster: instruction fetch dominates its stalls)
      upd_group<T, K, true, W>(d, buf, ls, lpc, H + r, j0, xa[q], xb[q], sa[q], sb[q]);
      vst<T, W>(X + o, xa[q]);
      if constexpr (KT<K>::two) vst<T, W>(X + plane + o, xb[q]);
    }
  }
}

template <class T, int K>
__device__ __forceinline__ void upd_body(const Desc& d, State* __restrict__ st, Slot* slot, int band,
                                         unsigned char* smem_raw) {
  constexpr bool PC = K == KK_PCONLY;
  constexpr int H = KT<K>::H;
  const int brows = d.upd_rows ? d.upd_rows : d.band_rows;
  if (band >= (d.upd_rows ? d.nupd : d.nbands)) return;
  if (!PC && !sweep_active(st, slot)) return;

  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, bc = d.bc, lognx = d.lognx;
  const int nc = PC ? d.ncomp : (KT<K>::two ? 2 : 1);
  const size_t plane = (size_t)nx * ny;
  const int y0 = band * brows;
  const int rows = min(brows, ny - y0);
  const int lrows = rows + 2 * H;
  const int lpc = lrows >> 1;
  const int nl = nc * lpc;
  const int ls = padded_len(nx);
  const T* WY = static_cast<const T*>(d.WY);
  const cx<T>* twx;
  const cx<T>* dcx;
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(place_tables<T>(smem_raw, d.twx, d.dcx, nx, d.precond != 0,
                                                         d.precond != 0 && bc == BC_NEUMANN, twx, dcx));
  cx<T>* scr = (d.fft_pp & 4) ? buf0 + nl * ls : buf0;
  cx<T>* buf = buf0;  // the buffer that holds Y (then P~) after the inverse transform
  const int hn = nx >> 1, lh = lognx - 1;
  if (SmemTables<T>::value && d.precond != 0 && bc == BC_NEUMANN) __syncthreads();

  // 1. Y on rows y0-H .. y0+rows+H-1 (boundary-mapped) into buf, two rows per line.  Both
  //    boundary kinds use the same (forward) transform call: the Neumann input is the conjugated
  //    DCT-III preparation, and the conjugate of its forward transform is the inverse transform.
  if (d.precond == 0 || bc == BC_PERIODIC) {
#pragma unroll 2
    for (int g = tid; g < (nl << lh); g += nt) {
      const int line = g >> lh, j = 2 * (g & (hn - 1));
      const int c = (PC ? nc > 1 : KT<K>::two) ? line / lpc : 0, m = line - c * lpc;
      const int ga = bcmap(y0 - H + 2 * m, ny, bc), gb = bcmap(y0 - H + 2 * m + 1, ny, bc);
      const T* Wc = WY + c * plane;
      const cx<T> a = *reinterpret_cast<const cx<T>*>(Wc + (size_t)ga * nx + j);
      const cx<T> b = *reinterpret_cast<const cx<T>*>(Wc + (size_t)gb * nx + j);
      buf0[line * ls + pidx(j)] = cx<T>{a.x, b.x};
      buf0[line * ls + pidx(j + 1)] = cx<T>{a.y, b.y};
    }
  } else {
    for (int g = tid; g < (nl << lh); g += nt) {
      const int line = g >> lh, k = g & (hn - 1);
      const int c = (PC ? nc > 1 : KT<K>::two) ? line / lpc : 0, m = line - c * lpc;
      const int ga = bcmap(y0 - H + 2 * m, ny, bc), gb = bcmap(y0 - H + 2 * m + 1, ny, bc);
      const T* Wa = WY + c * plane + (size_t)ga * nx;
      const T* Wb = WY + c * plane + (size_t)gb * nx;
      cx<T>* L = buf0 + line * ls;
      const cx<T> w = dcx[k];
      cx<T> zk, zkp;
      if (k == 0) {
        dct_inv_pre(cx<T>{Wa[0], Wb[0]}, cx<T>{T(0), T(0)}, w.x, w.y, zk, zkp);
        const cx<T> Xm{Wa[hn], Wb[hn]};
        const cx<T> wm = dcx[hn];
        cx<T> zm, zmp;
        dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
        L[pidx(0)] = cx<T>{zk.x, -zk.y};
        L[pidx(hn)] = cx<T>{zm.x, -zm.y};
      } else {
        dct_inv_pre(cx<T>{Wa[k], Wb[k]}, cx<T>{Wa[nx - k], Wb[nx - k]}, w.x, w.y, zk, zkp);
        L[pidx(k)] = cx<T>{zk.x, -zk.y};
        L[pidx(nx - k)] = cx<T>{zkp.x, -zkp.y};
      }
    }
  }
  __syncthreads();
  if (d.precond != 0) {
    buf = block_fft<T, -1>(buf0, scr, nl, lognx, ls, twx, tid, nt, (d.fft_pp & 8) != 0);
    if (bc == BC_PERIODIC) {
      post_inplace(buf, nl, lognx, ls, bc, dcx);
      __syncthreads();
    } else {
    // undo the conjugation and the Makhoul reordering in place (slot n holds column
    // mk_perm(n)), in chunks of lines so that each thread holds at most 16 values between the
    // two barriers
    {
      constexpr int MAXV = 16;
      int chunk = (nt * MAXV) >> lognx;
      if (chunk < 1) chunk = 1;
      for (int l0 = 0; l0 < nl; l0 += chunk) {
        const int cl = nl - l0 < chunk ? nl - l0 : chunk;
        const int total = cl << lognx;
        const int nthr = (total + MAXV - 1) / MAXV;
        cx<T> v[MAXV];
#pragma unroll
        for (int s = 0; s < MAXV; ++s) {
          const int g = tid + s * nthr;
          if (tid < nthr && g < total) {
            const cx<T> e = buf[(l0 + (g >> lognx)) * ls + pidx(g & (nx - 1))];
            v[s] = cx<T>{e.x, -e.y};
          }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < MAXV; ++s) {
          const int g = tid + s * nthr;
          if (tid < nthr && g < total)
            buf[(l0 + (g >> lognx)) * ls + pidx(mk_perm(g & (nx - 1), nx))] = v[s];
        }
        __syncthreads();
      }
    }
    }
  }

  if constexpr (PC) {
    T* X = static_cast<T*>(d.X);
    const int rl = rows >> 1;
    for (int g = tid; g < ((nc * rl) << lh); g += nt) {
      const int line = g >> lh, j = 2 * (g & (hn - 1));
      const int c = line / rl, m = line - c * rl;
      const cx<T> e0 = buf[(c * lpc + m) * ls + pidx(j)], e1 = buf[(c * lpc + m) * ls + pidx(j + 1)];
      T* Xa = X + c * plane + (size_t)(y0 + 2 * m) * nx + j;
      *reinterpret_cast<cx<T>*>(Xa) = cx<T>{e0.x, e1.x};
      *reinterpret_cast<cx<T>*>(Xa + nx) = cx<T>{e0.y, e1.y};
    }
    return;
  } else {
    // 2. P~ = P_n + (1 + omega) tau_p Y on all local rows (in place in buf);
    //    P_{n+1} = P_n + tau_p Y on the band rows.  Each thread owns two slots of a line.
    const int n = st->n;  // already counts this update
    const T* Pin = static_cast<const T*>(d.P[(n - 1) & 1]);
    T* Pout = static_cast<T*>(d.P[n & 1]);
    const T tp = T(d.tau_p), tpe = T((1.0 + d.omega) * d.tau_p);
    constexpr int G = 2;  // slot pairs whose P values are loaded together (2: measured best)
    const int totalp = nl << lh;
    for (int base = 0; base < totalp; base += G * nt) {
     cx<T> pag[G], pbg[G];
#pragma unroll
     for (int q = 0; q < G; ++q) {
      const int g = base + tid + q * nt;
      if (g < totalp) {
        const int line = g >> lh, j = 2 * (g & (hn - 1));
        const int c = (PC ? nc > 1 : KT<K>::two) ? line / lpc : 0, m = line - c * lpc;
        pag[q] = *reinterpret_cast<const cx<T>*>(Pin + c * plane + (size_t)bcmap(y0 - H + 2 * m, ny, bc) * nx + j);
        pbg[q] = *reinterpret_cast<const cx<T>*>(Pin + c * plane + (size_t)bcmap(y0 - H + 2 * m + 1, ny, bc) * nx + j);
      }
     }
#pragma unroll
     for (int q = 0; q < G; ++q) {
      const int g = base + tid + q * nt;
      if (g >= totalp) break;
      const int line = g >> lh, j = 2 * (g & (hn - 1));
      const int c = (PC ? nc > 1 : KT<K>::two) ? line / lpc : 0, m = line - c * lpc;
      const int la = 2 * m, lb = 2 * m + 1;
      const size_t oa = c * plane + (size_t)bcmap(y0 - H + la, ny, bc) * nx + j;
      const size_t ob = c * plane + (size_t)bcmap(y0 - H + lb, ny, bc) * nx + j;
      const cx<T> pa = pag[q];
      const cx<T> pb = pbg[q];
      cx<T>* s0 = buf + line * ls + pidx(j);
      cx<T>* s1 = buf + line * ls + pidx(j + 1);
      const cx<T> y0v = *s0, y1v = *s1;  // (row a, row b) at columns j, j+1
      *s0 = cx<T>{pa.x + tpe * y0v.x, pb.x + tpe * y0v.y};
      *s1 = cx<T>{pa.y + tpe * y1v.x, pb.y + tpe * y1v.y};
      if (la >= H && la < H + rows) *reinterpret_cast<cx<T>*>(Pout + oa) = cx<T>{pa.x + tp * y0v.x, pa.y + tp * y1v.x};
      if (lb >= H && lb < H + rows) *reinterpret_cast<cx<T>*>(Pout + ob) = cx<T>{pb.x + tp * y0v.y, pb.y + tp * y1v.y};
     }
    }
    __syncthreads();

    // 3. U_{n+1} = U_n - tau_u dF(U_n)^T P~ on band rows
    if (nx >= V16<T>::n) upd_points<T, K, V16<T>::n>(d, buf, y0, rows, ls, lpc);
    else upd_points<T, K, 1>(d, buf, y0, rows, ls, lpc);
  }
}

// ---------------------------------------------------------------------------------------
// k_updres: update n of the PDHG iteration fused with the residual of the next one
// ---------------------------------------------------------------------------------------

// U_{n+1} on rows y0-H .. y0+rows+H-1 of one band from P~ (in buf, rows y0-2H .. y0+rows+2H-1):
// band rows read U_n from X and write U_{n+1} back; halo rows read and write this block's own
// copy in d.halo; every row also goes to the staging rows xs for the residual.
template <class T, int K, int W>
__device__ __forceinline__ void updres_points(const Desc& d, const cx<T>* buf, T* xs, int band, int y0, int rows,
                                              int ls, int lpc) {
  constexpr bool DC = sizeof(T) == 4;
  constexpr int H = KT<K>::H;
  constexpr int HY = 2 * H;
  const int nx = d.nx, ny = d.ny, bc = d.bc;
  const int nc = KT<K>::two ? 2 : 1;
  const size_t plane = (size_t)nx * ny;
  const int srows = rows + 2 * H;
  T* X = static_cast<T*>(d.X);
  T* Hb = static_cast<T*>(d.halo) + (size_t)band * nc * 2 * H * nx;
  const T* Bs = static_cast<const T*>(d.base);
  const int lw = W == 4 ? 2 : (W == 2 ? 1 : 0);
  const int lv = d.lognx - lw;
  const int total = srows << lv;
  for (int v = threadIdx.x; v < total; v += blockDim.x) {
    const int r = (v >> lv) - H;  // -H .. rows+H-1
    const int j0 = (v & ((1 << lv) - 1)) * W;
    const bool own = r >= 0 && r < rows;
    const int slot = r < 0 ? r + H : r - rows + H;  // halo slot 0 .. 2H-1
    T* u0 = own ? X + (size_t)(y0 + r) * nx + j0 : Hb + (size_t)slot * nx + j0;
    T* u1 = own ? u0 + plane : Hb + (size_t)(2 * H + slot) * nx + j0;
    T xa[W], xb[W], sa[W], sb[W];
    vld<T, W>(u0, xa);
    if constexpr (KT<K>::two) vld<T, W>(u1, xb);
    if constexpr (DC && KT<K>::nonlinear) {
      const size_t ob = (size_t)bcmap(y0 + r, ny, bc) * nx + j0;
      vld<T, W>(Bs + ob, sa);
      if constexpr (KT<K>::two) vld<T, W>(Bs + plane + ob, sb);
    }
    upd_group<T, K, true, W>(d, buf, ls, lpc, HY + r, j0, xa, xb, sa, sb);
    vst<T, W>(u0, xa);
    if constexpr (KT<K>::two) vst<T, W>(u1, xb);
    T* x0 = xs + (size_t)(r + H) * nx + j0;
#pragma unroll
    for (int q = 0; q < W; ++q) x0[q] = xa[q];
    if constexpr (KT<K>::two) {
#pragma unroll
      for (int q = 0; q < W; ++q) x0[(size_t)srows * nx + q] = xb[q];
    }
  }
}

// One band of update n (the P and U updates of k_upd, with the transform spectrum and P~ on a
// halo of 2H rows so that U_{n+1} is known on H halo rows) followed by the residual of update
// n+1 on the band (k_res on the staged U_{n+1}: W = F(U_{n+1}), forward row transform into the
// other transform buffer, norm partials, stopping decision).  FP32 defect correction with a
// spectral preconditioner only.
template <class T, int K>
__device__ __forceinline__ void updres_body(const Desc& d, State* __restrict__ st, int band, unsigned char* smem_raw) {
  constexpr int H = KT<K>::H;
  constexpr int HY = 2 * H;
  if (band >= d.nupd) return;

  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = d.nx, ny = d.ny, bc = d.bc, lognx = d.lognx;
  const int nc = KT<K>::two ? 2 : 1;
  const size_t plane = (size_t)nx * ny;
  const int y0 = band * d.upd_rows;
  const int rows = min(d.upd_rows, ny - y0);
  const int lrows = rows + 2 * HY;
  const int lpc = lrows >> 1;
  const int nl = nc * lpc;
  const int ls = padded_len(nx);
  const cx<T>* twx;
  const cx<T>* dcx;
  cx<T>* buf = reinterpret_cast<cx<T>*>(place_tables<T>(smem_raw, d.twx, d.dcx, nx, true, bc == BC_NEUMANN, twx, dcx));
  T* xs = reinterpret_cast<T*>(buf + nl * ls);
  T* bs = xs + nc * (rows + 2 * H) * nx;
  const int hn = nx >> 1, lh = lognx - 1;
  if (!sweep_active(st, nullptr)) return;
  const int n = *((volatile const int*)&st->n);  // already counts this update
  const T* WY = static_cast<const T*>(d.WYb[(n - 1) & 1]);
  T* Wout = static_cast<T*>(d.WYb[n & 1]);
  if constexpr (sizeof(T) == 4 && base_stencil<K>()) {
    const T* Bg = static_cast<const T*>(d.base);
    for (int c = 0; c < nc; ++c)
      stage_rows<T>(bs + c * (rows + 2 * H) * nx, Bg + c * plane, nx, lognx, ny, bc, y0 - H, rows + 2 * H);
  }
  if (SmemTables<T>::value && bc == BC_NEUMANN) __syncthreads();

  // 1. the spectrum rows y0-2H .. y0+rows+2H-1 into buf, two rows per line (as k_upd)
  if (bc == BC_PERIODIC) {
    for (int g = tid; g < (nl << lh); g += nt) {
      const int line = g >> lh, j = 2 * (g & (hn - 1));
      const int c = KT<K>::two ? line / lpc : 0, m = line - c * lpc;
      const int ga = bcmap(y0 - HY + 2 * m, ny, bc), gb = bcmap(y0 - HY + 2 * m + 1, ny, bc);
      const T* Wc = WY + c * plane;
      const cx<T> a = ld_pair(Wc + (size_t)ga * nx + j);
      const cx<T> b = ld_pair(Wc + (size_t)gb * nx + j);
      buf[line * ls + pidx(j)] = cx<T>{a.x, b.x};
      buf[line * ls + pidx(j + 1)] = cx<T>{a.y, b.y};
    }
  } else {
    for (int g = tid; g < (nl << lh); g += nt) {
      const int line = g >> lh, k = g & (hn - 1);
      const int c = KT<K>::two ? line / lpc : 0, m = line - c * lpc;
      const int ga = bcmap(y0 - HY + 2 * m, ny, bc), gb = bcmap(y0 - HY + 2 * m + 1, ny, bc);
      const T* Wa = WY + c * plane + (size_t)ga * nx;
      const T* Wb = WY + c * plane + (size_t)gb * nx;
      cx<T>* L = buf + line * ls;
      const cx<T> w = dcx[k];
      cx<T> zk, zkp;
      if (k == 0) {
        dct_inv_pre(cx<T>{Wa[0], Wb[0]}, cx<T>{T(0), T(0)}, w.x, w.y, zk, zkp);
        const cx<T> Xm{Wa[hn], Wb[hn]};
        const cx<T> wm = dcx[hn];
        cx<T> zm, zmp;
        dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
        L[pidx(0)] = cx<T>{zk.x, -zk.y};
        L[pidx(hn)] = cx<T>{zm.x, -zm.y};
      } else {
        dct_inv_pre(cx<T>{Wa[k], Wb[k]}, cx<T>{Wa[nx - k], Wb[nx - k]}, w.x, w.y, zk, zkp);
        L[pidx(k)] = cx<T>{zk.x, -zk.y};
        L[pidx(nx - k)] = cx<T>{zkp.x, -zkp.y};
      }
    }
  }
  __syncthreads();
  // inverse row transform (the forward transform, conjugated for Neumann), in place
  {
    cx<T>* r = block_fft<T, -1>(buf, buf, nl, lognx, ls, twx, tid, nt, (d.fft_pp & 8) != 0);
    if (bc == BC_PERIODIC) {
      post_inplace(r, nl, lognx, ls, bc, dcx);
      __syncthreads();
    } else {
      constexpr int MAXV = 16;
      int chunk = (nt * MAXV) >> lognx;
      if (chunk < 1) chunk = 1;
      for (int l0 = 0; l0 < nl; l0 += chunk) {
        const int cl = nl - l0 < chunk ? nl - l0 : chunk;
        const int total = cl << lognx;
        const int nthr = (total + MAXV - 1) / MAXV;
        cx<T> v[MAXV];
#pragma unroll
        for (int q = 0; q < MAXV; ++q) {
          const int g = tid + q * nthr;
          if (tid < nthr && g < total) {
            const cx<T> e = r[(l0 + (g >> lognx)) * ls + pidx(g & (nx - 1))];
            v[q] = cx<T>{e.x, -e.y};
          }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXV; ++q) {
          const int g = tid + q * nthr;
          if (tid < nthr && g < total) r[(l0 + (g >> lognx)) * ls + pidx(mk_perm(g & (nx - 1), nx))] = v[q];
        }
        __syncthreads();
      }
    }
  }

  // 2. P~ = P_n + (1 + omega) tau_p Y on all local rows (in place); P_{n+1} on the band rows
  {
    const T* Pin = static_cast<const T*>(d.P[(n - 1) & 1]);
    T* Pout = static_cast<T*>(d.P[n & 1]);
    const T tp = T(d.tau_p), tpe = T((1.0 + d.omega) * d.tau_p);
    for (int g = tid; g < (nl << lh); g += nt) {
      const int line = g >> lh, j = 2 * (g & (hn - 1));
      const int c = KT<K>::two ? line / lpc : 0, m = line - c * lpc;
      const int la = 2 * m, lb = 2 * m + 1;
      const size_t oa = c * plane + (size_t)bcmap(y0 - HY + la, ny, bc) * nx + j;
      const size_t ob = c * plane + (size_t)bcmap(y0 - HY + lb, ny, bc) * nx + j;
      const cx<T> pa = ld_pair(Pin + oa);
      const cx<T> pb = ld_pair(Pin + ob);
      cx<T>* s0 = buf + line * ls + pidx(j);
      cx<T>* s1 = buf + line * ls + pidx(j + 1);
      const cx<T> y0v = *s0, y1v = *s1;
      *s0 = cx<T>{pa.x + tpe * y0v.x, pb.x + tpe * y0v.y};
      *s1 = cx<T>{pa.y + tpe * y1v.x, pb.y + tpe * y1v.y};
      if (la >= HY && la < HY + rows) *reinterpret_cast<cx<T>*>(Pout + oa) = cx<T>{pa.x + tp * y0v.x, pa.y + tp * y1v.x};
      if (lb >= HY && lb < HY + rows) *reinterpret_cast<cx<T>*>(Pout + ob) = cx<T>{pb.x + tp * y0v.y, pb.y + tp * y1v.y};
    }
  }
  __syncthreads();

  // 3. U_{n+1} on the band and H halo rows, staged in xs
  if (nx >= V16<T>::n) updres_points<T, K, V16<T>::n>(d, buf, xs, band, y0, rows, ls, lpc);
  else updres_points<T, K, 1>(d, buf, xs, band, y0, rows, ls, lpc);
  __syncthreads();

  // 4. W = F(U_{n+1}) on the band rows into buf (now free), forward row transform into Wout
  T acc0 = T(0), acc1 = T(0);
  if (nx >= V16<T>::n) res_points<T, K, V16<T>::n>(d, buf, xs, bs, y0, rows, ls, acc0, acc1);
  else res_points<T, K, 1>(d, buf, xs, bs, y0, rows, ls, acc0, acc1);
  __syncthreads();
  {
    const int rl = rows >> 1;
    const cx<T>* res = block_fft<T, -1>(buf, buf, nc * rl, lognx, ls, twx, tid, nt, (d.fft_pp & 8) != 0);
    for (int g = tid; g < ((nc * rl) << lh); g += nt) {
      const int line = g >> lh, k = g & (hn - 1);
      const int c = KT<K>::two ? line / rl : 0, m = line - c * rl;
      const cx<T>* L = res + line * ls;
      T* Wa = Wout + c * plane + (size_t)(y0 + 2 * m) * nx;
      T* Wb = Wa + nx;
      cx<T> ok, okp;
      fwd_post(L, nx, bc, dcx, k, ok, okp);
      Wa[k] = ok.x;
      Wb[k] = ok.y;
      if (k != 0) {
        Wa[nx - k] = okp.x;
        Wb[nx - k] = okp.y;
      } else {
        fwd_post(L, nx, bc, dcx, hn, ok, okp);
        Wa[hn] = ok.x;
        Wb[hn] = ok.y;
      }
    }
  }

  // 5. partial norms of F(U_{n+1}), ticket, stopping decision in the last block
  const double s0 = block_sum((double)acc0, red);
  const double s1 = KT<K>::two ? block_sum((double)acc1, red) : 0.0;
  if (tid == 0) {
    d.partials[band] = s0;
    if (KT<K>::two) d.partials[d.nupd + band] = s1;
  }
  if (last_block(st, d.nupd)) finalize_measure(d, st, red, nullptr, d.nupd);
}

template <class T, int K>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value) k_updres(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  updres_body<T, K>(d, st, blockIdx.x, smem_raw);
}

template <class T, int K>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value) k_upd(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  upd_body<T, K>(d, st, nullptr, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
template <class K_>
static cudaError_t allow_smem_k(K_ kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// Event-record flags for ev on stream s: inside a stream capture the events become external
// event-record nodes of the graph; outside one they are ordinary records (the external flag is
// for capture only).
static inline cudaError_t record_flags(cudaStream_t s, const cudaEvent_t* ev, unsigned* flags) {
  *flags = cudaEventRecordDefault;
  if (!ev) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e == cudaSuccess && cs == cudaStreamCaptureStatusActive) *flags = cudaEventRecordExternal;
  return e;
}

template <class T, int K>
static cudaError_t launch_iter_k(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev) {
  constexpr bool PC = K == KK_PCONLY;
  unsigned flags;
  cudaError_t e = record_flags(s, ev, &flags);
  if (e != cudaSuccess) return e;
  auto mark = [&](int i) {
    if (ev && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[i], s, flags);
  };
  mark(0);
  k_res<T, K><<<c.grid_bands, c.thr_res, c.smem_res, s>>>(d, st);
  mark(1);
  if (c.transform && e == cudaSuccess) e = launch_col<T>(d, st, c, s, PC);
  mark(2);
  k_upd<T, K><<<c.grid_upd ? c.grid_upd : c.grid_bands, c.thr_upd, c.smem_upd, s>>>(d, st);
  mark(3);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// One PDHG iteration with the fused update: first = true launches k_res, k_col and k_updres (the
// residual of U_0 comes first), first = false k_col and k_updres.  Events as in launch_iter_k.
template <int K>
static cudaError_t launch_fused_k(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev,
                                  bool first) {
  unsigned flags;
  cudaError_t e = record_flags(s, ev, &flags);
  if (e != cudaSuccess) return e;
  auto mark = [&](int i) {
    if (ev && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[i], s, flags);
  };
  mark(0);
  if (first && e == cudaSuccess) e = launch_res<float, K>(d, st, c, s);
  mark(1);
  if (e == cudaSuccess) e = launch_col<float>(d, st, c, s, false);
  mark(2);
  k_updres<float, K><<<c.grid_upd ? c.grid_upd : c.grid_bands, c.thr_updres, c.smem_updres, s>>>(d, st);
  mark(3);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// The kernels of one equation key K in arithmetic T: its iteration launcher, its k_res launcher
// (for the fused iteration, whose k_res instance must be the one whose limits were raised) and
// the shared-memory limits of k_res and k_upd.  One unit per group of keys, compiled in parallel.
#define RD_SWEEP_KIND(T, K)                                                                            \
  template <>                                                                                          \
  cudaError_t launch_iter_kind<T, K>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s,    \
                                     cudaEvent_t* ev) {                                                \
    return launch_iter_k<T, K>(d, st, c, s, ev);                                                       \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t launch_res<T, K>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s) {         \
    k_res<T, K><<<c.grid_bands, c.thr_res, c.smem_res, s>>>(d, st);                                    \
    return cudaGetLastError();                                                                         \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t allow_kind<T, K>(int optin) {                                                            \
    cudaError_t e = allow_smem_k(k_res<T, K>, optin);                                                  \
    return e != cudaSuccess ? e : allow_smem_k(k_upd<T, K>, optin);                                    \
  }

// The fused update kernel of equation key K (FP32 inner solve only).
#define RD_FUSED_KIND(K)                                                                               \
  template <>                                                                                          \
  cudaError_t launch_fused_kind<K>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s,      \
                                   cudaEvent_t* ev, bool first) {                                      \
    return launch_fused_k<K>(d, st, c, s, ev, first);                                                  \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t allow_fused_kind<K>(int optin) {                                                         \
    return allow_smem_k(k_updres<float, K>, optin);                                                    \
  }

// k_col and the per-key dispatch of arithmetic T.
#define RD_SWEEP_COMMON(T)                                                                             \
  template <>                                                                                          \
  cudaError_t launch_col<T>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, bool pc) {   \
    if (pc) k_col<T, true><<<c.grid_cols, c.thr_col, c.smem_col, s>>>(d, st);                          \
    else k_col<T, false><<<c.grid_cols, c.thr_col, c.smem_col, s>>>(d, st);                            \
    return cudaGetLastError();                                                                         \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t launch_iteration<T>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s,         \
                                  cudaEvent_t* ev) {                                                   \
    switch (kind_key(d)) {                                                                             \
      case KK_NONE_LAP: return launch_iter_kind<T, KK_NONE_LAP>(d, st, c, s, ev);                      \
      case KK_AC: return launch_iter_kind<T, KK_AC>(d, st, c, s, ev);                                  \
      case KK_CH_IMPL: return launch_iter_kind<T, KK_CH_IMPL>(d, st, c, s, ev);                        \
      case KK_CH_SPLIT: return launch_iter_kind<T, KK_CH_SPLIT>(d, st, c, s, ev);                      \
      case KK_GS: return launch_iter_kind<T, KK_GS>(d, st, c, s, ev);                                  \
      case KK_SCHNAK: return launch_iter_kind<T, KK_SCHNAK>(d, st, c, s, ev);                          \
      case KK_NONE_BIH: return launch_iter_kind<T, KK_NONE_BIH>(d, st, c, s, ev);                      \
      default: return launch_iter_kind<T, KK_PCONLY>(d, st, c, s, ev);                                 \
    }                                                                                                  \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t set_kernel_smem_limits<T>(int* usable) {                                                 \
    int dev = 0, optin = 0;                                                                            \
    cudaError_t e;                                                                                     \
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;                                            \
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) \
      return e;                                                                                        \
    if ((e = allow_kind<T, KK_NONE_LAP>(optin)) != cudaSuccess) return e;                              \
    if ((e = allow_kind<T, KK_AC>(optin)) != cudaSuccess) return e;                                    \
    if ((e = allow_kind<T, KK_CH_IMPL>(optin)) != cudaSuccess) return e;                               \
    if ((e = allow_kind<T, KK_CH_SPLIT>(optin)) != cudaSuccess) return e;                              \
    if ((e = allow_kind<T, KK_GS>(optin)) != cudaSuccess) return e;                                    \
    if ((e = allow_kind<T, KK_SCHNAK>(optin)) != cudaSuccess) return e;                                \
    if ((e = allow_kind<T, KK_NONE_BIH>(optin)) != cudaSuccess) return e;                              \
    if ((e = allow_kind<T, KK_PCONLY>(optin)) != cudaSuccess) return e;                                \
    if ((e = allow_smem_k(k_col<T, false>, optin)) != cudaSuccess) return e;                           \
    if ((e = allow_smem_k(k_col<T, true>, optin)) != cudaSuccess) return e;                            \
    if constexpr (sizeof(T) == 4) {                                                                    \
      if ((e = allow_fused_kind<KK_NONE_LAP>(optin)) != cudaSuccess) return e;                         \
      if ((e = allow_fused_kind<KK_AC>(optin)) != cudaSuccess) return e;                               \
      if ((e = allow_fused_kind<KK_CH_IMPL>(optin)) != cudaSuccess) return e;                          \
      if ((e = allow_fused_kind<KK_CH_SPLIT>(optin)) != cudaSuccess) return e;                         \
      if ((e = allow_fused_kind<KK_GS>(optin)) != cudaSuccess) return e;                               \
      if ((e = allow_fused_kind<KK_SCHNAK>(optin)) != cudaSuccess) return e;                           \
      if ((e = allow_fused_kind<KK_NONE_BIH>(optin)) != cudaSuccess) return e;                         \
    }                                                                                                  \
    if (usable) *usable = optin - 1024;                                                                \
    return cudaSuccess;                                                                                \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t launch_fused<T>(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev, \
                              bool first) {                                                            \
    if constexpr (sizeof(T) != 4) return cudaErrorNotSupported;                                        \
    switch (kind_key(d)) {                                                                             \
      case KK_NONE_LAP: return launch_fused_kind<KK_NONE_LAP>(d, st, c, s, ev, first);                 \
      case KK_AC: return launch_fused_kind<KK_AC>(d, st, c, s, ev, first);                             \
      case KK_CH_IMPL: return launch_fused_kind<KK_CH_IMPL>(d, st, c, s, ev, first);                   \
      case KK_CH_SPLIT: return launch_fused_kind<KK_CH_SPLIT>(d, st, c, s, ev, first);                 \
      case KK_GS: return launch_fused_kind<KK_GS>(d, st, c, s, ev, first);                             \
      case KK_SCHNAK: return launch_fused_kind<KK_SCHNAK>(d, st, c, s, ev, first);                     \
      case KK_NONE_BIH: return launch_fused_kind<KK_NONE_BIH>(d, st, c, s, ev, first);                 \
      default: return cudaErrorNotSupported;                                                           \
    }                                                                                                  \
  }

}  // namespace rd
