// Device code of the PDHG iteration on 3-D grids (the paper's scheme, Section 2.1 and
// Algorithm 1, with a third axis: the seven-point Laplacian, Lap^2 as its square, and the
// separable Hartley (periodic) / DCT-II (Neumann) transforms along x, y and z that diagonalise
// it).  Arrays are [ncomp][nz][ny][nx], x contiguous; scalar equations only.
//
// One iteration is seven kernels, each running d.blk3 blocks per instance in a grid-stride loop
// over its work (points, or tiles of lines), so that a batched instance does the same work in the
// same order whatever else shares the launch:
//   k3_res    W = F(U_n) point by point from the stencils in global memory (L2-resident at the
//             grid sizes served), the norm partials and, in the last block, the stopping
//             decision ||Res(U_n)||_2 <= delta (Section 2.1);
//   lines x   forward transform along x of W (rows, two per complex line);
//   lines y   forward transform along y (tiles of adjacent x columns);
//   lines z   forward transform along z, multiplication by 1 / (g_hat nx ny nz), inverse along z;
//   lines y   inverse along y;
//   lines x   inverse along x, then the dual update P_{n+1} = P_n + tau_p Y and the extrapolation
//             P~ = P_n + (1 + omega) tau_p Y (eqs. G-prox ... dynamic 1-2), P~ kept in W's buffer;
//   k3_upd    U_{n+1} = U_n - tau_u dF(U_n)^T P~ (eq. G-prox ... dynamic 3).
#pragma once

#include "rd_sweep.cuh"

namespace rd {

// one component of a 3-D grid array in global memory, boundary-mapped on every axis; a 2-D grid
// run on these kernels has nz = 1, and every z offset maps to its one plane (the descriptor's
// hz2 = 0 removes the z terms of the stencils)
template <class T>
struct G3 {
  const T* __restrict__ p;
  int nx, ny, nz, bc;
  __device__ __forceinline__ T operator()(int l, int i, int j) const {
    const int lz = nz > 1 ? bcmap(l, nz, bc) : 0;
    return p[((size_t)lz * ny + bcmap(i, ny, bc)) * nx + bcmap(j, nx, bc)];
  }
};

// The same array read at y and z offsets from one point's row (l0, i0) without boundary mapping,
// for rows whose stencil rows and planes all lie inside the grid, and with the x index mapped;
// pz = 0 on a 2-D grid (nz = 1), where every z offset maps to the point's own plane.  The test
// for it depends only on the row, so that a warp (32 consecutive points of one row when
// nx >= 32) takes one path.
template <class T>
struct G3r {
  const T* __restrict__ p;  // element (l0, i0, 0)
  int l0, i0, nx, bc;
  long pz;                  // elements per z plane (0 when nz = 1)
  __device__ __forceinline__ T operator()(int l, int i, int j) const {
    return p[(long)(l - l0) * pz + (long)(i - i0) * nx + bcmap(j, nx, bc)];
  }
};

// Asynchronous copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory by the whole block, 16 bytes per copy (cp.async, completion awaited by
// cp_async_wait_all and a block barrier).
__device__ __forceinline__ void cp_async_block(void* smem_dst, const void* gsrc, int bytes) {
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(smem_dst);
  const char* g0 = static_cast<const char*>(gsrc);
  for (int o = 16 * threadIdx.x; o < bytes; o += 16 * blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0 + o), "l"(g0 + o) : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Do the rows and planes of a radius-R stencil around row (l, i) lie inside the grid?
template <int R>
__device__ __forceinline__ bool inside_yz(const Desc& d, int l, int i) {
  return i >= R && i < d.ny - R && (d.nz == 1 || (l >= R && l < d.nz - R));
}
// stencil radius of the residual / adjoint of equation key K (13-point biharmonic: 2)
template <int K>
__device__ __forceinline__ constexpr int radius3() {
  return (K == KK_NONE_LAP || K == KK_AC) ? 1 : 2;
}

// seven-point Laplacian at (l, i, j) with centre value c
template <class T, class F>
__device__ __forceinline__ T lap7(const F& f, int l, int i, int j, T c, T hx2, T hy2, T hz2) {
  return (f(l, i, j + 1) + f(l, i, j - 1) - T(2) * c) * hx2 + (f(l, i + 1, j) + f(l, i - 1, j) - T(2) * c) * hy2 +
         (f(l + 1, i, j) + f(l - 1, i, j) - T(2) * c) * hz2;
}

// Lap^2 = sum_{a,b} D_aa D_bb on the periodic / two-deep mirror extension (25 points)
template <class T, class F>
__device__ __forceinline__ T lap25(const F& f, int l, int i, int j, T c, T hx2, T hy2, T hz2) {
  const T e = f(l, i, j + 1), w = f(l, i, j - 1), n = f(l, i + 1, j), s = f(l, i - 1, j);
  const T u = f(l + 1, i, j), dn = f(l - 1, i, j);
  const T xx = f(l, i, j + 2) - T(4) * (e + w) + T(6) * c + f(l, i, j - 2);
  const T yy = f(l, i + 2, j) - T(4) * (n + s) + T(6) * c + f(l, i - 2, j);
  const T zz = f(l + 2, i, j) - T(4) * (u + dn) + T(6) * c + f(l - 2, i, j);
  const T xy = f(l, i + 1, j + 1) + f(l, i + 1, j - 1) + f(l, i - 1, j + 1) + f(l, i - 1, j - 1) -
               T(2) * (e + w + n + s) + T(4) * c;
  const T xz = f(l + 1, i, j + 1) + f(l + 1, i, j - 1) + f(l - 1, i, j + 1) + f(l - 1, i, j - 1) -
               T(2) * (e + w + u + dn) + T(4) * c;
  const T yz = f(l + 1, i + 1, j) + f(l + 1, i - 1, j) + f(l - 1, i + 1, j) + f(l - 1, i - 1, j) -
               T(2) * (n + s + u + dn) + T(4) * c;
  return xx * (hx2 * hx2) + yy * (hy2 * hy2) + zz * (hz2 * hz2) +
         T(2) * (xy * (hx2 * hy2) + xz * (hx2 * hz2) + yz * (hy2 * hz2));
}

// W = F(X) at one point (scalar kinds; see the residual maps in rd_pdhg.h):
//   plain (DC = false): X = U, r = rhs of the step;
//   DC    (DC = true) : X = d, B = u, r = F(u); returns F(u + d) with the nonlinear increment
//                       expanded so that no large terms cancel.
template <class T, int K, bool DC, class A, class B>
__device__ __forceinline__ T residual3_pt(const Desc& d, const A& x, const B& bs, int l, int i, int j, T r) {
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), hz2 = T(d.hz2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const T c0 = x(l, i, j);
  if constexpr (K == KK_NONE_LAP || K == KK_NONE_BIH) {
    const T lin = K == KK_NONE_LAP ? c0 - dt * a * lap7(x, l, i, j, c0, hx2, hy2, hz2)
                                   : c0 + dt * a * lap25(x, l, i, j, c0, hx2, hy2, hz2);
    return DC ? r + lin : lin - r;
  } else if constexpr (K == KK_AC) {
    const T lin = c0 - dt * a * lap7(x, l, i, j, c0, hx2, hy2, hz2);
    if constexpr (!DC) {
      return lin - r + dt * b * (c0 * c0 * c0 - c0);
    } else {
      const T u = bs(l, i, j);
      return r + lin + dt * b * (c0 * (T(3) * u * u - T(1)) + c0 * c0 * (T(3) * u + c0));
    }
  } else {  // Cahn-Hilliard, fully implicit or convex split
    const T lin = c0 + dt * a * lap25(x, l, i, j, c0, hx2, hy2, hz2);
    constexpr T sh = K == KK_CH_IMPL ? T(1) : T(0);
    auto q = [&](int ll, int ii, int jj) -> T {
      const T xv = x(ll, ii, jj);
      if constexpr (!DC) {
        return xv * xv * xv - sh * xv;
      } else {
        const T u = bs(ll, ii, jj);
        return xv * (T(3) * u * u - sh) + xv * xv * (T(3) * u + xv);
      }
    };
    const T lq = lap7(q, l, i, j, q(l, i, j), hx2, hy2, hz2);
    return DC ? r + lin - dt * b * lq : lin - r - dt * b * lq;
  }
}

// dF(x)^T P~ at one point; x0 is the state (u + d in defect correction) at the point
template <class T, int K, class A>
__device__ __forceinline__ T gradT3_pt(const Desc& d, const A& p, T x0, int l, int i, int j) {
  const T hx2 = T(d.hx2), hy2 = T(d.hy2), hz2 = T(d.hz2), dt = T(d.dt), a = T(d.a), b = T(d.b);
  const T P = p(l, i, j);
  if constexpr (K == KK_NONE_LAP) {
    return P - dt * a * lap7(p, l, i, j, P, hx2, hy2, hz2);
  } else if constexpr (K == KK_NONE_BIH) {
    return P + dt * a * lap25(p, l, i, j, P, hx2, hy2, hz2);
  } else if constexpr (K == KK_AC) {
    return P - dt * a * lap7(p, l, i, j, P, hx2, hy2, hz2) + dt * b * (T(3) * x0 * x0 - T(1)) * P;
  } else {
    constexpr T sh = K == KK_CH_IMPL ? T(1) : T(0);
    return P + dt * a * lap25(p, l, i, j, P, hx2, hy2, hz2) -
           dt * b * (T(3) * x0 * x0 - sh) * lap7(p, l, i, j, P, hx2, hy2, hz2);
  }
}

// (l, i, j) of the point with flat index q of one component
__device__ __forceinline__ void point3(const Desc& d, size_t q, int& l, int& i, int& j) {
  j = (int)(q & (size_t)(d.nx - 1));
  i = (int)((q >> d.lognx) & (size_t)(d.ny - 1));
  l = (int)(q >> (d.lognx + d.logny));
}

// ---------------------------------------------------------------------------------------
// k3_res: W = F(U_n), norm partials, stopping decision
// ---------------------------------------------------------------------------------------
template <class T, int K>
__device__ __forceinline__ void res3_body(const Desc& d, State* __restrict__ st, Slot* slot, int b) {
  constexpr bool DC = sizeof(T) == 4;
  if (!sweep_active(st, slot)) return;
  __shared__ double red[32];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const G3<T> X{static_cast<const T*>(d.X), d.nx, d.ny, d.nz, d.bc};
  const G3<T> B{static_cast<const T*>(d.base), d.nx, d.ny, d.nz, d.bc};
  const T* __restrict__ R = static_cast<const T*>(d.rhs);
  T* __restrict__ W = static_cast<T*>(d.WY);
  const long pz = d.nz > 1 ? (long)d.nx * d.ny : 0;
  constexpr int RAD = radius3<K>();
  double acc = 0.0;
#pragma unroll 4
  for (size_t q = (size_t)b * blockDim.x + threadIdx.x; q < N; q += (size_t)d.blk3 * blockDim.x) {
    int l, i, j;
    point3(d, q, l, i, j);
    T w;
    if (inside_yz<RAD>(d, l, i)) {
      const size_t row = q - (size_t)j;
      const G3r<T> Xr{static_cast<const T*>(d.X) + row, l, i, d.nx, d.bc, pz};
      const G3r<T> Br{static_cast<const T*>(d.base) + row, l, i, d.nx, d.bc, pz};
      w = residual3_pt<T, K, DC>(d, Xr, Br, l, i, j, R[q]);
    } else {
      w = residual3_pt<T, K, DC>(d, X, B, l, i, j, R[q]);
    }
    W[q] = w;
    acc += (double)(w * w);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[b] = s;
  if (last_block(st, d.blk3)) finalize_measure(d, st, red, slot, d.blk3);
}

// ---------------------------------------------------------------------------------------
// k3_upd: U_{n+1} = U_n - tau_u dF(U_n)^T P~ with P~ in the transform buffer
// ---------------------------------------------------------------------------------------
template <class T, int K>
__device__ __forceinline__ void upd3_body(const Desc& d, State* __restrict__ st, Slot* slot, int b) {
  constexpr bool DC = sizeof(T) == 4;
  if (!sweep_active(st, slot)) return;
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const G3<T> Pt{static_cast<const T*>(d.WY), d.nx, d.ny, d.nz, d.bc};
  T* __restrict__ X = static_cast<T*>(d.X);
  const T* __restrict__ Bs = static_cast<const T*>(d.base);
  const T tu = T(d.tau_u);
  const long pz = d.nz > 1 ? (long)d.nx * d.ny : 0;
  constexpr int RAD = radius3<K>();
  for (size_t q = (size_t)b * blockDim.x + threadIdx.x; q < N; q += (size_t)d.blk3 * blockDim.x) {
    int l, i, j;
    point3(d, q, l, i, j);
    const T xq = X[q];
    T x0 = xq;
    if constexpr (DC && KT<K>::nonlinear) x0 += Bs[q];
    T g;
    if (inside_yz<RAD>(d, l, i)) {
      const G3r<T> Pr{static_cast<const T*>(d.WY) + (q - (size_t)j), l, i, d.nx, d.bc, pz};
      g = gradT3_pt<T, K>(d, Pr, x0, l, i, j);
    } else {
      g = gradT3_pt<T, K>(d, Pt, x0, l, i, j);
    }
    X[q] = xq - tu * g;
  }
}

// ---------------------------------------------------------------------------------------
// transform passes
// ---------------------------------------------------------------------------------------
enum Lines3Mode {
  L3_FWD = 0,   // forward real transform of spatial values: coefficient k at position k
  L3_FSI = 1,   // forward, times 1 / (g_hat nx ny nz), inverse (the last axis, z)
  L3_INV = 2,   // inverse of L3_FWD (up to the factor n folded into the symbol)
  L3_INVP = 3,  // L3_INV along x, then the dual update and P~ (PDHG iteration)
  L3_INVX = 4   // L3_INV along x into d.X (preconditioner-only solve)
};

// Lines of axis AX grouped in tiles of lw lines, two lines per complex line in shared memory:
// x: lw consecutive rows; y (z): lw adjacent x columns of one (component, z) plane (one
// (component, y) row of planes).  Returns the tile's first element; *sl = element stride along
// the line; *orow = the tile's index along the third axis (z for y lines, y for z lines).  For y
// and z the lw lines of a tile are contiguous in memory.
template <int AX>
__device__ __forceinline__ size_t tile3(const Desc& d, long t, int lw, size_t* sl, int* orow) {
  const size_t plane = (size_t)d.nx * d.ny;
  if (AX == 0) {
    *sl = 1;
    *orow = 0;
    return (size_t)t * lw * d.nx;
  }
  const long ntx = d.nx / lw;
  const long g = t / ntx;                 // (component, z) for y lines, (component, y) for z lines
  const size_t x0 = (size_t)(t - g * ntx) * lw;
  if (AX == 1) {
    *sl = d.nx;
    *orow = (int)(g & (long)(d.nz - 1));
    return (size_t)g * plane + x0;
  }
  const long c = g / d.ny, y = g - c * d.ny;
  *sl = plane;
  *orow = (int)y;
  return (size_t)c * plane * d.nz + (size_t)y * d.nx + x0;
}

// One transform pass over the tiles of axis AX.  The spectral scaling (L3_FSI) runs on the last
// axis of the grid: z on 3-D grids, y on 2-D grids (nz = 1), which the launchers route to these
// kernels when a line is too long for the band / column sweeps.  LOGN > 0: lines of 2^LOGN
// points (4096 or 8192), one radix-8 job per thread and pass (2^LOGN / 8 threads), with the
// pass sequence and line stride fixed at compile time.
template <class T, int AX, int MODE, int LOGN = 0>
__device__ __forceinline__ void lines3_body(const Desc& d, State* __restrict__ st, Slot* slot, int b,
                                            unsigned char* smem_raw) {
  const bool pc = d.mode == MODE_PRECOND_ONLY;
  if (!pc && !sweep_active(st, slot)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = AX == 0 ? d.nx : (AX == 1 ? d.ny : d.nz);
  const int logn = AX == 0 ? d.lognx : (AX == 1 ? d.logny : d.lognz);
  const int hn = n >> 1, lh = logn - 1;
  const bool per = d.bc == BC_PERIODIC;
  const int lw = d.lw3[AX];
  const int nl = lw >> 1;
  const int ls = padded_len(n);
  const long ntiles = AX == 0 ? (long)d.ncomp * d.nz * d.ny / lw
                              : (long)d.ncomp * (AX == 1 ? d.nz : d.ny) * (d.nx / lw);
  const cx<T>* tw;
  const cx<T>* dc;
  const void* twg = AX == 0 ? d.twx : (AX == 1 ? d.twy : d.twz);
  const void* dcg = AX == 0 ? d.dcx : (AX == 1 ? d.dcy : d.dcz);
  cx<T>* buf = reinterpret_cast<cx<T>*>(place_tables<T>(smem_raw, twg, dcg, n, true, !per, tw, dc));
  T* __restrict__ WY = static_cast<T*>(d.WY);
  constexpr bool INV = MODE == L3_INV || MODE == L3_INVP || MODE == L3_INVX;
  // the long x inverse pass with the dual update: the tile's rows of P are copied into shared
  // memory behind the line buffer while the transform runs, so that the epilogue's reads of P
  // do not wait on global memory after it (d.pf3: the copy fits)
  constexpr bool PFC = LOGN > 0 && AX == 0 && MODE == L3_INVP && sizeof(T) == 4;
  const bool pf = PFC && d.pf3;
  T* Ps = reinterpret_cast<T*>(buf + nl * ls);
  for (long t = b; t < ntiles; t += d.blk3) {
    size_t sl;
    int orow;
    const size_t base = tile3<AX>(d, t, lw, &sl, &orow);
    __syncthreads();  // the tables are loaded / the previous tile's buffer is free
    if constexpr (PFC)
      if (pf) cp_async_block(Ps, static_cast<const T*>(d.P[0]) + base, lw * d.nx * (int)sizeof(T));
    // 1. load: spatial values (forward modes; Neumann in Makhoul order), or coefficients k in
    //    natural order (inverse modes; Neumann: the conjugated DCT-III preparation)
    if constexpr (!INV) {
      if constexpr (AX == 0) {
        for (int g = tid; g < (nl << lh); g += nt) {
          const int p = g >> lh, jj = 2 * (g & (hn - 1));
          const T* ra = WY + base + (size_t)(2 * p) * d.nx;
          const cx<T> va = *reinterpret_cast<const cx<T>*>(ra + jj);
          const cx<T> vb = *reinterpret_cast<const cx<T>*>(ra + d.nx + jj);
          buf[p * ls + pidx(per ? jj : mk_slot(jj, n))] = cx<T>{va.x, vb.x};
          buf[p * ls + pidx(per ? jj + 1 : mk_slot(jj + 1, n))] = cx<T>{va.y, vb.y};
        }
      } else {
        for (int g = tid; g < n * nl; g += nt) {
          const int l = g / nl, p = g - l * nl;
          buf[p * ls + pidx(per ? l : mk_slot(l, n))] = *reinterpret_cast<const cx<T>*>(WY + base + l * sl + 2 * p);
        }
      }
    } else {
      // coefficient k of the tile's line pair p
      auto coef = [&](int p, int k) -> cx<T> {
        if constexpr (AX == 0) {
          const T* ra = WY + base + (size_t)(2 * p) * d.nx;
          return cx<T>{ra[k], ra[d.nx + k]};
        } else {
          return *reinterpret_cast<const cx<T>*>(WY + base + k * sl + 2 * p);
        }
      };
      if (per) {
        for (int g = tid; g < n * nl; g += nt) {
          const int p = AX == 0 ? g / n : g - (g / nl) * nl;
          const int k = AX == 0 ? g - p * n : g / nl;
          buf[p * ls + pidx(k)] = coef(p, k);
        }
      } else {
        for (int g = tid; g < (nl << lh); g += nt) {
          const int p = g >> lh, k = g & (hn - 1);
          cx<T>* L = buf + p * ls;
          const cx<T> w = dc[k];
          cx<T> zk, zkp;
          if (k == 0) {
            dct_inv_pre(coef(p, 0), cx<T>{T(0), T(0)}, w.x, w.y, zk, zkp);
            const cx<T> Xm = coef(p, hn);
            const cx<T> wm = dc[hn];
            cx<T> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<T>{zk.x, -zk.y};
            L[pidx(hn)] = cx<T>{zm.x, -zm.y};
          } else {
            dct_inv_pre(coef(p, k), coef(p, n - k), w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<T>{zk.x, -zk.y};
            L[pidx(n - k)] = cx<T>{zkp.x, -zkp.y};
          }
        }
      }
    }
    __syncthreads();
    cx<T>* cur;
    if constexpr (LOGN > 0) cur = block_fft_long<T, -1, 1, LOGN>(buf, nl, tw, tid, nt);
    else cur = block_fft_loop<T, -1>(buf, buf, nl, logn, ls, tw, tid, nt);
    if constexpr (MODE == L3_FSI) {
      // forward epilogue and the spectral scaling 1 / (g_hat nx ny nz), in place; then the
      // second (inverse) transform as in the 2-D column pass
      const T* mux = static_cast<const T*>(d.mux);
      const T* muy = static_cast<const T*>(d.muy);
      const T* muz = static_cast<const T*>(d.muz);
      const int c = (int)((base / ((size_t)d.nx * d.ny)) / d.nz);
      const T c1 = T(d.gc1[c]), c2 = T(d.gc2[c]), c3 = T(d.gc3[c]), inn = T(d.inv_nn);
      auto sym = [&](T mu) -> T {
        const T g = T(1) + mu * (c1 + mu * (c2 + c3 * mu));
        if constexpr (sizeof(T) == 4) return inn * __frcp_rn(g * g);
        else return inn / (g * g);
      };
      // eigenvalues: mu_line of the line's own axis at frequency k, plus those of the other
      // axes at the tile's position (x: the pair's two columns; the third axis: orow)
      const T* mul = AX == 2 ? muz : muy;
      const int x0 = (int)(base % d.nx);
      const T my = AX == 2 ? muy[orow] : muz[orow];
      for (int g = tid; g < (nl << lh); g += nt) {
        const int p = g >> lh, k = g & (hn - 1);
        cx<T>* L = cur + p * ls;
        cx<T> ok, okp;
        fwd_post(L, n, d.bc, dc, k, ok, okp);
        const int k2 = k == 0 ? hn : n - k;
        if (k == 0) {
          cx<T> tt;
          fwd_post(L, n, d.bc, dc, hn, okp, tt);
        }
        const T ma = mux[x0 + 2 * p] + my, mb = mux[x0 + 2 * p + 1] + my;
        const T m1 = mul[k], m2 = mul[k2];
        L[pidx(k)] = cx<T>{ok.x * sym(ma + m1), ok.y * sym(mb + m1)};
        L[pidx(k2)] = cx<T>{okp.x * sym(ma + m2), okp.y * sym(mb + m2)};
      }
      __syncthreads();
      if (!per) {
        for (int g = tid; g < (nl << lh); g += nt) {
          const int p = g >> lh, k = g & (hn - 1);
          cx<T>* L = cur + p * ls;
          const cx<T> w = dc[k];
          cx<T> zk, zkp;
          if (k == 0) {
            dct_inv_pre(L[pidx(0)], cx<T>{T(0), T(0)}, w.x, w.y, zk, zkp);
            const cx<T> Xm = L[pidx(hn)];
            const cx<T> wm = dc[hn];
            cx<T> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<T>{zk.x, -zk.y};
            L[pidx(hn)] = cx<T>{zm.x, -zm.y};
          } else {
            dct_inv_pre(L[pidx(k)], L[pidx(n - k)], w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<T>{zk.x, -zk.y};
            L[pidx(n - k)] = cx<T>{zkp.x, -zkp.y};
          }
        }
        __syncthreads();
      }
      if constexpr (LOGN > 0) cur = block_fft_long<T, -1, 1, LOGN>(cur, nl, tw, tid, nt);
      else cur = block_fft_loop<T, -1>(cur, cur, nl, logn, ls, tw, tid, nt);
    }
    if constexpr (MODE == L3_FWD) {
      // forward epilogue straight to global memory: coefficient k of both lines
      for (int g = tid; g < (nl << lh); g += nt) {
        const int p = g >> lh, k = g & (hn - 1);
        const cx<T>* L = cur + p * ls;
        cx<T> ok, okp;
        fwd_post(L, n, d.bc, dc, k, ok, okp);
        const int k2 = k == 0 ? hn : n - k;
        if (k == 0) {
          cx<T> tt;
          fwd_post(L, n, d.bc, dc, hn, okp, tt);
        }
        if constexpr (AX == 0) {
          T* ra = WY + base + (size_t)(2 * p) * d.nx;
          ra[k] = ok.x;
          ra[d.nx + k] = ok.y;
          ra[k2] = okp.x;
          ra[d.nx + k2] = okp.y;
        } else {
          *reinterpret_cast<cx<T>*>(WY + base + k * sl + 2 * p) = ok;
          *reinterpret_cast<cx<T>*>(WY + base + k2 * sl + 2 * p) = okp;
        }
      }
    } else {
      // spatial values: periodic -- the Hartley epilogue in place, slot j holds point j;
      // Neumann -- slot j holds the conjugate of point mk_perm(j)
      if (per) {
        post_inplace(cur, nl, logn, ls, d.bc, dc);
        __syncthreads();
      }
      if constexpr (AX == 0) {
        const T tp = T(d.tau_p), tpe = T((1.0 + d.omega) * d.tau_p);
        T* P = static_cast<T*>(d.P[0]);
        T* dst = MODE == L3_INVX ? static_cast<T*>(d.X) : WY;
        if constexpr (PFC) {
          if (pf) {
            cp_async_wait_all();
            __syncthreads();
          }
        }
        for (int g = tid; g < nl * n; g += nt) {
          const int p = g / n, j = g - p * n;
          const cx<T> v0 = cur[p * ls + pidx(j)];
          const int jj = per ? j : mk_perm(j, n);
          const T ya = v0.x, yb = per ? v0.y : -v0.y;
          const size_t oa = base + (size_t)(2 * p) * d.nx + jj, ob = oa + d.nx;
          if constexpr (MODE == L3_INVP) {
            T pa, pb;
            if (PFC && pf) {
              pa = Ps[oa - base];
              pb = Ps[ob - base];
            } else {
              pa = P[oa];
              pb = P[ob];
            }
            P[oa] = pa + tp * ya;
            P[ob] = pb + tp * yb;
            dst[oa] = pa + tpe * ya;
            dst[ob] = pb + tpe * yb;
          } else {
            dst[oa] = ya;
            dst[ob] = yb;
          }
        }
      } else {
        for (int g = tid; g < n * nl; g += nt) {
          const int j = g / nl, p = g - j * nl;
          const cx<T> v = cur[p * ls + pidx(j)];
          const int jj = per ? j : mk_perm(j, n);
          *reinterpret_cast<cx<T>*>(WY + base + jj * sl + 2 * p) = per ? v : cx<T>{v.x, -v.y};
        }
      }
    }
  }
}

// Shared-memory bytes of a transform pass block: the tables of the line length and the lw / 2
// complex lines of a tile (plus, with prefetch, the tile's lw rows of P).
template <class T>
__host__ __device__ inline int lines3_smem_bytes(int n, int lw, bool neumann, bool prefetch = false) {
  return table_bytes<T>(n, true, neumann) + (lw >> 1) * padded_len(n) * (int)sizeof(cx<T>) +
         (prefetch ? lw * n * (int)sizeof(T) : 0);
}


}  // namespace rd
