// The whole FP32 inner PDHG solve of a small 2-D grid in ONE thread block (Section 2.1,
// Algorithm 1's inner loop, on the correction equation of FP64 defect correction): every array
// of the solve -- the unknown d, the base state u, the right-hand side r = F(u), the dual P, the
// transform array -- lives in shared memory, and the phases of an iteration are separated by
// block barriers instead of kernel boundaries.  Per iteration:
//   A  W = F~(d) by the five- or thirteen-point stencil, ||W_c||^2 by a block reduction, and the
//      stopping rule (the same rule as the multi-kernel sweeps);
//   B  forward row transform of W (pair-packed Hartley / Makhoul DCT-II), spectrum to the array;
//   C  column transform forward, times 1 / (g_hat nx ny), inverse;
//   D  inverse row transform of Y = G^{-1} W, P_{n+1} = P_n + tau_p Y, P~ = P_n + (1+omega) tau_p Y;
//   E  d_{n+1} = d_n - tau_u dF(u + d_n)^T P~.
// A launch runs the solve from the state the FP64 residual armed until it stops, then writes d
// and the solve state back to global memory.  The paper's method is unchanged: only where the
// arrays live and how the phases are synchronised differ from the band / column kernels.
#pragma once

#include <cooperative_groups.h>

#include "rd_sweep.cuh"

namespace rd {

constexpr int kSmallThreads = 256;

__host__ __device__ inline int up16(int b) { return (b + 15) & ~15; }

// Shared-memory bytes of the small solve of an nx x ny grid with nc components: the FP32 tables
// (twiddles, DCT rotations, eigenvalues of both axes), five real arrays (d, u, r, P, transform
// array) and the complex line buffer of the larger of the row and column passes.
__host__ __device__ inline int small_smem_bytes(int nx, int ny, int nc, bool neumann) {
  int b = 0;
  b += up16(tw_entries(nx) * 8) + (neumann ? up16(nx * 8) : 0);
  b += up16(tw_entries(ny) * 8) + (neumann ? up16(ny * 8) : 0);
  b += up16(nx * 4) + up16(ny * 4);
  b += 5 * up16(nc * nx * ny * 4);
  const int lines_r = nc * (ny / 2) * padded_len(nx), lines_c = nc * (nx / 2) * padded_len(ny);
  b += up16((lines_r > lines_c ? lines_r : lines_c) * 8);
  return b;
}

template <int K>
__device__ __forceinline__ void small_solve_body(const Desc& d, State* __restrict__ gst, Slot* slot,
                                                 unsigned char* smem) {
  if (!sweep_active(gst, slot)) return;
  constexpr bool TWO = KT<K>::two;
  constexpr int NCC = TWO ? 2 : 1;
  const int nx = d.nx, ny = d.ny, lognx = d.lognx, logny = d.logny;
  const int N = nx * ny, NC = NCC * N;
  const bool per = d.bc == BC_PERIODIC;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hnx = nx >> 1, hny = ny >> 1, lhx = lognx - 1, lhy = logny - 1;
  const int lsx = padded_len(nx), lsy = padded_len(ny);
  // carve the shared memory (the layout of small_smem_bytes)
  unsigned char* p = smem;
  cx<float>* twx = reinterpret_cast<cx<float>*>(p);
  p += up16(tw_entries(nx) * 8);
  cx<float>* dcx = reinterpret_cast<cx<float>*>(p);
  p += per ? 0 : up16(nx * 8);
  cx<float>* twy = reinterpret_cast<cx<float>*>(p);
  p += up16(tw_entries(ny) * 8);
  cx<float>* dcy = reinterpret_cast<cx<float>*>(p);
  p += per ? 0 : up16(ny * 8);
  float* mux = reinterpret_cast<float*>(p);
  p += up16(nx * 4);
  float* muy = reinterpret_cast<float*>(p);
  p += up16(ny * 4);
  float* X = reinterpret_cast<float*>(p);
  p += up16(NC * 4);
  float* B = reinterpret_cast<float*>(p);
  p += up16(NC * 4);
  float* R = reinterpret_cast<float*>(p);
  p += up16(NC * 4);
  float* P = reinterpret_cast<float*>(p);
  p += up16(NC * 4);
  float* WY = reinterpret_cast<float*>(p);
  p += up16(NC * 4);
  cx<float>* buf = reinterpret_cast<cx<float>*>(p);

  __shared__ State s;
  __shared__ double red[32];
  __shared__ int go;
  load_table(twx, static_cast<const cx<float>*>(d.twx), tw_entries(nx));
  load_table(twy, static_cast<const cx<float>*>(d.twy), tw_entries(ny));
  if (!per) {
    load_table(dcx, static_cast<const cx<float>*>(d.dcx), nx);
    load_table(dcy, static_cast<const cx<float>*>(d.dcy), ny);
  }
  for (int k = tid; k < nx; k += nt) mux[k] = static_cast<const float*>(d.mux)[k];
  for (int k = tid; k < ny; k += nt) muy[k] = static_cast<const float*>(d.muy)[k];
  {
    const float* gX = static_cast<const float*>(d.X);
    const float* gB = static_cast<const float*>(d.base);
    const float* gR = static_cast<const float*>(d.rhs);
    const float* gP = static_cast<const float*>(d.P[0]);
    for (int q = tid; q < NC; q += nt) {
      X[q] = gX[q];
      B[q] = KT<K>::nonlinear ? gB[q] : 0.f;
      R[q] = gR[q];
      P[q] = gP[q];
    }
  }
  if (tid == 0) s = *gst;
  __syncthreads();

  const GField<float> x0{X, nx, ny, d.bc}, x1{X + N, nx, ny, d.bc};
  const GField<float> b0{B, nx, ny, d.bc}, b1{B + N, nx, ny, d.bc};
  const GField<float> t0{WY, nx, ny, d.bc}, t1{WY + N, nx, ny, d.bc};
  const float tu = float(d.tau_u), tp = float(d.tau_p), tpe = float((1.0 + d.omega) * d.tau_p);
  const float inn = float(d.inv_nn);
  for (;;) {
    // A. W = F~(d) into the row-pair lines, norms, the stopping rule
    float acc0 = 0.f, acc1 = 0.f;
    for (int q = tid; q < N; q += nt) {
      const int i = q >> lognx, j = q & (nx - 1);
      float w[2] = {0.f, 0.f};
      residual_pt<float, K, true>(d, x0, x1, b0, b1, i, j, R[q], TWO ? R[N + q] : 0.f, w);
      acc0 += w[0] * w[0];
      acc1 += w[1] * w[1];
      const int sj = per ? j : mk_slot(j, nx);
      reinterpret_cast<float*>(buf + (i >> 1) * lsx + pidx(sj))[i & 1] = w[0];
      if (TWO) reinterpret_cast<float*>(buf + (hny + (i >> 1)) * lsx + pidx(sj))[i & 1] = w[1];
    }
    const double q0 = block_sum((double)acc0, red);
    const double q1 = TWO ? block_sum((double)acc1, red) : 0.0;
    if (tid == 0) {
      measure_decide(d, &s, sqrt(q0) + (TWO ? sqrt(q1) : 0.0), slot);
      go = s.status == ST_ACTIVE;
    }
    __syncthreads();
    if (!go) break;
    // B. forward row transform; real coefficients of rows 2m, 2m+1 into WY
    {
      const cx<float>* res = block_fft_loop<float, -1>(buf, buf, NCC * hny, lognx, lsx, twx, tid, nt);
      for (int g = tid; g < ((NCC * hny) << lhx); g += nt) {
        const int line = g >> lhx, k = g & (hnx - 1);
        const int c = line / hny, m = line - c * hny;
        float* Wa = WY + c * N + (2 * m) * nx;
        float* Wb = Wa + nx;
        cx<float> ok, okp;
        fwd_post(res + line * lsx, nx, d.bc, dcx, k, ok, okp);
        Wa[k] = ok.x;
        Wb[k] = ok.y;
        if (k != 0) {
          Wa[nx - k] = okp.x;
          Wb[nx - k] = okp.y;
        } else {
          fwd_post(res + line * lsx, nx, d.bc, dcx, hnx, ok, okp);
          Wa[hnx] = ok.x;
          Wb[hnx] = ok.y;
        }
      }
      __syncthreads();
    }
    // C. column transform: forward, 1 / (g_hat nx ny), inverse (pairs of columns per line)
    {
      for (int g = tid; g < NCC * hnx * ny; g += nt) {
        const int line = g / ny, row = g - line * ny;
        const int c = line / hnx, pp = line - c * hnx;
        const float* Wr = WY + c * N + row * nx + 2 * pp;
        buf[line * lsy + pidx(per ? row : mk_slot(row, ny))] = cx<float>{Wr[0], Wr[1]};
      }
      __syncthreads();
      cx<float>* cur = block_fft_loop<float, -1>(buf, buf, NCC * hnx, logny, lsy, twy, tid, nt);
      for (int g = tid; g < ((NCC * hnx) << lhy); g += nt) {
        const int line = g >> lhy, k = g & (hny - 1);
        const int c = line / hnx, pp = line - c * hnx;
        const float c1 = float(d.gc1[c]), c2 = float(d.gc2[c]), c3 = float(d.gc3[c]);
        auto sym = [&](float mu) -> float {
          const float gg = 1.f + mu * (c1 + mu * (c2 + c3 * mu));
          return inn * __frcp_rn(gg * gg);
        };
        cx<float>* L = cur + line * lsy;
        cx<float> ok, okp;
        fwd_post(L, ny, d.bc, dcy, k, ok, okp);
        const int k2 = k == 0 ? hny : ny - k;
        if (k == 0) {
          cx<float> tt;
          fwd_post(L, ny, d.bc, dcy, hny, okp, tt);
        }
        const float ma = mux[2 * pp], mb = mux[2 * pp + 1], m1 = muy[k], m2 = muy[k2];
        L[pidx(k)] = cx<float>{ok.x * sym(ma + m1), ok.y * sym(mb + m1)};
        L[pidx(k2)] = cx<float>{okp.x * sym(ma + m2), okp.y * sym(mb + m2)};
      }
      __syncthreads();
      if (!per) {
        for (int g = tid; g < ((NCC * hnx) << lhy); g += nt) {
          const int line = g >> lhy, k = g & (hny - 1);
          cx<float>* L = cur + line * lsy;
          const cx<float> w = dcy[k];
          cx<float> zk, zkp;
          if (k == 0) {
            dct_inv_pre(L[pidx(0)], cx<float>{0.f, 0.f}, w.x, w.y, zk, zkp);
            const cx<float> Xm = L[pidx(hny)];
            const cx<float> wm = dcy[hny];
            cx<float> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<float>{zk.x, -zk.y};
            L[pidx(hny)] = cx<float>{zm.x, -zm.y};
          } else {
            dct_inv_pre(L[pidx(k)], L[pidx(ny - k)], w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<float>{zk.x, -zk.y};
            L[pidx(ny - k)] = cx<float>{zkp.x, -zkp.y};
          }
        }
        __syncthreads();
      }
      cur = block_fft_loop<float, -1>(cur, cur, NCC * hnx, logny, lsy, twy, tid, nt);
      if (per) {
        post_inplace(cur, NCC * hnx, logny, lsy, d.bc, dcy);
        __syncthreads();
      }
      for (int g = tid; g < NCC * hnx * ny; g += nt) {
        const int line = g / ny, n = g - line * ny;
        const int c = line / hnx, pp = line - c * hnx;
        const cx<float> v = cur[line * lsy + pidx(n)];
        float* Wr = WY + c * N + (per ? n : mk_perm(n, ny)) * nx + 2 * pp;
        Wr[0] = v.x;
        Wr[1] = per ? v.y : -v.y;
      }
      __syncthreads();
    }
    // D. inverse row transform of Y; P_{n+1} and P~ (into WY)
    {
      if (per) {
        for (int g = tid; g < NCC * hny * nx; g += nt) {
          const int line = g >> lognx, k = g & (nx - 1);
          const int c = line / hny, m = line - c * hny;
          const float* Wa = WY + c * N + (2 * m) * nx;
          buf[line * lsx + pidx(k)] = cx<float>{Wa[k], Wa[nx + k]};
        }
      } else {
        for (int g = tid; g < ((NCC * hny) << lhx); g += nt) {
          const int line = g >> lhx, k = g & (hnx - 1);
          const int c = line / hny, m = line - c * hny;
          const float* Wa = WY + c * N + (2 * m) * nx;
          const float* Wb = Wa + nx;
          cx<float>* L = buf + line * lsx;
          const cx<float> w = dcx[k];
          cx<float> zk, zkp;
          if (k == 0) {
            dct_inv_pre(cx<float>{Wa[0], Wb[0]}, cx<float>{0.f, 0.f}, w.x, w.y, zk, zkp);
            const cx<float> Xm{Wa[hnx], Wb[hnx]};
            const cx<float> wm = dcx[hnx];
            cx<float> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<float>{zk.x, -zk.y};
            L[pidx(hnx)] = cx<float>{zm.x, -zm.y};
          } else {
            dct_inv_pre(cx<float>{Wa[k], Wb[k]}, cx<float>{Wa[nx - k], Wb[nx - k]}, w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<float>{zk.x, -zk.y};
            L[pidx(nx - k)] = cx<float>{zkp.x, -zkp.y};
          }
        }
      }
      __syncthreads();
      cx<float>* cur = block_fft_loop<float, -1>(buf, buf, NCC * hny, lognx, lsx, twx, tid, nt);
      if (per) {
        post_inplace(cur, NCC * hny, lognx, lsx, d.bc, dcx);
        __syncthreads();
      }
      for (int q = tid; q < NC; q += nt) {
        const int c = q / N, r = q - c * N;
        const int i = r >> lognx, j = r & (nx - 1);
        const cx<float> v = cur[(c * hny + (i >> 1)) * lsx + pidx(per ? j : mk_slot(j, nx))];
        const float y = (i & 1) ? (per ? v.y : -v.y) : v.x;
        const float po = P[q];
        P[q] = po + tp * y;
        WY[q] = po + tpe * y;
      }
      __syncthreads();
    }
    // E. d_{n+1} = d_n - tau_u dF(u + d_n)^T P~
    for (int q = tid; q < N; q += nt) {
      const int i = q >> lognx, j = q & (nx - 1);
      float s0 = X[q], s1 = TWO ? X[N + q] : 0.f;
      if constexpr (KT<K>::nonlinear) {
        s0 += B[q];
        if constexpr (TWO) s1 += B[N + q];
      }
      float g[2] = {0.f, 0.f};
      gradT_pt<float, K>(d, t0, t1, s0, s1, i, j, g);
      X[q] -= tu * g[0];
      if constexpr (TWO) X[N + q] -= tu * g[1];
    }
    __syncthreads();
  }
  // the correction and the final solve state back to global memory
  float* gX = static_cast<float*>(d.X);
  for (int q = tid; q < NC; q += nt) gX[q] = X[q];
  if (tid == 0) {
    s.trips = (unsigned)s.n + 1u;
    s.ticket = 0u;
    *gst = s;
  }
}


// ---------------------------------------------------------------------------------------
// The same inner solve on a cluster of kClusterCtas blocks (distributed shared memory): block r
// owns rows [r R, (r+1) R) (R = ny / 8) of every array, with H halo rows above and below copied
// from its neighbours, and column slab [r C, (r+1) C) (C = nx / 8) of the column pass, gathered
// from and scattered back to the owners of the rows.  Cluster barriers separate the phases:
//   A  halo rows of d; W = F~(d) on own rows; row partials           -> barrier 1
//      every block sums the partials in rank order and takes the same stopping decision
//   B  forward row transform of own rows                             -> barrier 2
//   C  column slab: gather, transform, 1 / g_hat, inverse, scatter   -> barrier 3
//   D  inverse row transform of own rows, P_{n+1}, P~                -> barrier 4
//   E  halo rows of P~; d_{n+1} on own rows                          -> barrier 5
// ---------------------------------------------------------------------------------------
constexpr int kClusterCtas = 8;

__host__ __device__ inline int cluster_smem_bytes(int nx, int ny, int nc, int H, bool neumann) {
  const int R = ny / kClusterCtas, C = nx / kClusterCtas;
  int b = 0;
  b += up16(tw_entries(nx) * 8) + (neumann ? up16(nx * 8) : 0);
  b += up16(tw_entries(ny) * 8) + (neumann ? up16(ny * 8) : 0);
  b += up16(nx * 4) + up16(ny * 4);
  b += 3 * up16(nc * (R + 2 * H) * nx * 4);  // d, u, P~ / spectrum with halo rows
  b += 2 * up16(nc * R * nx * 4);            // r, P
  const int lines_r = nc * (R / 2) * padded_len(nx), lines_c = nc * (C / 2) * padded_len(ny);
  b += 2 * up16((lines_r > lines_c ? lines_r : lines_c) * 8);  // ping-pong line buffers
  return b;
}

template <int K>
__device__ __forceinline__ void small_cluster_body(const Desc& d, State* __restrict__ gst, Slot* slot,
                                                   unsigned char* smem) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  // the state is the same for every block of the cluster: all return, or none
  if (!sweep_active(gst, slot)) return;
  constexpr bool TWO = KT<K>::two;
  constexpr int NCC = TWO ? 2 : 1;
  constexpr int H = KT<K>::biharm ? 2 : 1;
  const int nx = d.nx, ny = d.ny, lognx = d.lognx, logny = d.logny;
  const int N = nx * ny;
  const int R = ny / kClusterCtas, C = nx / kClusterCtas;
  const int RH = R + 2 * H;
  const int y0 = rank * R, x0 = rank * C;
  const bool per = d.bc == BC_PERIODIC;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hnx = nx >> 1, hny = ny >> 1, lhx = lognx - 1, lhy = logny - 1;
  const int hR = R >> 1, hC = C >> 1;
  const int lsx = padded_len(nx), lsy = padded_len(ny);
  unsigned char* p = smem;
  cx<float>* twx = reinterpret_cast<cx<float>*>(p);
  p += up16(tw_entries(nx) * 8);
  cx<float>* dcx = reinterpret_cast<cx<float>*>(p);
  p += per ? 0 : up16(nx * 8);
  cx<float>* twy = reinterpret_cast<cx<float>*>(p);
  p += up16(tw_entries(ny) * 8);
  cx<float>* dcy = reinterpret_cast<cx<float>*>(p);
  p += per ? 0 : up16(ny * 8);
  float* mux = reinterpret_cast<float*>(p);
  p += up16(nx * 4);
  float* muy = reinterpret_cast<float*>(p);
  p += up16(ny * 4);
  float* X = reinterpret_cast<float*>(p);   // [c][RH][nx], own rows at H
  p += up16(NCC * RH * nx * 4);
  float* B = reinterpret_cast<float*>(p);   // [c][RH][nx]
  p += up16(NCC * RH * nx * 4);
  float* WY = reinterpret_cast<float*>(p);  // [c][RH][nx]: row spectrum, then P~ (with halo)
  p += up16(NCC * RH * nx * 4);
  float* Rr = reinterpret_cast<float*>(p);  // [c][R][nx]
  p += up16(NCC * R * nx * 4);
  float* P = reinterpret_cast<float*>(p);   // [c][R][nx]
  p += up16(NCC * R * nx * 4);
  cx<float>* buf = reinterpret_cast<cx<float>*>(p);
  {
    const int lr_ = NCC * hR * lsx, lc_ = NCC * hC * lsy;
    p += up16((lr_ > lc_ ? lr_ : lc_) * 8);
  }
  // second line buffer: the transform passes ping-pong between buf and alt (one barrier a pass)
  cx<float>* alt = reinterpret_cast<cx<float>*>(p);

  __shared__ State s;
  __shared__ double red[32];
  __shared__ double part[2];
  __shared__ double parts[kClusterCtas][2];
  __shared__ int go;
  load_table(twx, static_cast<const cx<float>*>(d.twx), tw_entries(nx));
  load_table(twy, static_cast<const cx<float>*>(d.twy), tw_entries(ny));
  if (!per) {
    load_table(dcx, static_cast<const cx<float>*>(d.dcx), nx);
    load_table(dcy, static_cast<const cx<float>*>(d.dcy), ny);
  }
  for (int k = tid; k < nx; k += nt) mux[k] = static_cast<const float*>(d.mux)[k];
  for (int k = tid; k < ny; k += nt) muy[k] = static_cast<const float*>(d.muy)[k];
  {
    const float* gX = static_cast<const float*>(d.X);
    const float* gB = static_cast<const float*>(d.base);
    const float* gR = static_cast<const float*>(d.rhs);
    const float* gP = static_cast<const float*>(d.P[0]);
    for (int q = tid; q < NCC * R * nx; q += nt) {
      const int c = q / (R * nx), rem = q - c * R * nx;
      const size_t g = (size_t)c * N + (size_t)y0 * nx + rem;
      X[c * RH * nx + H * nx + rem] = gX[g];
      B[c * RH * nx + H * nx + rem] = KT<K>::nonlinear ? gB[g] : 0.f;
      Rr[q] = gR[g];
      P[q] = gP[g];
    }
  }
  if (tid == 0) s = *gst;
  // halo rows of an array with the [c][RH][nx] layout from the blocks that own them (periodic
  // wrap or half-cell mirror of the global row index)
  auto halo = [&](float* A) {
    for (int q = tid; q < NCC * 2 * H * nx; q += nt) {
      const int c = q / (2 * H * nx), rem = q - c * 2 * H * nx;
      const int hr = rem / nx, j = rem - hr * nx;
      const int lr = hr < H ? hr - H : R + (hr - H);       // local row -H..-1, R..R+H-1
      const int g = bcmap(y0 + lr, ny, d.bc);
      const int owner = g / R, loc = g - owner * R;
      const float* src = cl.map_shared_rank(A, owner);
      A[c * RH * nx + (lr + H) * nx + j] = src[c * RH * nx + (loc + H) * nx + j];
    }
  };
  cl.sync();
  halo(X);
  if (KT<K>::nonlinear) halo(B);
  __syncthreads();

  const Rows<float, true> x0r{X, nx, d.bc}, x1r{X + RH * nx, nx, d.bc};
  const Rows<float, true> b0r{B, nx, d.bc}, b1r{B + RH * nx, nx, d.bc};
  const Rows<float, true> t0r{WY, nx, d.bc}, t1r{WY + RH * nx, nx, d.bc};
  const float tu = float(d.tau_u), tp = float(d.tau_p), tpe = float((1.0 + d.omega) * d.tau_p);
  const float inn = float(d.inv_nn);
  for (;;) {
    // A. W = F~(d) on own rows into the row-pair lines, partial norms
    float acc0 = 0.f, acc1 = 0.f;
    for (int q = tid; q < R * nx; q += nt) {
      const int r = q >> lognx, j = q & (nx - 1);
      float w[2] = {0.f, 0.f};
      residual_pt<float, K, true>(d, x0r, x1r, b0r, b1r, H + r, j, Rr[q], TWO ? Rr[R * nx + q] : 0.f, w);
      acc0 += w[0] * w[0];
      acc1 += w[1] * w[1];
      const int sj = per ? j : mk_slot(j, nx);
      reinterpret_cast<float*>(buf + (r >> 1) * lsx + pidx(sj))[r & 1] = w[0];
      if (TWO) reinterpret_cast<float*>(buf + (hR + (r >> 1)) * lsx + pidx(sj))[r & 1] = w[1];
    }
    const double q0 = block_sum((double)acc0, red);
    const double q1 = TWO ? block_sum((double)acc1, red) : 0.0;
    if (tid == 0) {
      part[0] = q0;
      part[1] = q1;
    }
    cl.sync();  // 1
    // the blocks' partials, read in parallel, summed by thread 0 in rank order
    if (tid < kClusterCtas) {
      const double* pk = cl.map_shared_rank(part, tid);
      parts[tid][0] = pk[0];
      parts[tid][1] = pk[1];
    }
    __syncthreads();
    if (tid == 0) {
      double t0 = 0.0, t1 = 0.0;
      for (int k = 0; k < kClusterCtas; ++k) {
        t0 += parts[k][0];
        t1 += parts[k][1];
      }
      measure_decide(d, &s, sqrt(t0) + (TWO ? sqrt(t1) : 0.0), rank == 0 ? slot : nullptr);
      go = s.status == ST_ACTIVE;
    }
    __syncthreads();
    if (!go) break;
    // B. forward row transform of own rows; spectrum into WY's own rows
    {
      const cx<float>* res = block_fft_loop<float, -1>(buf, alt, NCC * hR, lognx, lsx, twx, tid, nt);
      for (int g = tid; g < ((NCC * hR) << lhx); g += nt) {
        const int line = g >> lhx, k = g & (hnx - 1);
        const int c = line / hR, m = line - c * hR;
        float* Wa = WY + c * RH * nx + (H + 2 * m) * nx;
        float* Wb = Wa + nx;
        cx<float> ok, okp;
        fwd_post(res + line * lsx, nx, d.bc, dcx, k, ok, okp);
        Wa[k] = ok.x;
        Wb[k] = ok.y;
        if (k != 0) {
          Wa[nx - k] = okp.x;
          Wb[nx - k] = okp.y;
        } else {
          fwd_post(res + line * lsx, nx, d.bc, dcx, hnx, ok, okp);
          Wa[hnx] = ok.x;
          Wb[hnx] = ok.y;
        }
      }
    }
    cl.sync();  // 2
    // C. column slab [x0, x0 + C): gather from the row owners, transform, scatter back
    {
      for (int g = tid; g < NCC * hC * ny; g += nt) {
        const int line = g / ny, row = g - line * ny;
        const int c = line / hC, pp = line - c * hC;
        const int owner = row / R, loc = row - owner * R;
        const float* src = cl.map_shared_rank(WY, owner) + c * RH * nx + (H + loc) * nx + x0 + 2 * pp;
        buf[line * lsy + pidx(per ? row : mk_slot(row, ny))] = *reinterpret_cast<const cx<float>*>(src);
      }
      __syncthreads();
      cx<float>* cur = block_fft_loop<float, -1>(buf, alt, NCC * hC, logny, lsy, twy, tid, nt);
      for (int g = tid; g < ((NCC * hC) << lhy); g += nt) {
        const int line = g >> lhy, k = g & (hny - 1);
        const int c = line / hC, pp = line - c * hC;
        const float c1 = float(d.gc1[c]), c2 = float(d.gc2[c]), c3 = float(d.gc3[c]);
        auto sym = [&](float mu) -> float {
          const float gg = 1.f + mu * (c1 + mu * (c2 + c3 * mu));
          return inn * __frcp_rn(gg * gg);
        };
        cx<float>* L = cur + line * lsy;
        cx<float> ok, okp;
        fwd_post(L, ny, d.bc, dcy, k, ok, okp);
        const int k2 = k == 0 ? hny : ny - k;
        if (k == 0) {
          cx<float> tt;
          fwd_post(L, ny, d.bc, dcy, hny, okp, tt);
        }
        const float ma = mux[x0 + 2 * pp], mb = mux[x0 + 2 * pp + 1], m1 = muy[k], m2 = muy[k2];
        L[pidx(k)] = cx<float>{ok.x * sym(ma + m1), ok.y * sym(mb + m1)};
        L[pidx(k2)] = cx<float>{okp.x * sym(ma + m2), okp.y * sym(mb + m2)};
      }
      __syncthreads();
      if (!per) {
        for (int g = tid; g < ((NCC * hC) << lhy); g += nt) {
          const int line = g >> lhy, k = g & (hny - 1);
          cx<float>* L = cur + line * lsy;
          const cx<float> w = dcy[k];
          cx<float> zk, zkp;
          if (k == 0) {
            dct_inv_pre(L[pidx(0)], cx<float>{0.f, 0.f}, w.x, w.y, zk, zkp);
            const cx<float> Xm = L[pidx(hny)];
            const cx<float> wm = dcy[hny];
            cx<float> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<float>{zk.x, -zk.y};
            L[pidx(hny)] = cx<float>{zm.x, -zm.y};
          } else {
            dct_inv_pre(L[pidx(k)], L[pidx(ny - k)], w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<float>{zk.x, -zk.y};
            L[pidx(ny - k)] = cx<float>{zkp.x, -zkp.y};
          }
        }
        __syncthreads();
      }
      cur = block_fft_loop<float, -1>(cur, cur == buf ? alt : buf, NCC * hC, logny, lsy, twy, tid, nt);
      if (per) {
        post_inplace(cur, NCC * hC, logny, lsy, d.bc, dcy);
        __syncthreads();
      }
      for (int g = tid; g < NCC * hC * ny; g += nt) {
        const int line = g / ny, n = g - line * ny;
        const int c = line / hC, pp = line - c * hC;
        const cx<float> v = cur[line * lsy + pidx(n)];
        const int row = per ? n : mk_perm(n, ny);
        const int owner = row / R, loc = row - owner * R;
        float* dst = cl.map_shared_rank(WY, owner) + c * RH * nx + (H + loc) * nx + x0 + 2 * pp;
        *reinterpret_cast<cx<float>*>(dst) = cx<float>{v.x, per ? v.y : -v.y};
      }
    }
    cl.sync();  // 3
    // D. inverse row transform of own rows; P_{n+1}, P~ into WY's own rows
    {
      if (per) {
        for (int g = tid; g < NCC * hR * nx; g += nt) {
          const int line = g >> lognx, k = g & (nx - 1);
          const int c = line / hR, m = line - c * hR;
          const float* Wa = WY + c * RH * nx + (H + 2 * m) * nx;
          buf[line * lsx + pidx(k)] = cx<float>{Wa[k], Wa[nx + k]};
        }
      } else {
        for (int g = tid; g < ((NCC * hR) << lhx); g += nt) {
          const int line = g >> lhx, k = g & (hnx - 1);
          const int c = line / hR, m = line - c * hR;
          const float* Wa = WY + c * RH * nx + (H + 2 * m) * nx;
          const float* Wb = Wa + nx;
          cx<float>* L = buf + line * lsx;
          const cx<float> w = dcx[k];
          cx<float> zk, zkp;
          if (k == 0) {
            dct_inv_pre(cx<float>{Wa[0], Wb[0]}, cx<float>{0.f, 0.f}, w.x, w.y, zk, zkp);
            const cx<float> Xm{Wa[hnx], Wb[hnx]};
            const cx<float> wm = dcx[hnx];
            cx<float> zm, zmp;
            dct_inv_pre(Xm, Xm, wm.x, wm.y, zm, zmp);
            L[pidx(0)] = cx<float>{zk.x, -zk.y};
            L[pidx(hnx)] = cx<float>{zm.x, -zm.y};
          } else {
            dct_inv_pre(cx<float>{Wa[k], Wb[k]}, cx<float>{Wa[nx - k], Wb[nx - k]}, w.x, w.y, zk, zkp);
            L[pidx(k)] = cx<float>{zk.x, -zk.y};
            L[pidx(nx - k)] = cx<float>{zkp.x, -zkp.y};
          }
        }
      }
      __syncthreads();
      cx<float>* cur = block_fft_loop<float, -1>(buf, alt, NCC * hR, lognx, lsx, twx, tid, nt);
      if (per) {
        post_inplace(cur, NCC * hR, lognx, lsx, d.bc, dcx);
        __syncthreads();
      }
      for (int q = tid; q < NCC * R * nx; q += nt) {
        const int c = q / (R * nx), rem = q - c * R * nx;
        const int r = rem >> lognx, j = rem & (nx - 1);
        const cx<float> v = cur[(c * hR + (r >> 1)) * lsx + pidx(per ? j : mk_slot(j, nx))];
        const float y = (r & 1) ? (per ? v.y : -v.y) : v.x;
        const float po = P[q];
        P[q] = po + tp * y;
        WY[c * RH * nx + (H + r) * nx + j] = po + tpe * y;
      }
    }
    cl.sync();  // 4
    // E. halo rows of P~; d_{n+1} = d_n - tau_u dF(u + d_n)^T P~ on own rows
    halo(WY);
    __syncthreads();
    for (int q = tid; q < R * nx; q += nt) {
      const int r = q >> lognx, j = q & (nx - 1);
      const int o0 = (H + r) * nx + j, o1 = RH * nx + o0;
      float s0 = X[o0], s1 = TWO ? X[o1] : 0.f;
      if constexpr (KT<K>::nonlinear) {
        s0 += B[o0];
        if constexpr (TWO) s1 += B[o1];
      }
      float g[2] = {0.f, 0.f};
      gradT_pt<float, K>(d, t0r, t1r, s0, s1, H + r, j, g);
      X[o0] -= tu * g[0];
      if constexpr (TWO) X[o1] -= tu * g[1];
    }
    cl.sync();  // 5
    halo(X);
    __syncthreads();
  }
  // own rows of the correction and (block 0) the final state back to global memory; the last
  // barrier keeps every block's shared memory alive until the others have read it
  float* gX = static_cast<float*>(d.X);
  for (int q = tid; q < NCC * R * nx; q += nt) {
    const int c = q / (R * nx), rem = q - c * R * nx;
    gX[(size_t)c * N + (size_t)y0 * nx + rem] = X[c * RH * nx + H * nx + rem];
  }
  if (rank == 0 && tid == 0) {
    s.trips = (unsigned)s.n + 1u;
    s.ticket = 0u;
    *gst = s;
  }
  cl.sync();
}

}  // namespace rd
