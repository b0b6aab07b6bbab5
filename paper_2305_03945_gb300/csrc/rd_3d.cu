// Kernels of the PDHG iteration on 3-D grids (see rd_3d.cuh) for single solves, their launchers,
// and the FP64 step-level kernels of 3-D grids (step set-up, FP64 residual of defect correction).
#include <algorithm>

#include "rd_3d.cuh"
#include "rd_launch3.h"

namespace rd {

template <class T, int K>
__global__ void __launch_bounds__(256) k3_res(const __grid_constant__ Desc d, State* __restrict__ st) {
  res3_body<T, K>(d, st, nullptr, blockIdx.x);
}

template <class T, int K>
__global__ void __launch_bounds__(256) k3_upd(const __grid_constant__ Desc d, State* __restrict__ st) {
  upd3_body<T, K>(d, st, nullptr, blockIdx.x);
}

template <class T, int AX, int MODE>
__global__ void __launch_bounds__(256) k3_lines(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  lines3_body<T, AX, MODE>(d, st, nullptr, blockIdx.x, smem_raw);
}

// The same passes for lines of 2^LOGN = 4096 and 8192 points (2-D grids beyond the band /
// column sweeps): blocks of 2^LOGN / 8 threads (one radix-8 job each per FFT pass: with two jobs
// per thread and 128 registers the passes spilled), the pass sequence fixed at compile time.
template <class T, int AX, int MODE, int LOGN>
__global__ void __launch_bounds__(LOGN > 12 ? 1024 : 512) k3_lines_long(const __grid_constant__ Desc d, State* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  lines3_body<T, AX, MODE, LOGN>(d, st, nullptr, blockIdx.x, smem_raw);
}

// rhs of the step from U^k (the explicit part of the convex split), ||U^k||^2 and a fresh solve
// state; d.blk3 blocks of 256 threads.
__global__ void __launch_bounds__(256) k3_begin(const Desc* __restrict__ d64, State* __restrict__ st,
                                                const double* __restrict__ uk, double* __restrict__ rhs, double tol,
                                                int tol_kind) {
  const Desc& d = *d64;
  __shared__ double red[32];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const G3<double> f{uk, d.nx, d.ny, d.nz, d.bc};
  double acc = 0.0;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    const double u = uk[q];
    double v = u;
    if (d.kind == RX_CH_SPLIT) {
      int l, i, j;
      point3(d, q, l, i, j);
      v = u - d.dt * d.b * lap7(f, l, i, j, u, d.hx2, d.hy2, d.hz2);
    }
    rhs[q] = v;
    acc += u * u;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[blockIdx.x] = s;
  if (last_block(st, gridDim.x)) {
    __threadfence();
    const double tot = sum_partials(d.partials, gridDim.x, red);
    if (threadIdx.x == 0) begin_state(st, tot, tol, tol_kind);
  }
}

// W = F(u) in FP64 on a 3-D grid, with the optional outputs and the outer decision of k_resid64.
template <int K>
__global__ void __launch_bounds__(256)
    k3_resid64(const Desc* __restrict__ d64, State* __restrict__ outer, State* __restrict__ inner,
               const double* __restrict__ u, const double* __restrict__ rhs, double* __restrict__ w64,
               float* __restrict__ r32, float* __restrict__ u32, float* __restrict__ z0, float* __restrict__ z1,
               int decide, double rtol, int max_outer) {
  if (decide && *((volatile const int*)&outer->status) != ST_ACTIVE) return;
  const Desc& d = *d64;
  __shared__ double red[32];
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const G3<double> f{u, d.nx, d.ny, d.nz, d.bc};
  double acc = 0.0;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    int l, i, j;
    point3(d, q, l, i, j);
    const double w = residual3_pt<double, K, false>(d, f, f, l, i, j, rhs[q]);
    if (w64) w64[q] = w;
    if (r32) r32[q] = (float)w;
    if (u32) u32[q] = (float)u[q];
    if (z0) z0[q] = 0.f;
    if (z1) z1[q] = 0.f;
    acc += w * w;
  }
  if (!decide) return;
  const int nb = gridDim.x;
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) d.partials[blockIdx.x] = s;
  if (last_block(outer, nb)) {
    __threadfence();
    const double tot = sqrt(sum_partials(d.partials, nb, red));
    if (threadIdx.x == 0) outer_decide(d, outer, inner, tot, rtol, max_outer);
  }
}

namespace {

inline cudaError_t record(cudaStream_t s, cudaEvent_t* ev, int i, unsigned flags) {
  return ev ? cudaEventRecordWithFlags(ev[i], s, flags) : cudaSuccess;
}

template <class T, int AX, int MODE>
cudaError_t launch_lines(const Desc& d, State* st, cudaStream_t s) {
  const int n = AX == 0 ? d.nx : (AX == 1 ? d.ny : d.nz);
  const bool pf = AX == 0 && MODE == L3_INVP && sizeof(T) == 4 && d.thr3[AX] > 256 && d.pf3;
  const int smem = lines3_smem_bytes<T>(n, d.lw3[AX], d.bc == BC_NEUMANN, pf);
  // the passes of a 2-D grid (x: forward, inverse with the dual update, inverse; y: the scaled
  // pass) on lines of 4096 and 8192 points, which plan3 gives n / 8 threads
  constexpr bool two_d_pass = (AX == 0 && (MODE == L3_FWD || MODE == L3_INVP || MODE == L3_INVX)) ||
                              (AX == 1 && MODE == L3_FSI);
  if constexpr (two_d_pass) {
    if (d.thr3[AX] > 256) {
      if (n == 8192) {
        k3_lines_long<T, AX, MODE, 13><<<d.blk3, d.thr3[AX], smem, s>>>(d, st);
      } else if constexpr (sizeof(T) == 4) {
        k3_lines_long<T, AX, MODE, 12><<<d.blk3, d.thr3[AX], smem, s>>>(d, st);
      } else {
        return cudaErrorNotSupported;  // FP64 lines up to 4096 points run on the band / column sweeps
      }
      return cudaGetLastError();
    }
  }
  k3_lines<T, AX, MODE><<<d.blk3, d.thr3[AX], smem, s>>>(d, st);
  return cudaGetLastError();
}

template <class T, int K>
cudaError_t launch_iter3_k(const Desc& d, State* st, cudaStream_t s, cudaEvent_t* ev) {
  unsigned flags = cudaEventRecordDefault;
  if (ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive) flags = cudaEventRecordExternal;
  }
  cudaError_t e = record(s, ev, 0, flags);
  if (e == cudaSuccess) {
    k3_res<T, K><<<d.blk3, 256, 0, s>>>(d, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = record(s, ev, 1, flags);
  if (d.precond != 0) {
    if (e == cudaSuccess) e = launch_lines<T, 0, L3_FWD>(d, st, s);
    if (d.nz > 1) {
      if (e == cudaSuccess) e = launch_lines<T, 1, L3_FWD>(d, st, s);
      if (e == cudaSuccess) e = launch_lines<T, 2, L3_FSI>(d, st, s);
      if (e == cudaSuccess) e = launch_lines<T, 1, L3_INV>(d, st, s);
    } else if (e == cudaSuccess) {
      e = launch_lines<T, 1, L3_FSI>(d, st, s);  // 2-D grid: the scaling on the y pass
    }
    if (e == cudaSuccess) e = launch_lines<T, 0, L3_INVP>(d, st, s);
  }
  if (e == cudaSuccess) e = record(s, ev, 2, flags);
  if (e == cudaSuccess) {
    k3_upd<T, K><<<d.blk3, 256, 0, s>>>(d, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = record(s, ev, 3, flags);
  return e;
}

template <class K_>
cudaError_t allow3_k(K_ kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace

template <class T>
cudaError_t launch_iteration3(const Desc& d, State* st, cudaStream_t s, cudaEvent_t* ev) {
  if (d.precond == 0 && d.mode == MODE_PRECOND_ONLY) return cudaErrorInvalidValue;
  switch (kind_key(d)) {
    case KK_NONE_LAP: return launch_iter3_k<T, KK_NONE_LAP>(d, st, s, ev);
    case KK_AC: return launch_iter3_k<T, KK_AC>(d, st, s, ev);
    case KK_CH_IMPL: return launch_iter3_k<T, KK_CH_IMPL>(d, st, s, ev);
    case KK_CH_SPLIT: return launch_iter3_k<T, KK_CH_SPLIT>(d, st, s, ev);
    case KK_NONE_BIH: return launch_iter3_k<T, KK_NONE_BIH>(d, st, s, ev);
    default: return cudaErrorNotSupported;
  }
}

template <class T>
cudaError_t launch_precond3(const Desc& d, State* st, cudaStream_t s) {
  cudaError_t e = launch_lines<T, 0, L3_FWD>(d, st, s);
  if (d.nz > 1) {
    if (e == cudaSuccess) e = launch_lines<T, 1, L3_FWD>(d, st, s);
    if (e == cudaSuccess) e = launch_lines<T, 2, L3_FSI>(d, st, s);
    if (e == cudaSuccess) e = launch_lines<T, 1, L3_INV>(d, st, s);
  } else if (e == cudaSuccess) {
    e = launch_lines<T, 1, L3_FSI>(d, st, s);
  }
  if (e == cudaSuccess) e = launch_lines<T, 0, L3_INVX>(d, st, s);
  return e;
}

template <class T, int LOGN>
cudaError_t allow_long(int optin) {
  cudaError_t e;
  if ((e = allow3_k(k3_lines_long<T, 0, L3_FWD, LOGN>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines_long<T, 1, L3_FSI, LOGN>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines_long<T, 0, L3_INVP, LOGN>, optin)) != cudaSuccess) return e;
  return allow3_k(k3_lines_long<T, 0, L3_INVX, LOGN>, optin);
}

template <class T>
cudaError_t allow3(int optin) {
  cudaError_t e;
  if ((e = allow3_k(k3_lines<T, 0, L3_FWD>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 1, L3_FWD>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 2, L3_FSI>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 1, L3_FSI>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 1, L3_INV>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 0, L3_INVP>, optin)) != cudaSuccess) return e;
  if ((e = allow3_k(k3_lines<T, 0, L3_INVX>, optin)) != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4)
    if ((e = allow_long<T, 12>(optin)) != cudaSuccess) return e;
  return allow_long<T, 13>(optin);
}

template cudaError_t launch_iteration3<float>(const Desc&, State*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_iteration3<double>(const Desc&, State*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_precond3<double>(const Desc&, State*, cudaStream_t);
template cudaError_t allow3<float>(int);
template cudaError_t allow3<double>(int);

bool plan3(int nx, int ny, int nz, int nc, int elem_bytes, bool neumann, int smem_limit, Desc& d, const char** why) {
  const size_t npts = (size_t)nx * ny * nz;
  d.pf3 = 0;
  d.blk3 = (int)std::max<size_t>(1, std::min<size_t>(1024, (npts + 2047) / 2048));
  const int n_ax[3] = {nx, ny, nz};
  const int lanes = elem_bytes == 4 ? 16 : 8;
  // lines available to a tile: x passes take consecutive rows, y and z passes adjacent x columns
  const int avail[3] = {nc * ny * nz, nx, nx};
  for (int a = 0; a < 3; ++a) {
    const int n = n_ax[a];
    const int line_thr = n >= 8 ? n / 8 : 1;
    if (line_thr > 256) {
      // 2-D grids only (nz = 1): x and y lines of up to 8192 points, one or two pair lines per
      // tile, on blocks of n / 8 threads
      if (nz > 1 || n > 8192) {
        *why = nz > 1 ? "3-D grid side longer than a 256-thread block transforms (2048 points)"
                      : "grid side longer than 8192 points";
        return false;
      }
      const int smem = elem_bytes == 4 ? lines3_smem_bytes<float>(n, 2, neumann) : lines3_smem_bytes<double>(n, 2, neumann);
      if (smem > smem_limit) {
        *why = "transform line does not fit in shared memory";
        return false;
      }
      // y (column) tiles: two pair lines when they fit, for 16-byte row segments (measured on
      // 8192^2 in FP32: the three transform passes of an iteration 1.87 -> 1.55 ms)
      int lwl = 2;
      if (a == 1 && nx >= 4) {
        const int s4 = elem_bytes == 4 ? lines3_smem_bytes<float>(n, 4, neumann) : lines3_smem_bytes<double>(n, 4, neumann);
        if (s4 <= smem_limit) lwl = 4;
      }
      d.lw3[a] = lwl;
      d.thr3[a] = line_thr;
      // x lines in FP32: the inverse pass with the dual update prefetches its rows of P
      if (a == 0 && elem_bytes == 4) d.pf3 = lines3_smem_bytes<float>(n, lwl, neumann, true) <= smem_limit;
      continue;
    }
    int lw = std::min(lanes, avail[a]);
    if (lw < 2) lw = 2;
    auto smem = [&](int w) {
      return (elem_bytes == 4 ? lines3_smem_bytes<float>(n, w, neumann) : lines3_smem_bytes<double>(n, w, neumann));
    };
    while (lw > 2 && smem(lw) > smem_limit / 2) lw >>= 1;
    if (smem(lw) > smem_limit) {
      *why = "3-D transform tile does not fit in shared memory";
      return false;
    }
    int thr = (lw / 2) * line_thr;
    thr = std::max(thr, line_thr);
    thr = std::max(32, std::min(256, (thr + 31) / 32 * 32));
    d.lw3[a] = lw;
    d.thr3[a] = thr;
  }
  return true;
}

cudaError_t launch_begin3(const Desc& hd, const Desc* d64, State* st, const double* uk, double* rhs, double tol,
                          int tol_kind, cudaStream_t s) {
  k3_begin<<<hd.blk3, 256, 0, s>>>(d64, st, uk, rhs, tol, tol_kind);
  return cudaGetLastError();
}

cudaError_t launch_resid64_3(const Desc& hd, const Desc* d64, State* outer, State* inner, const double* u,
                             const double* rhs, double* w64, float* r32, float* u32, float* z0, float* z1, int decide,
                             double rtol, int max_outer, cudaStream_t s) {
  const int g = hd.blk3;
  switch (kind_key(hd)) {
    case KK_AC: k3_resid64<KK_AC><<<g, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_CH_IMPL: k3_resid64<KK_CH_IMPL><<<g, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_CH_SPLIT: k3_resid64<KK_CH_SPLIT><<<g, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    case KK_NONE_BIH: k3_resid64<KK_NONE_BIH><<<g, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
    default: k3_resid64<KK_NONE_LAP><<<g, 256, 0, s>>>(d64, outer, inner, u, rhs, w64, r32, u32, z0, z1, decide, rtol, max_outer); break;
  }
  return cudaGetLastError();
}

}  // namespace rd
