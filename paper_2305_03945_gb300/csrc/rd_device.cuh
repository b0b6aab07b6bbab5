// Device building blocks of the PDHG sweeps: complex arithmetic, the block-cooperative
// shared-memory Stockham FFT, the real-pair Hartley / DCT-II / DCT-III line transforms that
// diagonalise the periodic and Neumann Laplacians, boundary index maps and stencils.
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

template <class T> struct cx { T x, y; };

template <class T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }

__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// a * w for the forward transform (DIR < 0) or a * conj(w) for the inverse (DIR > 0), where the
// twiddle table holds w_k = exp(-2 pi i k / N).
template <class T, int DIR>
__device__ __forceinline__ cx<T> cmul_tw(cx<T> a, cx<T> w) {
  if (DIR < 0) return {a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x};
  return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
}

// cos(2 pi q / 16) for integer q
template <class T>
__device__ __forceinline__ T cos16(int q) {
  switch (q & 15) {
    case 0: return T(1);
    case 1: case 15: return T(0.92387953251128675613);
    case 2: case 14: return T(0.70710678118654752440);
    case 3: case 13: return T(0.38268343236508977173);
    case 4: case 12: return T(0);
    case 5: case 11: return T(-0.38268343236508977173);
    case 6: case 10: return T(-0.70710678118654752440);
    case 7: case 9: return T(-0.92387953251128675613);
    default: return T(-1);
  }
}

// v * exp(DIR * 2 pi i q / 16); q is a compile-time constant after unrolling.
template <class T, int DIR>
__device__ __forceinline__ cx<T> mul_w16(cx<T> v, int q) {
  q &= 15;
  if (q == 0) return v;
  if (q == 8) return {-v.x, -v.y};
  if (q == 4) return DIR < 0 ? cx<T>{v.y, -v.x} : cx<T>{-v.y, v.x};
  if (q == 12) return DIR < 0 ? cx<T>{-v.y, v.x} : cx<T>{v.y, -v.x};
  const T c = cos16<T>(q);
  const T s = T(DIR) * cos16<T>(q - 4);  // DIR * sin(2 pi q / 16)
  return {v.x * c - v.y * s, v.x * s + v.y * c};
}

// In-register DFT of length R (2, 4, 8 or 16): v[k] <- sum_m v[m] exp(DIR 2 pi i m k / R),
// radix-2 decimation in time on bit-reversed input.  All loops have unit stride and constant
// trip counts so that v stays in registers.
template <class T, int R, int DIR>
__device__ __forceinline__ void dft_reg(cx<T>* v) {
  constexpr int LOGR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int j = 0;
#pragma unroll
    for (int b = 0; b < LOGR; ++b) j |= ((i >> b) & 1) << (LOGR - 1 - b);
    if (j > i) {
      const cx<T> t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int st = 0; st < LOGR; ++st) {
    const int half = 1 << st;
#pragma unroll
    for (int s = 0; s < R / (2 * half); ++s) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int i0 = s * 2 * half + k;
        const cx<T> a = v[i0];
        const cx<T> b = mul_w16<T, DIR>(v[i0 + half], k * (8 >> st));
        v[i0] = cadd(a, b);
        v[i0 + half] = csub(a, b);
      }
    }
  }
}

// Values each FFT thread holds per Stockham pass (radix 8), and the block-size cap of the sweep
// kernels: FP32 blocks of <= 256 threads at <= 128 registers (two blocks per SM: the sweep
// grids put at most two blocks on an SM, and at 80 registers the transform passes spilled),
// FP64 blocks of <= 512 threads at <= 128 registers.  One line of length N needs N/8 threads,
// so rows and columns are limited to 2048 points in FP32 and 4096 in FP64.
template <class T> struct FftRadix { static constexpr int value = 8; };
template <class T> struct MaxThreads { static constexpr int value = sizeof(T) == 4 ? 256 : 512; };
template <class T> struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

// Threads needed to transform ONE line of length N in one go.
template <class T>
__host__ __device__ inline int fft_line_threads(int N) {
  const int r = FftRadix<T>::value;
  return N >= r ? N / r : 1;
}

template <class T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Twiddles w^r, r = 1..R-1, of one Stockham job from the table entries w^1, w^2, w^4, w^8
// (w = exp(-2 pi i step / N)) and products of them.  The table lives in shared memory.
template <class T, int R>
__device__ __forceinline__ void job_twiddles(const cx<T>* __restrict__ tw, int step, cx<T>* w) {
  w[1] = tw[step];
  if constexpr (R > 2) {
    w[2] = tw[2 * step];
    w[3] = cmul(w[1], w[2]);
  }
  if constexpr (R > 4) {
    w[4] = tw[4 * step];
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
  }
  if constexpr (R > 8) {
    w[8] = tw[8 * step];
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
  }
}

// One Stockham pass of radix R (Govindaraju et al., SC 2008 formulation): job j of a line reads
// entries j + r N/R of src, twiddles them by w^{r (j mod Ns) N/(Ns R)}, applies the radix-R DFT
// and writes entries (j div Ns) Ns R + (j mod Ns) + r Ns of dst.  With src == dst all reads
// happen before a barrier and all writes after it.  Sizes enter as base-2 logarithms.  Each
// thread holds J * RM / R jobs (J radix-RM jobs' worth of values), so that J > 1 lets a block
// transform lines of up to J * RM points per thread.
template <class T, int R, int DIR, int J = 1>
__device__ __forceinline__ void stockham_pass(const cx<T>* src, cx<T>* dst, int nlines, int logN, int ls, int logNs,
                                              const cx<T>* __restrict__ tw, int tid) {
  constexpr int RM = FftRadix<T>::value;
  constexpr int S = J * RM / R;
  constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
  const int lj = logN - LR;  // log2 jobs per line
  const int jpl = 1 << lj;
  const int total = nlines << lj;
  const int nthr = (total + S - 1) / S;
  const int Ns = 1 << logNs;
  const int tws = logN - logNs - LR;  // log2(N / (Ns R))
  cx<T> v[S][R];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = tid + s * nthr;
    if (tid < nthr && g < total) {
      const cx<T>* L = src + (g >> lj) * ls;
      const int j = g & (jpl - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[s][r] = L[pidx(j + (r << lj))];
    }
  }
  if (src == dst) __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = tid + s * nthr;
    if (tid < nthr && g < total) {
      const int j = g & (jpl - 1);
      const int k = j & (Ns - 1);
      if (k != 0) {
        cx<T> w[R];
        job_twiddles<T, R>(tw, k << tws, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[s][r] = cmul_tw<T, DIR>(v[s][r], w[r]);
      }
      dft_reg<T, R, DIR>(v[s]);
      cx<T>* L = dst + (g >> lj) * ls;
      const int d = ((j - k) << LR) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) L[pidx(d + (r << logNs))] = v[s][r];
    }
  }
  __syncthreads();
}

// Stockham pass with every size known at compile time.  With the padding pidx(i) = i + i/16,
// element r of a job sits at a constant offset from element 0 whenever the stride between the
// elements is a multiple of 16 (or the job's elements are contiguous), so the index arithmetic
// folds into immediate offsets.
template <class T, int R, int DIR, int LOGN, int LOGNS>
__device__ __forceinline__ void stockham_pass_c(const cx<T>* src, cx<T>* dst, int nlines, int ls,
                                                const cx<T>* __restrict__ tw, int tid) {
  constexpr int RM = FftRadix<T>::value;
  constexpr int S = RM / R;
  constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
  constexpr int LJ = LOGN - LR;
  constexpr int JPL = 1 << LJ;
  constexpr int NS = 1 << LOGNS;
  constexpr int TWS = LOGN - LOGNS - LR;
  constexpr bool LD_CONST = (JPL % 16) == 0;
  constexpr int LD_STRIDE = JPL + JPL / 16;
  constexpr bool ST_CONST = NS == 1 || (NS % 16) == 0;
  constexpr int ST_STRIDE = NS == 1 ? 1 : NS + NS / 16;
  const int total = nlines << LJ;
  const int nthr = (total + S - 1) / S;
  cx<T> v[S][R];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = tid + s * nthr;
    if (tid < nthr && g < total) {
      const cx<T>* L = src + (g >> LJ) * ls;
      const int j = g & (JPL - 1);
      if constexpr (LD_CONST) {
        const cx<T>* p = L + pidx(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][r] = p[r * LD_STRIDE];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][r] = L[pidx(j + (r << LJ))];
      }
    }
  }
  if (src == dst) __syncthreads();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int g = tid + s * nthr;
    if (tid < nthr && g < total) {
      const int j = g & (JPL - 1);
      const int k = j & (NS - 1);
      if (NS > 1 && k != 0) {
        cx<T> w[R];
        job_twiddles<T, R>(tw, k << TWS, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[s][r] = cmul_tw<T, DIR>(v[s][r], w[r]);
      }
      dft_reg<T, R, DIR>(v[s]);
      cx<T>* L = dst + (g >> LJ) * ls;
      const int d = ((j - k) << LR) + k;
      if constexpr (ST_CONST) {
        cx<T>* p = L + pidx(d);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * ST_STRIDE] = v[s][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) L[pidx(d + (r << LOGNS))] = v[s][r];
      }
    }
  }
  __syncthreads();
}

// Radix plan of a length-2^LOGN transform: passes of radix 8 from Ns = 1, the remainder last.
// Each pass reads `a` and writes `b` (the same buffer when b == a); returns the buffer holding
// the result.
template <class T, int DIR, int LOGN, int LOGNS>
__device__ __forceinline__ cx<T>* fft_passes_c(cx<T>* a, cx<T>* b, int nlines, int ls, const cx<T>* __restrict__ tw,
                                               int tid) {
  constexpr int RM = FftRadix<T>::value;
  constexpr int LRM = RM == 8 ? 3 : 4;
  constexpr int REM = LOGN - LOGNS;
  if constexpr (REM > 0) {
    constexpr int B = REM >= LRM ? LRM : REM;
    constexpr int R = 1 << B;
    stockham_pass_c<T, R, DIR, LOGN, LOGNS>(a, b, nlines, ls, tw, tid);
    return fft_passes_c<T, DIR, LOGN, LOGNS + B>(b, a, nlines, ls, tw, tid);
  } else {
    return a;
  }
}

template <class T, int DIR, int LOGN>
__device__ __forceinline__ cx<T>* block_fft_c(cx<T>* buf, cx<T>* scr, int nlines, int ls,
                                              const cx<T>* __restrict__ tw, int tid, int nthreads) {
  constexpr int RM = FftRadix<T>::value;
  int chunk = (nthreads * RM) >> LOGN;
  if (chunk < 1) chunk = 1;
  cx<T>* res = buf;
  for (int l0 = 0; l0 < nlines; l0 += chunk) {
    const int nl = nlines - l0 < chunk ? nlines - l0 : chunk;
    res = fft_passes_c<T, DIR, LOGN, 0>(buf + l0 * ls, scr + l0 * ls, nl, ls, tw, tid) - l0 * ls;
  }
  return res;
}

// Unnormalised complex DFT of `nlines` padded lines in shared memory (DIR = -1 forward,
// +1 inverse), in chunks of as many lines as `nthreads` threads can hold, ping-ponging between
// buf and scr (one barrier per pass), or in place when scr == buf (two barriers per pass, half
// the shared memory).  Returns the buffer (buf or scr) that holds the result.
// Called by every thread of the block (it contains barriers); needs nthreads >=
// fft_line_threads<T>(N).  With `unrolled`, lengths 64 .. 2048 run passes specialised and
// unrolled at compile time for that length; otherwise one looped pass body serves every pass
// (fewer distinct instructions, more index arithmetic; measured slower on GB300).
// block_fft_loop with J > 1 holds J radix-8 jobs per thread and pass, for lines longer than
// 8 x nthreads points (it needs nthreads * 8 * J >= N).
template <class T, int DIR, int J = 1>
__device__ cx<T>* block_fft_loop(cx<T>* buf, cx<T>* scr, int nlines, int logN, int ls, const cx<T>* __restrict__ tw,
                                 int tid, int nthreads);

template <class T, int DIR>
__device__ cx<T>* block_fft(cx<T>* buf, cx<T>* scr, int nlines, int logN, int ls, const cx<T>* __restrict__ tw,
                            int tid, int nthreads, bool unrolled) {
  if (unrolled) switch (logN) {
    case 6: return block_fft_c<T, DIR, 6>(buf, scr, nlines, ls, tw, tid, nthreads);
    case 7: return block_fft_c<T, DIR, 7>(buf, scr, nlines, ls, tw, tid, nthreads);
    case 8: return block_fft_c<T, DIR, 8>(buf, scr, nlines, ls, tw, tid, nthreads);
    case 9: return block_fft_c<T, DIR, 9>(buf, scr, nlines, ls, tw, tid, nthreads);
    case 10: return block_fft_c<T, DIR, 10>(buf, scr, nlines, ls, tw, tid, nthreads);
    case 11: return block_fft_c<T, DIR, 11>(buf, scr, nlines, ls, tw, tid, nthreads);
    default: break;
  }
  return block_fft_loop<T, DIR>(buf, scr, nlines, logN, ls, tw, tid, nthreads);
}

// The looped form of block_fft: one pass body for every pass of every length.
template <class T, int DIR, int J>
__device__ cx<T>* block_fft_loop(cx<T>* buf, cx<T>* scr, int nlines, int logN, int ls, const cx<T>* __restrict__ tw,
                                 int tid, int nthreads) {
  constexpr int RM = FftRadix<T>::value;
  constexpr int LRM = RM == 8 ? 3 : 4;
  int chunk = (nthreads * RM * J) >> logN;
  if (chunk < 1) chunk = 1;
  cx<T>* res = buf;
  for (int l0 = 0; l0 < nlines; l0 += chunk) {
    const int nl = nlines - l0 < chunk ? nlines - l0 : chunk;
    cx<T>* a = buf + l0 * ls;
    cx<T>* b = scr + l0 * ls;
    int logNs = 0, rem = logN;
    while (rem > 0) {
      const int bb = rem >= LRM ? LRM : rem;
      if (bb == 4) stockham_pass<T, (RM >= 16 ? 16 : RM), DIR, J>(a, b, nl, logN, ls, logNs, tw, tid);
      else if (bb == 3) stockham_pass<T, 8, DIR, J>(a, b, nl, logN, ls, logNs, tw, tid);
      else if (bb == 2) stockham_pass<T, 4, DIR, J>(a, b, nl, logN, ls, logNs, tw, tid);
      else stockham_pass<T, 2, DIR, J>(a, b, nl, logN, ls, logNs, tw, tid);
      cx<T>* t = a;
      a = b;
      b = t;
      logNs += bb;
      rem -= bb;
    }
    res = a - l0 * ls;
  }
  return res;
}

// Transform of lines of a length 2^LOGN known at compile time (lines of 4096 and 8192 points),
// with J radix-8 jobs per thread and pass: the pass sequence unrolled at compile time, in place,
// as block_fft_loop with scr == buf.
template <class T, int DIR, int J, int LOGN, int LOGNS>
__device__ __forceinline__ void fft_passes_j(cx<T>* a, int nlines, int ls, const cx<T>* __restrict__ tw, int tid) {
  constexpr int REM = LOGN - LOGNS;
  if constexpr (REM > 0) {
    constexpr int B = REM >= 3 ? 3 : REM;
    stockham_pass<T, 1 << B, DIR, J>(a, a, nlines, LOGN, ls, LOGNS, tw, tid);
    fft_passes_j<T, DIR, J, LOGN, LOGNS + B>(a, nlines, ls, tw, tid);
  }
}

// (the line stride is padded_len(2^LOGN), a compile-time constant: with it the index arithmetic
// of the passes folds into immediates)
template <class T, int DIR, int J, int LOGN>
__device__ __forceinline__ cx<T>* block_fft_long(cx<T>* buf, int nlines, const cx<T>* __restrict__ tw, int tid,
                                                 int nthreads) {
  constexpr int RM = FftRadix<T>::value;
  constexpr int LS = ((1 << LOGN) + (1 << (LOGN - 4)) + 2) & ~1;
  int chunk = (nthreads * RM * J) >> LOGN;
  if (chunk < 1) chunk = 1;
  for (int l0 = 0; l0 < nlines; l0 += chunk) {
    const int nl = nlines - l0 < chunk ? nlines - l0 : chunk;
    fft_passes_j<T, DIR, J, LOGN, 0>(buf + l0 * LS, nl, LS, tw, tid);
  }
  return buf;
}

// ---------------------------------------------------------------------------------------
// Real-pair line transforms.  A complex line holds two real lines a (.x) and b (.y).
//   periodic : separable discrete Hartley transform H[k] = sum_j x_j cas(2 pi j k / N); the
//              cas vectors are eigenvectors of the periodic second difference, and H H = N I.
//   Neumann  : DCT-II X[k] = sum_j x_j cos(pi k (2j+1) / (2N)) by Makhoul's N-point method
//              (J. Makhoul, IEEE TASSP 1980): reorder even samples ascending and odd samples
//              descending, DFT, rotate by exp(-i pi k / 2N); its exact inverse (DCT-III up to
//              the factor N) runs the same steps backwards.
// ---------------------------------------------------------------------------------------

// Makhoul reordering: slot n of the reordered line holds sample perm(n).
__device__ __forceinline__ int mk_perm(int n, int N) { return n < (N >> 1) ? 2 * n : 2 * (N - 1 - n) + 1; }
// slot that holds sample j
__device__ __forceinline__ int mk_slot(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }

// Forward epilogue for frequency k in [0, N/2] of a pair line whose complex DFT is L.
// Returns the real-transform coefficients (a_k, b_k) in ok and (a_{N-k}, b_{N-k}) in okp
// (okp is meaningful only for 0 < k).
template <class T>
__device__ __forceinline__ void fwd_post(const cx<T>* L, int N, int bc, const cx<T>* __restrict__ dc,
                                         int k, cx<T>& ok, cx<T>& okp) {
  const int kp = (N - k) & (N - 1);
  const cx<T> z = L[pidx(k)], zp = L[pidx(kp)];
  if (bc == BC_PERIODIC) {
    ok.x = T(0.5) * (z.x + zp.x - z.y + zp.y);
    ok.y = T(0.5) * (z.x - zp.x + z.y + zp.y);
    okp.x = T(0.5) * (zp.x + z.x - zp.y + z.y);
    okp.y = T(0.5) * (zp.x - z.x + zp.y + z.y);
  } else {
    const cx<T> w = dc[k];  // (cos, sin)(pi k / 2N)
    const T c = w.x, s = w.y;
    ok.x = T(0.5) * (c * (z.x + zp.x) + s * (z.y - zp.y));
    ok.y = T(0.5) * (c * (z.y + zp.y) - s * (z.x - zp.x));
    okp.x = T(0.5) * (s * (zp.x + z.x) + c * (zp.y - z.y));
    okp.y = T(0.5) * (s * (zp.y + z.y) - c * (zp.x - z.x));
  }
}

// Inverse-DCT prologue for frequency k in [0, N/2]: from coefficients X_k = (a_k, b_k) and
// X_{N-k} (zero when k = 0) build the complex DFT inputs z_k and z_{N-k} of the reordered
// pair line.
template <class T>
__device__ __forceinline__ void dct_inv_pre(cx<T> Xk, cx<T> Xkp, T c, T s, cx<T>& zk, cx<T>& zkp) {
  zk.x = c * Xk.x + s * Xkp.x - s * Xk.y + c * Xkp.y;
  zk.y = s * Xk.x - c * Xkp.x + c * Xk.y + s * Xkp.y;
  zkp.x = s * Xkp.x + c * Xk.x - c * Xkp.y + s * Xk.y;
  zkp.y = c * Xkp.x - s * Xk.x + s * Xkp.y + c * Xk.y;
}

// In-place epilogue over all lines: slot k <- forward coefficients (optionally multiplied by
// per-slot scale factors).
template <class T>
__device__ __forceinline__ void fwd_post_inplace(cx<T>* buf, int nlines, int N, int ls, int bc,
                                                 const cx<T>* __restrict__ dc, int tid, int nthreads) {
  const int half = (N >> 1) + 1;
  for (int g = tid; g < nlines * half; g += nthreads) {
    const int line = g / half, k = g - line * half;
    cx<T>* L = buf + line * ls;
    cx<T> ok, okp;
    fwd_post(L, N, bc, dc, k, ok, okp);
    L[pidx(k)] = ok;
    if (k != 0) L[pidx(N - k)] = okp;
  }
}

// ---------------------------------------------------------------------------------------
// boundary index map and stencils
// ---------------------------------------------------------------------------------------

// Index i in [-2, n+1] mapped into [0, n): periodic wrap, or the half-cell mirror
// U_{-1} = U_0, U_{-2} = U_1, U_n = U_{n-1}, U_{n+1} = U_{n-2} (Remark 1).  Needs n >= 2.
__device__ __forceinline__ int bcmap(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == BC_PERIODIC) return i < 0 ? i + n : i - n;
  return i < 0 ? -1 - i : 2 * n - 1 - i;
}

template <class T>
struct GField {  // one component of a grid array in global memory
  const T* __restrict__ p;
  int nx, ny, bc;
  __device__ __forceinline__ T operator()(int i, int j) const {
    return p[(size_t)bcmap(i, ny, bc) * nx + bcmap(j, nx, bc)];
  }
};

// five-point Laplacian at (i, j) with centre value c
template <class T, class F>
__device__ __forceinline__ T lap5(const F& f, int i, int j, T c, T hx2, T hy2) {
  return (f(i, j + 1) + f(i, j - 1) - T(2) * c) * hx2 + (f(i + 1, j) + f(i - 1, j) - T(2) * c) * hy2;
}

// thirteen-point Lap^2 = Dxx^2 + 2 Dxx Dyy + Dyy^2 on the periodic / two-deep mirror extension
template <class T, class F>
__device__ __forceinline__ T lap13(const F& f, int i, int j, T c, T hx2, T hy2) {
  const T e = f(i, j + 1), w = f(i, j - 1), n = f(i + 1, j), s = f(i - 1, j);
  const T xx = f(i, j + 2) - T(4) * (e + w) + T(6) * c + f(i, j - 2);
  const T yy = f(i + 2, j) - T(4) * (n + s) + T(6) * c + f(i - 2, j);
  const T xy = f(i + 1, j + 1) + f(i + 1, j - 1) + f(i - 1, j + 1) + f(i - 1, j - 1) -
               T(2) * (e + w + n + s) + T(4) * c;
  return xx * (hx2 * hx2) + T(2) * xy * (hx2 * hy2) + yy * (hy2 * hy2);
}

// Shared-memory bytes of the residual band kernel: the complex transform buffer first, then
// the staged real rows of the unknown (and of the defect-correction base state); every region
// starts 16-byte aligned.
// FP32 sweeps keep their twiddle / DCT rotation tables in shared memory; FP64 sweeps (which
// need twice the bytes per line) read them from global memory.
template <class T> struct SmemTables { static constexpr bool value = sizeof(T) == 4; };

// Entries of the twiddle table that transforms of length n read: w^k for k < n/2 only (a
// radix-R pass, R <= 8, reads w^step, w^(2 step), w^(4 step) up to w^((R/2) step) with
// step < n/R; see job_twiddles), rounded up to an even count so that what follows in shared
// memory stays 16-byte aligned.
__host__ __device__ inline int tw_entries(int n) { return n >= 4 ? n >> 1 : 2; }
// Shared-memory bytes of the tables a sweep block loads: the half twiddle table (tw) and the
// DCT rotation table of n entries (dc); none for FP64, whose tables stay in global memory.
template <class T>
__host__ __device__ inline int table_bytes(int n, bool tw, bool dc) {
  if (!SmemTables<T>::value) return 0;
  return ((tw ? tw_entries(n) : 0) + (dc ? n : 0)) * (int)sizeof(cx<T>);
}

template <class T>
__host__ __device__ inline int res_smem_bytes(int nc, int rows, int H, int nx, int stage_base, int pp, int tabs) {
  const int ls = padded_len(nx);
  const int buf = nc * (rows >> 1) * ls * (int)sizeof(cx<T>) * (pp ? 2 : 1);
  const int stg = nc * (rows + 2 * H) * nx * (int)sizeof(T);
  return tabs + buf + stg * (stage_base ? 2 : 1);
}

// Shared-memory bytes of a kernel holding `nlines` transform lines of length n plus the
// twiddle and DCT rotation tables of that length.
template <class T>
__host__ __device__ inline int lines_smem_bytes(int nlines, int n, int pp, int tabs) {
  return tabs + nlines * padded_len(n) * (pp ? 2 : 1) * (int)sizeof(cx<T>);
}

// Copy n entries of a complex table from global to shared memory (called by the whole block).
template <class T>
__device__ __forceinline__ void load_table(cx<T>* dst, const cx<T>* __restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = ldg(src + k);
}

// The twiddle / rotation tables a sweep reads: staged into shared memory at `smem` (FP32) or
// the global tables themselves (FP64).  Returns the first shared-memory byte after the tables.
template <class T>
__device__ __forceinline__ unsigned char* place_tables(unsigned char* smem, const void* tw_g, const void* dc_g, int n,
                                                       bool load_tw, bool load_dc, const cx<T>*& tw,
                                                       const cx<T>*& dc) {
  if constexpr (SmemTables<T>::value) {
    cx<T>* t = reinterpret_cast<cx<T>*>(smem);
    if (load_tw) load_table(t, static_cast<const cx<T>*>(tw_g), tw_entries(n));
    tw = t;
    if (load_tw) t += tw_entries(n);
    if (load_dc) load_table(t, static_cast<const cx<T>*>(dc_g), n);
    dc = t;
    if (load_dc) t += n;
    return reinterpret_cast<unsigned char*>(t);
  } else {
    tw = static_cast<const cx<T>*>(tw_g);
    dc = static_cast<const cx<T>*>(dc_g);
    return smem;
  }
}

// block-wide sum of a double, valid in thread 0; sh must hold 32 doubles
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0;
  if (warp == 0) {
    t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

}  // namespace rd
