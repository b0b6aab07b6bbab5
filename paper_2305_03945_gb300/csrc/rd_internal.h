// Internal types shared by the host runtime and the sm_103a kernels of the PDHG solver.
#pragma once

#include <cstddef>
#include <cstdint>

namespace rd {

enum Bc { BC_PERIODIC = 0, BC_NEUMANN = 1 };
enum Op { OP_LAP = 0, OP_BIHARM = 1 };
enum Kind { RX_NONE = 0, RX_AC = 1, RX_CH_IMPL = 2, RX_CH_SPLIT = 3, RX_GS = 4, RX_SCHNAK = 5 };
enum Mode { MODE_PDHG = 0, MODE_PRECOND_ONLY = 1 };

// per-solve status kept on the device
enum StStatus { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_NOT_CONVERGED = 2, ST_DIVERGED = 3, ST_IDLE = 4 };

constexpr double kDivergeFactor = 1e8;  // measure > 1e8 * first measure  ->  diverged
constexpr int kRadix = 16;              // values each FFT thread holds per Stockham pass

// Padded index inside a shared-memory complex line: one pad slot every 16 entries, so that the
// stride-16 stores of the first Stockham pass spread over all banks.
__host__ __device__ inline int pidx(int i) { return i + (i >> 4); }
// line stride in complex entries; even, so every line starts 16-byte aligned
__host__ __device__ inline int padded_len(int n) { return (n + (n >> 4) + 2) & ~1; }

// One solve instance: grid, equation, PDHG parameters and device buffers.
// All pointers are device pointers owned by the host handle.  T-typed buffers hold the
// precision of the sweep (double for plain FP64, float for the defect-correction inner solve).
struct Desc {
  int nx, ny, ncomp, lognx, logny;
  int bc, op, kind, precond;
  int dc;            // 1: the unknown is the FP32 correction d of u + d (defect correction)
  int mode;          // Mode
  int band_rows;     // rows per CTA of the band kernels (even)
  int nbands;        // ceil(ny / band_rows)
  int col_width;     // columns per CTA of the column transform (even, divides nx)
  int ncolblk;       // nx / col_width
  int meas_div_dt;   // 1: stopping measure is sum ||F_c|| / dt, else sum ||F_c||
  int stall_window;  // > 0: stop (as converged) when the measure has not halved for this many updates
  double hx2, hy2;   // 1/h_x^2, 1/h_y^2
  double dt, a, b;
  double p[6];
  double tau_u, tau_p, omega;
  void* X;           // unknown: U (plain) or d (DC)
  const void* base;  // DC: u rounded to FP32; plain: unused
  const void* rhs;   // plain: rhs of the step (FP64); DC: r = F(u) rounded to FP32
  void* P[2];        // dual variable, ping-pong by iteration parity
  void* WY;          // transform buffer: F(U) row-transformed, then G^{-1}-scaled spectrum
  const void* scale; // [ncomp][ny][nx] 1 / (g_hat nx ny) in T
  const void* twx;   // nx complex T: exp(-2 pi i k / nx)
  const void* twy;   // ny complex T
  const void* dcx;   // nx complex T: (cos, sin)(pi k / (2 nx))
  const void* dcy;   // ny complex T
  double* partials;  // [ncomp][nbands] FP64 block partial sums
};

struct State {
  int n;             // PDHG updates taken in this solve
  int status;        // StStatus
  int max_iter;
  int pad;
  double r;          // last stopping measure
  double r0;         // first stopping measure of this solve
  double thresh;     // stopping threshold on the measure
  double aux;        // begin kernel: ||U^k||_2
  double mass;       // h_x h_y sum of all components (mass kernel)
  double best;       // smallest measure at which the measure last halved (stall detection)
  int best_n;        // update count at that point
  unsigned int ticket;
};

}  // namespace rd
