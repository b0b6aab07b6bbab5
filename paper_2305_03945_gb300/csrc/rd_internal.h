// Internal types shared by the host runtime and the sm_103a kernels of the PDHG solver.
#pragma once

#include <cstddef>
#include <cstdint>

namespace rd {

enum Bc { BC_PERIODIC = 0, BC_NEUMANN = 1 };
enum Op { OP_LAP = 0, OP_BIHARM = 1, OP_FCH = 2 };
enum Kind { RX_NONE = 0, RX_AC = 1, RX_CH_IMPL = 2, RX_CH_SPLIT = 3, RX_GS = 4, RX_SCHNAK = 5, RX_FCH = 6 };
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
  int batched;       // 1: member of a batch (Slot control block, device-side phase machine)
  int fft_pp;        // bit 0 k_res, bit 1 k_col, bit 2 k_upd: transforms ping-pong between two buffers;
                     // bit 3: size-specialised unrolled transform passes (else looped passes)
  int upd_rows;      // rows per CTA of k_upd / k_updres (0: band_rows); k_res keeps band_rows
  int nupd;          // ceil(ny / upd_rows)
  int fused;         // 1: iterations after the first run k_col + k_updres (fused update and residual)
  double hx2, hy2;   // 1/h_x^2, 1/h_y^2
  double dt, a, b;
  double p[6];
  double tau_u, tau_p, omega;
  void* X;           // unknown: U (plain) or d (DC)
  const void* base;  // DC: u rounded to FP32; plain: unused
  const void* rhs;   // plain: rhs of the step (FP64); DC: r = F(u) rounded to FP32
  void* P[2];        // dual variable, ping-pong by iteration parity
  void* WY;          // transform buffer: F(U) row-transformed, then G^{-1}-scaled spectrum
  const void* scale; // unused by the sweeps (kept for layout); see mux / muy
  const void* mux;   // nx entries of T: 4/h_x^2 sin^2(pi kx / (d nx)), d = 1 periodic, 2 Neumann
  const void* muy;   // ny entries of T
  double gc1[2];     // per component: g_hat = (1 + gc1 mu + gc2 mu^2 + gc3 mu^3)^2, mu = mux + muy
  double gc2[2];
  double gc3[2];     // + gc3 mu^3 (sixth-order functionalized Cahn-Hilliard; 0 otherwise)
  double inv_nn;     // 1 / (nx ny): normalisation of the unnormalised transform pair
  const void* twx;   // nx complex T: exp(-2 pi i k / nx)
  const void* twy;   // ny complex T
  const void* dcx;   // nx complex T: (cos, sin)(pi k / (2 nx))
  const void* dcy;   // ny complex T
  double* partials;  // [ncomp][nbands] FP64 block partial sums
  // batch only (FP64 descriptor): the FP32 arrays the outer loop writes or clears
  float* f32_d;      // correction d
  float* f32_p0;     // dual P_0 of the inner solve
  float* f32_r;      // r = F(u) rounded to FP32
  float* f32_u;      // u rounded to FP32
  // fused update + residual (fused = 1): the transform buffer ping-pongs by update parity
  // (WYb[(n-1)&1] holds the spectrum of update n, k_updres writes F(U_n) into WYb[n&1]); every
  // k_updres block keeps U on its own halo rows in `halo` ([band][component][2H][nx]), written
  // and read by that block only
  void* WYb[2];
  void* halo;
  // 3-D grids (nz > 1; 0 or 1 on a 2-D grid): arrays [ncomp][nz][ny][nx], seven-point Laplacian
  // (the scheme with a third axis), transforms along x, y and z.  Every 3-D kernel runs blk3
  // blocks per instance in a grid-stride loop (fixed per instance, so that results do not depend
  // on what else shares a launch); lw3[a] lines of axis a per tile of the transform passes.
  int nz, lognz;
  double hz2;        // 1/h_z^2
  const void* muz;   // nz entries of T
  const void* twz;   // nz complex T
  const void* dcz;   // nz complex T
  int blk3;
  int lw3[3];
  int thr3[3];       // threads per block of the transform pass of each axis
  int pf3;           // 1: the long x inverse pass prefetches its P rows into shared memory
};

struct State {
  int n;             // PDHG updates taken in this solve
  int status;        // StStatus
  int max_iter;
  unsigned int trips;  // k_res launches since the solve was armed (counted by k_loop_cond)
  double r;          // last stopping measure
  double r0;         // first stopping measure of this solve
  double thresh;     // stopping threshold on the measure
  double aux;        // begin kernel: ||U^k||_2
  double mass;       // h_x h_y sum of all components (mass kernel)
  double best;       // smallest measure at which the measure last halved (stall detection)
  int best_n;        // update count at that point
  unsigned int ticket;
  int total;         // defect-correction outer state: PDHG updates of this step's inner solves
  int launches;      // defect-correction outer state: k_res launches of this step's inner solves
  int stall_mul;     // inner solve: its stall window is Desc::stall_window times this (0 = 1);
                     // the outer rule doubles it after a round that did not halve the residual
};

// Stall-window factor of the next inner solve: doubled (up to 64) after an outer round whose FP64
// residual `meas` did not halve from the previous round's `prev` (the inner solve was cut off by
// its stall rule before it made progress, as in slowly converging steps), else back to 1.
__host__ __device__ inline int next_stall_mul(int n, double meas, double prev, int mul) {
  if (mul < 1) mul = 1;
  if (n >= 1 && !(meas <= 0.5 * prev)) return mul < 64 ? 2 * mul : 64;
  return 1;
}

// Phases of one slot of a batch (device-side control of FP64 defect correction and time steps).
enum Phase {
  PH_IDLE = 0,    // empty slot
  PH_BEGIN = 1,   // new step: build rhs from U^k and the outer threshold
  PH_RESID = 2,   // FP64 residual r = F(u), stopping decision, arm the FP32 inner solve
  PH_INNER = 3,   // FP32 PDHG iterations on the correction equation
  PH_AXPY = 4,    // u += d in FP64
  PH_DONE = 5,    // all steps converged
  PH_FAILED = 6   // diverged, or the outer loop did not converge
};

// Control block of one batch slot.
struct Slot {
  State outer;            // FP64 defect-correction loop of the current step
  State inner;            // FP32 PDHG solve of the correction equation
  int phase;              // Phase
  int steps_done;
  int nsteps;
  int max_outer;          // outer rounds allowed per step
  double tol;             // stopping threshold (RD_TOL_* of tol_kind)
  double rtol;            // inner tolerance factor
  long long inner_total;  // PDHG updates over all steps
  int outer_total;        // FP64 residual passes over all steps
  int tol_kind;
};

}  // namespace rd
