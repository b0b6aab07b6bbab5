// Host-side launchers of the PDHG kernels (defined in rd_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "rd_internal.h"

namespace rd {

// Launch shape of one PDHG iteration over `ninst` instances (grid.y = instance).
struct LaunchCfg {
  int grid_bands;    // max row bands over the instances
  int grid_cols;     // max ncomp * column blocks
  int thr_res, thr_col, thr_upd;
  int smem_res, smem_col, smem_upd;
  int transform;     // 0 when G = I (no spectral solve)
  int grid_upd;      // k_upd bands (0: grid_bands)
  int thr_updres, smem_updres;  // fused update + residual kernel (k_updres)
};

// Equation keys of the sweep templates (kind_key maps a Desc to one).
enum KKey {
  KK_NONE_LAP = 0, KK_AC = 1, KK_CH_IMPL = 2, KK_CH_SPLIT = 3, KK_GS = 4, KK_SCHNAK = 5,
  KK_NONE_BIH = 6, KK_PCONLY = 7
};

// Per-key pieces of the sweep, specialised for every (T, K) in the rd_sweep_*.cu units (one unit
// per group of keys, so that the kernels compile in parallel): one iteration, a k_res launch, and
// the shared-memory limits of k_res and k_upd.
template <class T, int K>
cudaError_t launch_iter_kind(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev);
template <class T, int K>
cudaError_t launch_res(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s);
template <class T, int K>
cudaError_t allow_kind(int optin);
// The fused FP32 iteration of key K and the shared-memory limit of its k_updres (rd_fused_*.cu).
template <int K>
cudaError_t launch_fused_kind(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev,
                              bool first);
template <int K>
cudaError_t allow_fused_kind(int optin);
// The column-transform kernel k_col (pc: the preconditioner-only variant), rd_sweep_col.cu.
template <class T>
cudaError_t launch_col(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, bool pc);

// Raise the dynamic shared-memory limit of the PDHG kernels; *usable receives the bytes a launch may ask.
template <class T> cudaError_t set_kernel_smem_limits(int* usable);
// One PDHG iteration (k_res, k_col, k_upd) of the solve described by d (passed by value to the
// kernels); with ev != NULL, events ev[0..3] are recorded around the three kernels.
template <class T>
cudaError_t launch_iteration(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev);
// One PDHG iteration with the fused update (d.fused = 1, FP32 only): k_res (first only), k_col,
// k_updres; events ev[0..3] around them as in launch_iteration.
template <class T>
cudaError_t launch_fused(const Desc& d, State* st, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev, bool first);


// The step-level kernels (begin, FP64 residual, mass) run point_blocks(nx, ny) blocks of 256
// threads, two points per thread; d.partials must hold ncomp * point_blocks(nx, ny) doubles.
inline int point_blocks(int nx, int ny) { return (int)(((size_t)nx * ny / 2 + 255) / 256); }

cudaError_t launch_begin(const Desc* d64, State* st, const double* uk, double* rhs, double tol, int tol_kind,
                         int nblocks, cudaStream_t s);
cudaError_t launch_resid64(const Desc& hd, const Desc* d64, State* outer, State* inner, const double* u,
                           const double* rhs, double* w64, float* r32, float* u32, float* z0, float* z1, int decide,
                           double rtol, int max_outer, int nblocks, cudaStream_t s);

// Work arrays of the sixth-order functionalized Cahn-Hilliard iteration (rd_fch.cu): P~, mu(U),
// A(U) mu / A(U) Lap P~, Lap P~; each ny * nx doubles.
struct FchBuffers {
  double* Pt;
  double* M;
  double* N;
  double* Q;
};
// W = F(U) of that equation (st != NULL: also the stopping decision of the solve st, on at most
// max_blocks blocks of d.partials).
cudaError_t launch_fch_residual(const Desc& d, State* st, const FchBuffers& b, const double* U, const double* Uk,
                                double* W, int max_blocks, cudaStream_t s);
// One PDHG iteration of that equation on d (X = U, rhs = U^k, P[0] = P); dpc is the
// preconditioner-only descriptor whose X holds W (and then G^{-1} W), run on st_pc with cpc.
// Events ev[0..3] (may be NULL) around the residual, the preconditioner solve and the update.
cudaError_t launch_fch_iteration(const Desc& d, const Desc& dpc, State* st, State* st_pc, const LaunchCfg& cpc,
                                 const FchBuffers& b, int max_blocks, cudaStream_t s, cudaEvent_t* ev);

// Set the thread-local detail string returned by rd_last_error().
void set_last_error(const char* msg);

// Device-side loop decision (one thread): adds `sweeps` to st->trips and clears the graph
// conditional `cond` when the solve has ended (or the launch bound is passed).
cudaError_t launch_loop_cond(State* st, unsigned long long cond, unsigned sweeps, cudaStream_t s);
cudaError_t launch_axpy_dc(double* u, const float* dlt, size_t n, State* outer, const State* inner, cudaStream_t s);
cudaError_t launch_mass(const Desc* d64, State* st, const double* u, const State* gate, int nblocks, cudaStream_t s);

}  // namespace rd
