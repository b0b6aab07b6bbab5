// C ABI of the GB300 PDHG solver: handle lifecycle, workspace and table set-up, CUDA-graph
// capture of the PDHG iteration, and the step / solve drivers (Algorithm 1 of arxiv 2305.03945).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rd_pdhg.h"
#include "rd_device.cuh"
#include "rd_launch.h"
#include "rd_launch3.h"
#include "rd_launch_small.h"

using namespace rd;

namespace {

thread_local std::string g_last_error;

rd_status fail(rd_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define RD_CUDA(expr)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA,                  \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                         \
    }                                                                                          \
  } while (0)

constexpr int kSmemLimit = 226 * 1024;  // planning limit; checked against the device at create
constexpr int kTargetBlocks = 152;  // one wave on a GB300
// The FP32 inner solve of defect correction stops, as converged, once its residual has not
// halved over this many updates: it has reached the FP32 rounding floor of the correction
// equation and the FP64 outer loop takes over.
constexpr int kDcStallWindow = 8;  // default of rd_opts.dc_stall_window

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }
int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <class T>
int band_threads(int nlines, int nx) {
  const int r = FftRadix<T>::value;
  int t = (int)(((long long)nlines * nx + r - 1) / r);
  const int line = fft_line_threads<T>(nx);
  if (t < line) t = line;
  t = round_up(t, 32);
  if (t < 64) t = 64;
  if (t > MaxThreads<T>::value) t = MaxThreads<T>::value;
  return t;
}

// Resident blocks per SM of a sweep kernel with `threads` threads and `smem` bytes of dynamic
// shared memory: registers per thread as fixed by the kernels' launch bounds, 64 K registers,
// 2048 threads, 228 KB of shared memory (1 KB reserved per block) and 32 blocks per SM.
template <class T>
int blocks_per_sm(int threads, int smem) {
  const int regs = std::min(255, (65536 / (MaxThreads<T>::value * MinBlocks<T>::value)) & ~7);
  const int warps = (threads + 31) / 32;
  const int by_regs = 65536 / (warps * ((regs * 32 + 255) / 256 * 256));
  const int by_thr = 2048 / (warps * 32);
  const int by_smem = (228 * 1024) / (smem + 1024);
  return std::max(0, std::min(std::min(by_regs, by_thr), std::min(by_smem, 32)));
}

// Transforms ping-pong between two buffers (one barrier per pass instead of two) when the
// second buffer fits and costs no resident blocks.
// fft_buffers: 0 = that rule, 1 = never, 2 = whenever the second buffer fits.
template <class T>
bool use_pingpong(int fft_buffers, int threads, int smem_inplace, int smem_pp) {
  if (fft_buffers == 1 || smem_pp > kSmemLimit) return false;
  return fft_buffers == 2 || blocks_per_sm<T>(threads, smem_pp) >= blocks_per_sm<T>(threads, smem_inplace);
}

// Launch shape for one precision.  Returns false when the grid does not fit.
template <class T>
// stage_base: the residual kernel stages the defect-correction base rows (Cahn-Hilliard in FP32).
// band_req: rows per CTA of k_res (0: planner); upd_req: rows per CTA of k_upd (0: as k_res).
bool plan_launch(int nx, int ny, int nc, int H, int transform, int neumann, int band_req, int col_req, int upd_req,
                 int stage_base, int fft_buffers, int fft_unrolled, Desc& d, LaunchCfg& c, std::string& why) {
  const int tabx = table_bytes<T>(nx, transform != 0, transform && neumann);  // k_res, k_upd
  const int taby = table_bytes<T>(ny, true, neumann != 0);                    // k_col
  if (fft_line_threads<T>(nx) > MaxThreads<T>::value || fft_line_threads<T>(ny) > MaxThreads<T>::value) {
    why = "grid side too long for this precision";
    return false;
  }
  int B = 0;
  if (band_req > 0) {
    B = band_req;
    if (B % 2 || B > ny) {
      why = "band_rows must be even and <= ny";
      return false;
    }
  } else {
    for (int cand = 16; cand >= 2; cand /= 2) {
      if (cand > ny) continue;
      const int nb = (ny + cand - 1) / cand;
      const int sm =
          std::max(lines_smem_bytes<T>(nc * ((cand + 2 * H) / 2), nx, 0, tabx), res_smem_bytes<T>(nc, cand, H, nx, stage_base, 0, tabx));
      if (sm > kSmemLimit) continue;
      if (nb >= kTargetBlocks || cand == 2) {
        B = cand;
        break;
      }
    }
    if (B == 0) B = 2;
  }
  const int U = upd_req > 0 ? upd_req : B;  // k_upd band rows
  if (U % 2 || U > ny) {
    why = "k_upd band rows must be even and <= ny";
    return false;
  }
  int smem_res = res_smem_bytes<T>(nc, B, H, nx, stage_base, 0, tabx);
  int smem_upd = lines_smem_bytes<T>(nc * ((U + 2 * H) / 2), nx, 0, tabx);
  if (smem_upd > kSmemLimit || smem_res > kSmemLimit) {
    why = "row band does not fit in shared memory";
    return false;
  }
  int C = 0;
  const int cmin = std::max(2, std::min(nx, 16 / (int)sizeof(T)));
  if (col_req > 0) {
    C = col_req;
    if (C % 2 || C > nx || nx % C) {
      why = "col_width must be even and divide nx";
      return false;
    }
  } else {
    C = cmin;
    for (int cand = cmin * 2; cand <= nx; cand *= 2) {
      if (nc * (nx / cand) < 2 * kTargetBlocks) break;
      if (lines_smem_bytes<T>(cand / 2, ny, 0, taby) > kSmemLimit / 2) break;

      C = cand;
    }
  }
  int smem_col = lines_smem_bytes<T>(C / 2, ny, 0, taby);
  if (smem_col > kSmemLimit) {
    why = "column block does not fit in shared memory";
    return false;
  }
  d.band_rows = B;
  d.nbands = (ny + B - 1) / B;
  d.col_width = C;
  d.ncolblk = nx / C;
  d.upd_rows = U;
  d.nupd = (ny + U - 1) / U;
  c.grid_bands = d.nbands;
  c.grid_upd = d.nupd;
  c.grid_cols = nc * d.ncolblk;
  c.thr_res = band_threads<T>(nc * (B / 2), nx);
  c.thr_upd = band_threads<T>(nc * ((U + 2 * H) / 2), nx);
  c.thr_col = band_threads<T>(C / 2, ny);
  d.fft_pp = 0;
  if (use_pingpong<T>(fft_buffers, c.thr_res, smem_res, res_smem_bytes<T>(nc, B, H, nx, stage_base, 1, tabx))) {
    d.fft_pp |= 1;
    smem_res = res_smem_bytes<T>(nc, B, H, nx, stage_base, 1, tabx);
  }
  if (use_pingpong<T>(fft_buffers, c.thr_col, smem_col, lines_smem_bytes<T>(C / 2, ny, 1, taby))) {
    d.fft_pp |= 2;
    smem_col = lines_smem_bytes<T>(C / 2, ny, 1, taby);
  }
  if (use_pingpong<T>(fft_buffers, c.thr_upd, smem_upd, lines_smem_bytes<T>(nc * ((U + 2 * H) / 2), nx, 1, tabx))) {
    d.fft_pp |= 4;
    smem_upd = lines_smem_bytes<T>(nc * ((U + 2 * H) / 2), nx, 1, tabx);
  }
  if (fft_unrolled) d.fft_pp |= 8;
  c.smem_res = smem_res;
  c.smem_upd = smem_upd;
  c.smem_col = smem_col;
  c.transform = transform;
  return true;
}

}  // namespace

void rd::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

struct rd_pdhg {
  int nx = 0, ny = 0, nc = 1;
  int nz = 1;       // 3-D grids: points along z (1 on a 2-D grid)
  int nd3 = 0;      // 1: a 3-D grid (the rd_3d.cu kernels)
  int small = 0;    // every FP32 inner solve in one launch (rd_small.cu): 1 one block, 2 a cluster
  double hz = 0;
  size_t npts = 0;  // nc * nx * ny * nz
  int bc = 0, op = 0, kind = 0, precond = 1;
  double pc_shift = 0;  // RD_PC_STABILIZED: the constant in place of the nonlinear factor
  double dt = 0, tau = 0, sigma = 0, hx = 0, hy = 0;
  rd_reaction rx{};
  rd_opts opts{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t body_stream = nullptr;  // captures the body of the device-side loop
  cudaStream_t body_stream2 = nullptr; // captures a loop body nested in another (inner solves in the outer rounds)
  int dc = 0;
  // FP64 state and plain-path workspaces
  double* U64 = nullptr;
  double* rhs64 = nullptr;
  double* P64[2] = {nullptr, nullptr};
  double* WY64 = nullptr;
  double* mu64[2] = {nullptr, nullptr};  // mu_x, mu_y
  cx<double>* tw64[4] = {nullptr, nullptr, nullptr, nullptr};  // twx, twy, dcx, dcy
  double* mu64z = nullptr;                                     // 3-D: mu_z, twz, dcz
  cx<double>* tw64z[2] = {nullptr, nullptr};
  float* mu32z = nullptr;
  cx<float>* tw32z[2] = {nullptr, nullptr};
  // FP32 defect-correction workspaces
  float* D32 = nullptr;
  float* P32[2] = {nullptr, nullptr};
  float* WY32 = nullptr;
  float* WY32b = nullptr;   // fused update: second transform buffer
  float* halo32 = nullptr;  // fused update: per-band copies of U on the halo rows
  size_t halo_bytes = 0;
  float* mu32[2] = {nullptr, nullptr};
  float* r32 = nullptr;
  float* u32 = nullptr;
  cx<float>* tw32[4] = {nullptr, nullptr, nullptr, nullptr};
  double* partials = nullptr;
  // sixth-order functionalized Cahn-Hilliard (FP64 only): its own stencil passes (rd_fch.cu)
  int fch = 0;
  FchBuffers fchb{};
  Desc* d_desc = nullptr;   // [0] FP64 plain / outer, [1] FP32 inner, [2] FP64 precond-only
  State* d_state = nullptr; // [0] plain / outer, [1] inner, [2] misc
  State* h_state = nullptr; // pinned mirror
  Desc h_desc[3]{};
  LaunchCfg cfg64{}, cfg32{}, cfgpc{};
  // Step graphs.  FP64: [0] the whole step.  Defect correction: [0] the first outer round of a
  // step (with the step set-up), [1] every later round.
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // RD_LOOP_HOST: graph_k PDHG iterations without conditional nodes, relaunched by the host
  cudaGraph_t hgraph = nullptr;
  cudaGraphExec_t hexec = nullptr;
  cudaGraph_t hgraph1 = nullptr;      // fused update: the first launch of an inner solve
  cudaGraphExec_t hexec1 = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // around the first iteration's kernels
  int kernels_per_iter = 0;
  rd_stats stats{};
  std::vector<void*> allocs;
};

namespace {

template <class P>
rd_status dalloc(rd_pdhg* h, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RD_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  h->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return RD_OK;
}

#define RD_TRY(expr)               \
  do {                             \
    rd_status s_ = (expr);         \
    if (s_ != RD_OK) return s_;    \
  } while (0)

// twiddle tables exp(-2 pi i k / n) and (cos, sin)(pi k / (2n)), evaluated in long double
void host_twiddles(int n, std::vector<double>& tw, std::vector<double>& dc) {
  const long double pi = 3.141592653589793238462643383279502884L;
  tw.resize(2 * n);
  dc.resize(2 * n);
  for (int k = 0; k < n; ++k) {
    const long double t = 2.0L * pi * (long double)k / (long double)n;
    tw[2 * k] = (double)cosl(t);
    tw[2 * k + 1] = (double)(-sinl(t));
    const long double q = pi * (long double)k / (2.0L * (long double)n);
    dc[2 * k] = (double)cosl(q);
    dc[2 * k + 1] = (double)sinl(q);
  }
}

// Eigenvalues of -Lap along each axis, mu(k) = 4/h^2 sin^2(pi k / (d n)) (d = 1 periodic,
// 2 Neumann), evaluated in long double; the preconditioner symbol is
// g_hat(kx, ky) = (1 + gc1 mu + gc2 mu^2)^2 with mu = mu_x(kx) + mu_y(ky).
void host_mu(const rd_pdhg* h, std::vector<double>& mx, std::vector<double>& my) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double dd = h->bc == RD_BC_PERIODIC ? 1.0L : 2.0L;
  mx.resize(h->nx);
  my.resize(h->ny);
  for (int k = 0; k < h->nx; ++k) {
    const long double sn = sinl(pi * k / (dd * h->nx));
    mx[k] = (double)(4.0L / ((long double)h->hx * h->hx) * sn * sn);
  }
  for (int k = 0; k < h->ny; ++k) {
    const long double sn = sinl(pi * k / (dd * h->ny));
    my[k] = (double)(4.0L / ((long double)h->hy * h->hy) * sn * sn);
  }
}

// mu_z(k) of a 3-D grid, the same formula along z
void host_mu_z(const rd_pdhg* h, std::vector<double>& mz) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double dd = h->bc == RD_BC_PERIODIC ? 1.0L : 2.0L;
  mz.resize(h->nz);
  for (int k = 0; k < h->nz; ++k) {
    const long double sn = sinl(pi * k / (dd * h->nz));
    mz[k] = (double)(4.0L / ((long double)h->hz * h->hz) * sn * sn);
  }
}

// RD_PC_STABILIZED (scalar reactions): the Jacobian of F with its nonlinear factor replaced by
// the constant s (Section 3.3's construction of G), squared:
//   Allen-Cahn      (1 + b dt s) + a dt mu      = c0 (1 + (a dt / c0) mu): gc1 = a dt / c0 and
//                   the constant c0^2 folded into the normalisation inv_nn
//   Cahn-Hilliard   1 + b s dt mu + a dt mu^2   (s in place of W''(U), or of 3 U^2 for the split)
//   sixth order     1 + dt a (s b - a) mu^2 + dt a^2 mu^3 (RD_PC_LINEAR: s = 2)
void symbol_coefficients(const rd_pdhg* h, Desc& d) {
  const bool stab = h->precond == RD_PC_STABILIZED;
  const double s = h->pc_shift;
  double c0 = 1.0;
  for (int c = 0; c < 2; ++c) {
    double D = h->rx.a;
    if (h->kind == RD_RX_GRAY_SCOTT || h->kind == RD_RX_SCHNAKENBERG) D = h->rx.p[c < h->nc ? c : 0];
    d.gc3[c] = 0.0;
    if (h->op == RD_OP_LAPLACIAN) {
      if (stab) c0 = 1.0 + h->rx.b * h->dt * s;
      d.gc1[c] = D * h->dt / c0;
      d.gc2[c] = 0.0;
    } else if (h->op == RD_OP_FUNCTIONALIZED) {
      // G = (I - dt Lap (a Lap - (2b - a) I) a Lap)^2: 1 + dt a (2b - a) mu^2 + dt a^2 mu^3
      d.gc1[c] = 0.0;
      d.gc2[c] = h->dt * h->rx.a * ((stab ? s : 2.0) * h->rx.b - h->rx.a);
      d.gc3[c] = h->dt * h->rx.a * h->rx.a;
    } else {
      d.gc1[c] = stab ? h->rx.b * s * h->dt : 0.0;
      d.gc2[c] = h->rx.a * h->dt;
    }
  }
  d.inv_nn = 1.0 / ((double)h->nx * (double)h->ny * (double)h->nz * c0 * c0);
}

rd_status status_of(int st) {
  switch (st) {
    case ST_CONVERGED: return RD_OK;
    case ST_NOT_CONVERGED: return RD_ERR_NOT_CONVERGED;
    case ST_DIVERGED: return RD_ERR_DIVERGED;
    default: return RD_ERR_NOT_CONVERGED;
  }
}

// One PDHG iteration of the sixth-order equation (FP64): its stencil passes around the
// preconditioner-only transform kernels, which read and write P64[1] (h_desc[2].X).
cudaError_t fch_iteration(rd_pdhg* h, cudaStream_t s, cudaEvent_t* ev) {
  const int cap = 2 * std::max(std::max(h->h_desc[0].nbands, h->ny / 2 + 1), point_blocks(h->nx, h->ny));
  return launch_fch_iteration(h->h_desc[0], h->h_desc[2], h->d_state + 0, h->d_state + 2, h->cfgpc, h->fchb, cap, s, ev);
}

// Capture one step graph.  Layout (FP64 plain, first = true):
//   k_begin, P_0 = 0, iteration 1, k_loop_cond, WHILE { graph_k iterations, k_loop_cond }, k_mass
// and for defect correction, with ROUND = the inner solve (iteration 1, k_loop_cond and the
// WHILE node above; or one small-solve launch), k_axpy_dc, k_resid64:
//   first = true : k_begin, k_resid64, ROUND, k_loop_cond(outer), WHILE { ROUND, k_loop_cond(outer) }, k_mass
//   first = false: ROUND, k_mass   (one host-driven round, the fallback beyond the loop's bound)
// Iteration 1 and the first outer round sit outside the loops so that the profiling events
// (which a conditional body cannot hold) bracket the first iteration's kernels.  k_loop_cond,
// run after iteration 1 (the first outer round) and at the end of every trip, sets its loop's
// condition: 1 while the solve (the outer state) is active, 0 once it has ended or after
// max_iter + slack launches.  k_axpy_dc,
// k_resid64 and k_mass act only while (resp. once no longer) the outer state is active.
// Step-level launches of either grid kind: the step set-up and the FP64 residual.
cudaError_t begin_any(rd_pdhg* h, State* st, const double* uk, double tol, int tol_kind, int nb, cudaStream_t s) {
  if (h->nd3) return launch_begin3(h->h_desc[0], h->d_desc + 0, st, uk, h->rhs64, tol, tol_kind, s);
  return launch_begin(h->d_desc + 0, st, uk, h->rhs64, tol, tol_kind, nb, s);
}

cudaError_t resid64_any(rd_pdhg* h, State* outer, State* inner, const double* u, double* w64, float* r32, float* u32,
                        float* z0, float* z1, int decide, int nb, cudaStream_t s) {
  if (h->nd3)
    return launch_resid64_3(h->h_desc[0], h->d_desc + 0, outer, inner, u, h->rhs64, w64, r32, u32, z0, z1, decide,
                            h->opts.dc_inner_rtol, h->opts.dc_max_outer, s);
  return launch_resid64(h->h_desc[0], h->d_desc + 0, outer, inner, u, h->rhs64, w64, r32, u32, z0, z1, decide,
                        h->opts.dc_inner_rtol, h->opts.dc_max_outer, nb, s);
}

// The one-block inner solve with the profiling events around it (ev[0..3]; the time lands in
// kernel_ms[0]).
cudaError_t small_launch(rd_pdhg* h, cudaStream_t s, cudaEvent_t* ev) {
  unsigned flags = cudaEventRecordDefault;
  if (ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive) flags = cudaEventRecordExternal;
  }
  cudaError_t e = ev ? cudaEventRecordWithFlags(ev[0], s, flags) : cudaSuccess;
  if (e == cudaSuccess) e = launch_small(h->h_desc[1], h->d_state + 1, h->small, s);
  for (int i = 1; i < 4 && ev && e == cudaSuccess; ++i) e = cudaEventRecordWithFlags(ev[i], s, flags);
  return e;
}

// Blocks of the step-level kernels (k_begin, k_resid64, k_mass: two points per thread).
int step_blocks(const rd_pdhg* h) { return point_blocks(h->nx, h->ny * h->nz); }

rd_status capture_step_graph(rd_pdhg* h, bool first, cudaGraph_t* out, cudaGraphExec_t* exec) {
  const int K = h->opts.graph_k;
  cudaStream_t cs = h->cap_stream;
  const int nb = step_blocks(h);
  const Desc* d64 = h->d_desc + 0;
  State* st0 = h->d_state + 0;
  State* st1 = h->d_state + 1;
  State* sti = h->dc ? st1 : st0;
  cudaGraph_t g = nullptr;
  RD_CUDA(cudaGraphCreate(&g, 0));
  *out = g;
  // defect correction: the first graph holds the whole step, the outer rounds after the first in
  // a WHILE node on the outer state (each round: the inner solve -- one launch, or iteration 1
  // and a WHILE node over the rest -- then u += d, the FP64 residual and decision, the loop
  // condition); the second graph, one host-driven round, is the fallback should the device loop
  // reach its bound
  const bool outer_loop = h->dc && first;
  cudaGraphConditionalHandle cond = 0, cond_o = 0;
  if (!h->small) RD_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  if (outer_loop) RD_CUDA(cudaGraphConditionalHandleCreate(&cond_o, g, 1, cudaGraphCondAssignDefault));
  const Desc dd = h->dc ? h->h_desc[1] : h->h_desc[0];
  auto iteration = [&](cudaStream_t st, cudaEvent_t* ev, bool first_it) {
    if (h->small) return small_launch(h, st, ev);
    if (h->fch) return fch_iteration(h, st, ev);
    if (h->nd3) return h->dc ? launch_iteration3<float>(dd, sti, st, ev) : launch_iteration3<double>(dd, sti, st, ev);
    if (h->dc && dd.fused) return launch_fused<float>(dd, sti, h->cfg32, st, ev, first_it);
    return h->dc ? launch_iteration<float>(dd, sti, h->cfg32, st, ev) : launch_iteration<double>(dd, sti, h->cfg64, st, ev);
  };
  auto abort_capture = [&](cudaStream_t st, const char* what, cudaError_t e) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(st, &tmp);
    if (tmp && tmp != g) cudaGraphDestroy(tmp);
    return fail(RD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  // appends a WHILE node on handle `c` to the capture in stream `st` and captures body(bs) into
  // its body graph; make_handle(body graph) may create handles on that graph first
  auto while_node = [&](cudaStream_t st, cudaGraphConditionalHandle c, cudaStream_t bs, auto make_handle,
                        auto body) -> cudaError_t {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t r = cudaStreamGetCaptureInfo(st, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    if (r != cudaSuccess) return r;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = c;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    if ((r = cudaGraphAddNode(&wn, cg, deps, nullptr, ndeps, &cp)) != cudaSuccess) return r;
    if ((r = cudaStreamUpdateCaptureDependencies(st, &wn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
      return r;
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    if ((r = make_handle(bg)) != cudaSuccess) return r;
    if ((r = cudaStreamBeginCaptureToGraph(bs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return r;
    r = body(bs);
    cudaGraph_t body_out = nullptr;
    const cudaError_t r2 = cudaStreamEndCapture(bs, &body_out);
    return r != cudaSuccess ? r : r2;
  };
  auto no_handle = [](cudaGraph_t) { return cudaSuccess; };
  // one inner solve on stream st: iteration 1 (with the profiling events when ev), then the
  // WHILE node on handle c (body captured on stream bs) over graph_k iterations per trip
  auto inner_solve = [&](cudaStream_t st, cudaEvent_t* ev, cudaGraphConditionalHandle c, cudaStream_t bs) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    // fused update: the per-band halo copies of U start at U_0 = d = 0
    if (dd.fused) r = cudaMemsetAsync(h->halo32, 0, h->halo_bytes, st);
    if (r == cudaSuccess) r = iteration(st, ev, true);
    if (h->small || r != cudaSuccess) return r;
    if ((r = launch_loop_cond(sti, c, 1u, st)) != cudaSuccess) return r;
    return while_node(st, c, bs, no_handle, [&](cudaStream_t b) {
      cudaError_t q = cudaSuccess;
      for (int k = 0; k < K && q == cudaSuccess; ++k) q = iteration(b, nullptr, false);
      if (q == cudaSuccess) q = launch_loop_cond(sti, c, (unsigned)K, b);
      return q;
    });
  };
  // one outer round after the FP64 residual that armed it
  auto round = [&](cudaStream_t st, cudaEvent_t* ev, cudaGraphConditionalHandle c, cudaStream_t bs) -> cudaError_t {
    cudaError_t r = inner_solve(st, ev, c, bs);
    if (r == cudaSuccess) r = launch_axpy_dc(h->U64, h->D32, h->npts, st0, st1, st);
    if (r == cudaSuccess) r = resid64_any(h, st0, st1, h->U64, nullptr, h->r32, h->u32, h->D32, h->P32[0], 1, nb, st);
    return r;
  };
  RD_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (first) {
    e = begin_any(h, st0, h->U64, h->opts.tol, h->opts.tol_kind, nb, cs);
    if (e == cudaSuccess && !h->dc) e = cudaMemsetAsync(h->P64[0], 0, h->npts * sizeof(double), cs);
    if (e == cudaSuccess && h->dc) e = resid64_any(h, st0, st1, h->U64, nullptr, h->r32, h->u32, h->D32, h->P32[0], 1, nb, cs);
    if (e != cudaSuccess) return abort_capture(cs, "step set-up during capture", e);
  }
  cudaEvent_t* ev1 = h->opts.profile ? h->ev : nullptr;
  if (!h->dc) {
    // FP64: the PDHG loop of the step
    if ((e = inner_solve(cs, ev1, cond, h->body_stream)) != cudaSuccess)
      return abort_capture(cs, "the PDHG loop", e);
  } else if (outer_loop) {
    // the first outer round outside the outer loop (the profiling events cannot sit in a conditional body)
    e = round(cs, ev1, cond, h->body_stream);
    if (e == cudaSuccess) e = launch_loop_cond(st0, cond_o, 1u, cs);
    if (e != cudaSuccess) return abort_capture(cs, "the first outer round", e);
    cudaGraphConditionalHandle cond_i = 0;
    e = while_node(
        cs, cond_o, h->body_stream,
        [&](cudaGraph_t bg) {
          return h->small ? cudaSuccess : cudaGraphConditionalHandleCreate(&cond_i, bg, 1, cudaGraphCondAssignDefault);
        },
        [&](cudaStream_t b) {
          cudaError_t q = round(b, nullptr, cond_i, h->body_stream2);
          if (q == cudaSuccess) q = launch_loop_cond(st0, cond_o, 1u, b);
          return q;
        });
    if (e != cudaSuccess) return abort_capture(cs, "the outer-round loop", e);
  } else {
    if ((e = round(cs, ev1, cond, h->body_stream)) != cudaSuccess)
      return abort_capture(cs, "the outer round", e);
  }
  if (h->dc) {
    e = launch_mass(d64, h->d_state + 2, h->U64, st0, nb, cs);
  } else {
    e = launch_mass(d64, h->d_state + 2, h->U64, nullptr, nb, cs);
  }
  if (e != cudaSuccess) return abort_capture(cs, "kernel launch during capture", e);
  cudaGraph_t g_out = nullptr;
  RD_CUDA(cudaStreamEndCapture(cs, &g_out));
  RD_CUDA(cudaGraphInstantiate(exec, g, 0));
  return RD_OK;
}

// RD_LOOP_HOST: one graph of graph_k PDHG iterations (profiling events around the first).  With
// the fused update a second graph starts each inner solve: it clears the halo copies and its
// first iteration launches k_res; the profiling events sit in that graph only.
rd_status capture_iter_graph(rd_pdhg* h, bool start, cudaGraph_t* graph, cudaGraphExec_t* exec) {
  const int K = h->opts.graph_k;
  const Desc& dd = h->dc ? h->h_desc[1] : h->h_desc[0];
  const bool fused = h->dc && dd.fused;
  cudaStream_t cs = h->cap_stream;
  RD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (fused && start) e = cudaMemsetAsync(h->halo32, 0, h->halo_bytes, cs);
  for (int k = 0; k < (h->small ? 1 : K) && e == cudaSuccess; ++k) {
    cudaEvent_t* ev = (k == 0 && h->opts.profile && (start || !fused)) ? h->ev : nullptr;
    if (h->small) e = small_launch(h, cs, ev);
    else if (h->fch) e = fch_iteration(h, cs, ev);
    else if (h->nd3) e = h->dc ? launch_iteration3<float>(dd, h->d_state + 1, cs, ev)
                               : launch_iteration3<double>(dd, h->d_state + 0, cs, ev);
    else if (fused) e = launch_fused<float>(dd, h->d_state + 1, h->cfg32, cs, ev, start && k == 0);
    else if (h->dc) e = launch_iteration<float>(dd, h->d_state + 1, h->cfg32, cs, ev);
    else e = launch_iteration<double>(dd, h->d_state + 0, h->cfg64, cs, ev);
  }
  if (e != cudaSuccess) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    return fail(RD_ERR_CUDA, std::string("kernel launch during capture: ") + cudaGetErrorString(e));
  }
  RD_CUDA(cudaStreamEndCapture(cs, graph));
  RD_CUDA(cudaGraphInstantiate(exec, *graph, 0));
  return RD_OK;
}

rd_status capture_graphs(rd_pdhg* h) {
  const LaunchCfg& lc = h->dc ? h->cfg32 : h->cfg64;
  h->kernels_per_iter = h->small ? 1
                    : h->fch ? (lc.transform ? 10 : 7)
                    : h->nd3 ? (lc.transform ? (h->nz > 1 ? 7 : 5) : 2)
                             : (h->dc && h->h_desc[1].fused ? 2 : (lc.transform ? 3 : 2));
  if (h->opts.profile)
    for (int i = 0; i < 4; ++i)
      if (!h->ev[i]) RD_CUDA(cudaEventCreate(&h->ev[i]));
  if (h->opts.solve_loop == RD_LOOP_HOST) {
    RD_TRY(capture_iter_graph(h, false, &h->hgraph, &h->hexec));
    if (h->dc && h->h_desc[1].fused) RD_TRY(capture_iter_graph(h, true, &h->hgraph1, &h->hexec1));
    return RD_OK;
  }
  RD_TRY(capture_step_graph(h, true, &h->graph[0], &h->gexec[0]));
  if (h->dc) RD_TRY(capture_step_graph(h, false, &h->graph[1], &h->gexec[1]));
  return RD_OK;
}

void destroy_graphs(rd_pdhg* h) {
  for (int k = 0; k < 2; ++k) {
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    if (h->graph[k]) cudaGraphDestroy(h->graph[k]);
    h->gexec[k] = nullptr;
    h->graph[k] = nullptr;
  }
  if (h->hexec) cudaGraphExecDestroy(h->hexec);
  if (h->hgraph) cudaGraphDestroy(h->hgraph);
  if (h->hexec1) cudaGraphExecDestroy(h->hexec1);
  if (h->hgraph1) cudaGraphDestroy(h->hgraph1);
  h->hexec = h->hexec1 = nullptr;
  h->hgraph = h->hgraph1 = nullptr;
}

// A new time step h_t: the descriptors' dt and preconditioner symbol coefficients (everything
// else that depends on h_t is formed from them in the kernels), then the graphs, which hold the
// descriptors by value, are captured again.
rd_status set_dt_impl(rd_pdhg* h, double dt) {
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(RD_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (dt == h->dt) return RD_OK;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  h->dt = dt;
  for (int i = 0; i < 3; ++i) {
    h->h_desc[i].dt = dt;
    symbol_coefficients(h, h->h_desc[i]);
  }
  RD_CUDA(cudaMemcpy(h->d_desc, h->h_desc, 3 * sizeof(Desc), cudaMemcpyHostToDevice));
  destroy_graphs(h);
  return capture_graphs(h);
}

rd_status validate(const rd_grid* grid, rd_bc bc, rd_operator op, const rd_reaction* rx, double dt, double tau,
                   double sigma, const rd_precond* pc, const rd_opts* o) {
  if (!grid || !rx) return fail(RD_ERR_INVALID_ARG, "grid and reaction must not be NULL");
  if (grid->ndim != 2 && grid->ndim != 3) return fail(RD_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (grid->ndim == 3) {
    if (rx->kind != RD_RX_NONE && rx->kind != RD_RX_ALLEN_CAHN && rx->kind != RD_RX_CH_IMPLICIT &&
        rx->kind != RD_RX_CH_SPLIT)
      return fail(RD_ERR_UNSUPPORTED, "3-D grids are built for the scalar kinds (none, Allen-Cahn, Cahn-Hilliard)");
  }
  for (int k = 0; k < grid->ndim; ++k) {
    if (grid->n[k] < 2) return fail(RD_ERR_INVALID_ARG, "grid sides need n >= 2");
    if (!pow2(grid->n[k])) return fail(RD_ERR_UNSUPPORTED, "grid sides must be powers of two");
    if (!(grid->length[k] > 0) || !std::isfinite(grid->length[k])) return fail(RD_ERR_INVALID_ARG, "lengths must be > 0");
  }
  if (bc != RD_BC_PERIODIC && bc != RD_BC_NEUMANN) return fail(RD_ERR_INVALID_ARG, "bad boundary condition");
  if (op != RD_OP_LAPLACIAN && op != RD_OP_NEG_BIHARMONIC && op != RD_OP_FUNCTIONALIZED)
    return fail(RD_ERR_INVALID_ARG, "bad operator");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(RD_ERR_INVALID_ARG, "dt must be > 0");
  if (!(tau > 0) || !(sigma > 0) || !std::isfinite(tau) || !std::isfinite(sigma))
    return fail(RD_ERR_INVALID_ARG, "tau and sigma must be > 0");
  if (rx->kind < RD_RX_NONE || rx->kind > RD_RX_FCH) return fail(RD_ERR_INVALID_ARG, "bad reaction kind");
  if ((rx->kind == RD_RX_FCH) != (op == RD_OP_FUNCTIONALIZED))
    return fail(RD_ERR_INVALID_ARG, "RD_RX_FCH goes with RD_OP_FUNCTIONALIZED and only with it");
  if (rx->kind == RD_RX_FCH && o && o->precision != RD_PREC_FP64)
    return fail(RD_ERR_UNSUPPORTED, "the sixth-order equation is built for RD_PREC_FP64 only");
  const bool two = rx->kind == RD_RX_GRAY_SCOTT || rx->kind == RD_RX_SCHNAKENBERG;
  if (rx->ncomp != (two ? 2 : 1)) return fail(RD_ERR_INVALID_ARG, "ncomp does not match the reaction kind");
  if (!(rx->a >= 0) || !(rx->b >= 0)) return fail(RD_ERR_INVALID_ARG, "a and b must be >= 0");
  if ((rx->kind == RD_RX_ALLEN_CAHN || two) && op != RD_OP_LAPLACIAN)
    return fail(RD_ERR_INVALID_ARG, "this reaction needs RD_OP_LAPLACIAN");
  if ((rx->kind == RD_RX_CH_IMPLICIT || rx->kind == RD_RX_CH_SPLIT) && op != RD_OP_NEG_BIHARMONIC)
    return fail(RD_ERR_INVALID_ARG, "Cahn-Hilliard needs RD_OP_NEG_BIHARMONIC");
  if (two && (!(rx->p[0] >= 0) || !(rx->p[1] >= 0))) return fail(RD_ERR_INVALID_ARG, "diffusivities must be >= 0");
  if (pc && pc->kind != RD_PC_NONE && pc->kind != RD_PC_LINEAR && pc->kind != RD_PC_STABILIZED)
    return fail(RD_ERR_INVALID_ARG, "bad preconditioner kind");
  if (pc && pc->kind == RD_PC_STABILIZED) {
    if (rx->kind != RD_RX_ALLEN_CAHN && rx->kind != RD_RX_CH_IMPLICIT && rx->kind != RD_RX_CH_SPLIT &&
        rx->kind != RD_RX_FCH)
      return fail(RD_ERR_UNSUPPORTED, "the stabilized preconditioner is built for the scalar reactions");
    if (!(pc->s >= 0) || !std::isfinite(pc->s)) return fail(RD_ERR_INVALID_ARG, "stabilized shift s must be >= 0");
  } else if (pc && pc->s != 0.0) {
    return fail(RD_ERR_INVALID_ARG, "the shift s belongs to RD_PC_STABILIZED and must be 0 otherwise");
  }
  if (o) {
    if (!(o->tol >= 0)) return fail(RD_ERR_INVALID_ARG, "tol must be >= 0");
    if (o->tol_kind != RD_TOL_RES_ABS && o->tol_kind != RD_TOL_F_REL) return fail(RD_ERR_INVALID_ARG, "bad tol_kind");
    if (o->max_iter < 0) return fail(RD_ERR_INVALID_ARG, "max_iter must be >= 0");
    if (!(o->omega >= 0) || !std::isfinite(o->omega)) return fail(RD_ERR_INVALID_ARG, "omega must be >= 0");
    if (o->precision != RD_PREC_FP64 && o->precision != RD_PREC_FP32_DC) return fail(RD_ERR_INVALID_ARG, "bad precision");
    if (o->graph_k < 1 || o->graph_k > 256) return fail(RD_ERR_INVALID_ARG, "graph_k must be in [1, 256]");
    if (o->fft_buffers < 0 || o->fft_buffers > 2) return fail(RD_ERR_INVALID_ARG, "fft_buffers must be 0, 1 or 2");
    if (o->solve_loop != RD_LOOP_GRAPH && o->solve_loop != RD_LOOP_HOST) return fail(RD_ERR_INVALID_ARG, "bad solve_loop");
    if (o->fft_unrolled != 0 && o->fft_unrolled != 1) return fail(RD_ERR_INVALID_ARG, "fft_unrolled must be 0 or 1");
    if (o->autotune != 0 && o->autotune != 1) return fail(RD_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (o->fused_update != 0 && o->fused_update != 1) return fail(RD_ERR_INVALID_ARG, "fused_update must be 0 or 1");
    if (o->small_solve != 0 && o->small_solve != 1) return fail(RD_ERR_INVALID_ARG, "small_solve must be 0 or 1");
    if (o->precision == RD_PREC_FP32_DC && o->dc_stall_window < 1)
      return fail(RD_ERR_INVALID_ARG, "dc_stall_window must be >= 1");
    if (o->upd_rows < 0 || o->band_rows < 0 || o->col_width < 0) return fail(RD_ERR_INVALID_ARG, "negative tile size");
    if (o->precision == RD_PREC_FP32_DC && (!(o->dc_inner_rtol > 0) || o->dc_max_outer < 1))
      return fail(RD_ERR_INVALID_ARG, "bad defect-correction options");
  }
  return RD_OK;
}

// opts.autotune: on the handle's own arrays (zeroed, with a solve state that never stops, so that
// every candidate runs the full sweeps) time each kernel over kTuneIters iterations and keep the
// fastest tiles per kernel: band rows of k_res and of k_upd (each over 2..16 rows), column width
// of k_col (over 2..64 columns); the three are independent.  Candidates that the planner rejects
// or that exceed the device's shared memory are skipped.  The choice is reported in rd_stats
// (plan_band_rows, plan_upd_rows, plan_col_width).
constexpr int kTuneIters = 8;

template <class T>
rd_status autotune_plan(rd_pdhg* h, int H, int transform, int stage_base, int usable) {
  const int ti = h->dc ? 1 : 0;
  cudaStream_t s = h->stream;
  const size_t n = h->npts;
  if (h->dc) {
    for (void* p : {(void*)h->D32, (void*)h->P32[0], (void*)h->P32[1], (void*)h->WY32, (void*)h->r32, (void*)h->u32})
      RD_CUDA(cudaMemsetAsync(p, 0, n * sizeof(float), s));
  } else {
    for (void* p : {(void*)h->U64, (void*)h->rhs64, (void*)h->P64[0], (void*)h->P64[1], (void*)h->WY64})
      RD_CUDA(cudaMemsetAsync(p, 0, n * sizeof(double), s));
  }
  State run{};
  run.status = ST_ACTIVE;
  run.max_iter = 1 << 30;
  run.thresh = -1.0;  // never met: the sweeps stay active
  State* dst = h->d_state + 2;
  // per-kernel time (ms, best of three) of kTuneIters iterations for one plan; false if it failed
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < 4; ++i) RD_CUDA(cudaEventCreate(&ev[i]));
  auto time_plan = [&](const Desc& dt, const LaunchCfg& ct, float* kms) -> bool {
    for (int k = 0; k < 3; ++k) kms[k] = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      if (cudaMemcpyAsync(dst, &run, sizeof(State), cudaMemcpyHostToDevice, s) != cudaSuccess) return false;
      if (launch_iteration<T>(dt, dst, ct, s, nullptr) != cudaSuccess) return false;  // warm-up
      float acc[3] = {0.f, 0.f, 0.f};
      for (int it = 0; it < kTuneIters; ++it) {
        if (launch_iteration<T>(dt, dst, ct, s, ev) != cudaSuccess) return false;
        if (cudaStreamSynchronize(s) != cudaSuccess) return false;
        for (int k = 0; k < 3; ++k) {
          float t = 0.f;
          if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) != cudaSuccess) return false;
          acc[k] += t;
        }
      }
      for (int k = 0; k < 3; ++k) kms[k] = std::min(kms[k], acc[k]);
    }
    return true;
  };
  auto fits = [&](const LaunchCfg& ct) { return std::max(ct.smem_res, std::max(ct.smem_col, ct.smem_upd)) <= usable; };
  std::string why;
  const Desc& d0 = h->h_desc[ti];
  // band rows: k_res and k_upd timed at each height (column width as planned)
  float best_res = 1e30f, best_upd = 1e30f, best_col = 1e30f;
  int bestB = 0, bestU = 0, bestC = 0;
  for (int B = 2; B <= 16 && B <= h->ny; B *= 2) {
    Desc dt = d0;
    LaunchCfg ct{};
    if (!plan_launch<T>(h->nx, h->ny, h->nc, H, transform, h->bc == RD_BC_NEUMANN, B, d0.col_width, B, stage_base,
                        h->opts.fft_buffers, h->opts.fft_unrolled, dt, ct, why) ||
        !fits(ct))
      continue;
    float kms[3];
    if (!time_plan(dt, ct, kms)) {
      cudaGetLastError();
      continue;
    }
    if (kms[0] < best_res) best_res = kms[0], bestB = B;
    if (kms[2] < best_upd) best_upd = kms[2], bestU = B;
  }
  // column width: k_col timed at each width (band rows as planned)
  if (transform) {
    for (int Cw = 2; Cw <= 64 && Cw <= h->nx; Cw *= 2) {
      if (h->nx % Cw) continue;
      Desc dt = d0;
      LaunchCfg ct{};
      if (!plan_launch<T>(h->nx, h->ny, h->nc, H, transform, h->bc == RD_BC_NEUMANN, d0.band_rows, Cw, d0.upd_rows,
                          stage_base, h->opts.fft_buffers, h->opts.fft_unrolled, dt, ct, why) ||
          !fits(ct))
        continue;
      float kms[3];
      if (!time_plan(dt, ct, kms)) {
        cudaGetLastError();
        continue;
      }
      if (kms[1] < best_col) best_col = kms[1], bestC = Cw;
    }
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (bestB == 0 || bestU == 0) return RD_OK;  // nothing measured: keep the planner's choice
  if (bestC == 0) bestC = d0.col_width;
  Desc& d = h->h_desc[ti];
  LaunchCfg& lc = h->dc ? h->cfg32 : h->cfg64;
  LaunchCfg tuned{};
  Desc dtn = d;
  if (!plan_launch<T>(h->nx, h->ny, h->nc, H, transform, h->bc == RD_BC_NEUMANN, bestB, bestC, bestU, stage_base,
                      h->opts.fft_buffers, h->opts.fft_unrolled, dtn, tuned, why) || !fits(tuned))
    return RD_OK;  // the combination does not fit: keep the planner's choice
  d = dtn;
  lc = tuned;
  if (h->dc) {
    h->h_desc[0].band_rows = d.band_rows;
    h->h_desc[0].nbands = d.nbands;
    h->h_desc[0].col_width = d.col_width;
    h->h_desc[0].ncolblk = d.ncolblk;
    h->h_desc[0].upd_rows = d.upd_rows;
    h->h_desc[0].nupd = d.nupd;
  } else {
    h->cfgpc = lc;
    Desc& dp = h->h_desc[2];
    dp.band_rows = d.band_rows;
    dp.nbands = d.nbands;
    dp.col_width = d.col_width;
    dp.ncolblk = d.ncolblk;
    dp.upd_rows = d.upd_rows;
    dp.nupd = d.nupd;
    dp.fft_pp = d.fft_pp;
  }
  RD_CUDA(cudaMemcpy(h->d_desc, h->h_desc, 3 * sizeof(Desc), cudaMemcpyHostToDevice));
  return RD_OK;
}

// Fused update (opts.fused_update, FP32 defect correction, either loop): iterations after the
// first run k_col + k_updres, which needs a second transform buffer and per-band halo copies of
// U.  Left off when its block does not fit the device's shared memory, and, with opts.autotune,
// when a fused iteration is not at least 5% faster than an unfused one on this grid.
rd_status plan_fused(rd_pdhg* h, int H, int stage_base, int usable) {
  Desc& d = h->h_desc[1];
  LaunchCfg& lc = h->cfg32;
  const int U = d.upd_rows, nc = h->nc, nx = h->nx;
  const int lines = nc * ((U + 4 * H) / 2);
  const int smem = table_bytes<float>(nx, true, h->bc == RD_BC_NEUMANN) + lines * padded_len(nx) * (int)sizeof(cx<float>) +
                   nc * (U + 2 * H) * nx * (int)sizeof(float) * (stage_base ? 2 : 1);
  if (smem > usable) return RD_OK;
  RD_TRY(dalloc(h, &h->WY32b, h->npts * sizeof(float)));
  h->halo_bytes = (size_t)d.nupd * nc * 2 * H * nx * sizeof(float);
  RD_TRY(dalloc(h, &h->halo32, h->halo_bytes));
  Desc df = d;
  df.fused = 1;
  df.WYb[0] = h->WY32;
  df.WYb[1] = h->WY32b;
  df.halo = h->halo32;
  lc.thr_updres = band_threads<float>(lines, nx);
  lc.smem_updres = smem;
  if (h->opts.autotune) {
    // keep the fused update only if a fused iteration is faster than an unfused one here:
    // kTuneIters iterations of each on the handle's zeroed arrays, a solve that never stops
    cudaStream_t s = h->stream;
    for (void* p : {(void*)h->D32, (void*)h->P32[0], (void*)h->P32[1], (void*)h->WY32, (void*)h->WY32b,
                    (void*)h->r32, (void*)h->u32})
      RD_CUDA(cudaMemsetAsync(p, 0, h->npts * sizeof(float), s));
    RD_CUDA(cudaMemsetAsync(h->halo32, 0, h->halo_bytes, s));
    State run{};
    run.status = ST_ACTIVE;
    run.max_iter = 1 << 30;
    run.thresh = -1.0;
    State* dst = h->d_state + 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RD_CUDA(cudaEventCreate(&e0));
    RD_CUDA(cudaEventCreate(&e1));
    float t[2] = {1e30f, 1e30f};
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      for (int f = 0; f < 2 && ok; ++f) {
        RD_CUDA(cudaMemcpyAsync(dst, &run, sizeof(State), cudaMemcpyHostToDevice, s));
        ok = (f ? launch_fused<float>(df, dst, lc, s, nullptr, true) : launch_iteration<float>(d, dst, lc, s, nullptr)) ==
             cudaSuccess;
        RD_CUDA(cudaEventRecord(e0, s));
        for (int k = 0; k < kTuneIters && ok; ++k)
          ok = (f ? launch_fused<float>(df, dst, lc, s, nullptr, false) : launch_iteration<float>(d, dst, lc, s, nullptr)) ==
               cudaSuccess;
        RD_CUDA(cudaEventRecord(e1, s));
        RD_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        RD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t[f] = std::min(t[f], ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) cudaGetLastError();
    // stream-launched timing flatters the fused loop by a few percent against the graph loop
    // (measured): demand a 5% margin
    if (!ok || t[1] >= 0.95f * t[0]) return RD_OK;
  }
  d = df;
  RD_CUDA(cudaMemcpy(h->d_desc, h->h_desc, 3 * sizeof(Desc), cudaMemcpyHostToDevice));
  return RD_OK;
}

rd_status create_impl(rd_pdhg* h, const rd_grid* grid, rd_bc bc, rd_operator op, const rd_reaction* rx, double dt,
                      double tau, double sigma, const rd_precond* pc, const rd_opts* o, void* stream) {
  h->nx = grid->n[0];
  h->ny = grid->n[1];
  if (o) h->opts = *o; else rd_opts_default(&h->opts);
  h->dc = h->opts.precision == RD_PREC_FP32_DC;
  // 2-D grids with a side longer than the band / column sweeps transform (2048 points in FP32,
  // 4096 in FP64) run on the line-transform kernels of 3-D grids with nz = 1
  const bool long2d = grid->ndim == 2 && std::max(h->nx, h->ny) > (h->dc ? 2048 : 4096);
  if (long2d && rx->kind != RD_RX_NONE && rx->kind != RD_RX_ALLEN_CAHN && rx->kind != RD_RX_CH_IMPLICIT &&
      rx->kind != RD_RX_CH_SPLIT)
    return fail(RD_ERR_UNSUPPORTED, "2-D sides beyond 2048 (FP32) / 4096 (FP64) points are built for the scalar kinds");
  h->nd3 = grid->ndim == 3 || long2d;
  h->nz = grid->ndim == 3 ? grid->n[2] : 1;
  h->nc = rx->ncomp;
  h->npts = (size_t)h->nc * h->nx * h->ny * h->nz;
  h->bc = bc;
  h->op = op;
  h->kind = rx->kind;
  h->precond = pc ? pc->kind : RD_PC_LINEAR;
  h->pc_shift = pc && pc->kind == RD_PC_STABILIZED ? pc->s : 0.0;
  h->rx = *rx;
  h->dt = dt;
  h->tau = tau;
  h->sigma = sigma;
  h->hx = grid->length[0] / h->nx;
  h->hy = grid->length[1] / h->ny;
  h->hz = grid->ndim == 3 ? grid->length[2] / h->nz : 1.0;
  h->stream = static_cast<cudaStream_t>(stream);
  RD_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  RD_CUDA(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
  RD_CUDA(cudaStreamCreateWithFlags(&h->body_stream2, cudaStreamNonBlocking));

  const int H = op == RD_OP_NEG_BIHARMONIC ? 2 : 1;  // the sixth-order kind plans only the preconditioner
  h->fch = rx->kind == RD_RX_FCH;
  const int transform = h->precond != RD_PC_NONE;

  Desc base{};
  base.nx = h->nx;
  base.ny = h->ny;
  base.ncomp = h->nc;
  base.lognx = ilog2(h->nx);
  base.logny = ilog2(h->ny);
  base.bc = bc;
  base.op = op;
  base.kind = rx->kind;
  base.precond = h->precond;
  base.hx2 = 1.0 / (h->hx * h->hx);
  base.hy2 = 1.0 / (h->hy * h->hy);
  base.dt = dt;
  base.a = rx->a;
  base.b = rx->b;
  for (int k = 0; k < 6; ++k) base.p[k] = rx->p[k];
  base.tau_u = tau;
  base.tau_p = sigma;
  base.omega = h->opts.omega;
  base.nz = h->nz;
  base.lognz = ilog2(h->nz);
  base.hz2 = grid->ndim == 3 ? 1.0 / (h->hz * h->hz) : 0.0;  // 0: no z terms in the stencils

  std::string why;
  Desc d64 = base, d32 = base;
  if (h->nd3) {
    // 3-D grids: the rd_3d.cu kernels with their own plan (no band / column tiles, no autotuner,
    // no fused update)
    const char* w3 = nullptr;
    if (!plan3(h->nx, h->ny, h->nz, h->nc, 8, bc == RD_BC_NEUMANN, kSmemLimit, d64, &w3))
      return fail(RD_ERR_UNSUPPORTED, std::string("FP64 path: ") + w3);
    if (h->dc && !plan3(h->nx, h->ny, h->nz, h->nc, 4, bc == RD_BC_NEUMANN, kSmemLimit, d32, &w3))
      return fail(RD_ERR_UNSUPPORTED, std::string("FP32 path: ") + w3);
    h->cfg64.transform = h->cfg32.transform = transform;
  } else if (!plan_launch<double>(h->nx, h->ny, h->nc, H, transform, bc == RD_BC_NEUMANN, h->opts.band_rows, h->opts.col_width,
                           h->opts.upd_rows, 0, h->opts.fft_buffers, h->opts.fft_unrolled, d64, h->cfg64, why))
    if (!h->dc) return fail(RD_ERR_UNSUPPORTED, "FP64 path: " + why);
  if (h->dc && !h->nd3) {
    // the FP64 kernels of the defect-correction loop only need the band decomposition
    if (!plan_launch<float>(h->nx, h->ny, h->nc, H, transform, bc == RD_BC_NEUMANN, h->opts.band_rows, h->opts.col_width,
                           h->opts.upd_rows, rx->kind == RD_RX_CH_IMPLICIT || rx->kind == RD_RX_CH_SPLIT, h->opts.fft_buffers, h->opts.fft_unrolled, d32, h->cfg32, why))
      return fail(RD_ERR_UNSUPPORTED, "FP32 path: " + why);
    d64.band_rows = d32.band_rows;
    d64.nbands = d32.nbands;
    d64.col_width = d32.col_width;
    d64.ncolblk = d32.ncolblk;
    d64.upd_rows = d32.upd_rows;
    d64.nupd = d32.nupd;
  }

  const size_t n = h->npts;
  RD_TRY(dalloc(h, &h->U64, n * sizeof(double)));
  RD_TRY(dalloc(h, &h->rhs64, n * sizeof(double)));
  const int nb = std::max(d64.nbands, d32.nbands);
  // partials: per band (any band height the autotuner may try) or per step-kernel block
  const int nb_any = std::max(nb, h->ny / 2 + 1);
  const int nb3 = h->nd3 ? std::max(std::max(d64.blk3, d32.blk3), point_blocks(h->nx, h->ny * h->nz)) : 0;
  RD_TRY(dalloc(h, &h->partials,
                (size_t)2 * std::max(std::max(std::max(nb_any, point_blocks(h->nx, h->ny)), nb3), 1) * sizeof(double)));
  RD_TRY(dalloc(h, &h->d_desc, 3 * sizeof(Desc)));
  RD_TRY(dalloc(h, &h->d_state, 3 * sizeof(State)));
  if (h->fch) {
    RD_TRY(dalloc(h, &h->fchb.Pt, n * sizeof(double)));
    RD_TRY(dalloc(h, &h->fchb.M, n * sizeof(double)));
    RD_TRY(dalloc(h, &h->fchb.N, n * sizeof(double)));
    RD_TRY(dalloc(h, &h->fchb.Q, n * sizeof(double)));
  }
  RD_CUDA(cudaMallocHost(&h->h_state, 3 * sizeof(State)));

  std::vector<double> twx, dcx, twy, dcy, mx, my, twz, dcz, mz;
  host_twiddles(h->nx, twx, dcx);
  host_twiddles(h->ny, twy, dcy);
  host_mu(h, mx, my);
  if (h->nd3) {
    host_twiddles(h->nz, twz, dcz);
    host_mu_z(h, mz);
  }

  if (!h->dc) {
    RD_TRY(dalloc(h, &h->P64[0], n * sizeof(double)));
    RD_TRY(dalloc(h, &h->P64[1], n * sizeof(double)));
    RD_TRY(dalloc(h, &h->WY64, n * sizeof(double)));
    RD_TRY(dalloc(h, &h->tw64[0], (size_t)h->nx * sizeof(cx<double>)));
    RD_TRY(dalloc(h, &h->tw64[1], (size_t)h->ny * sizeof(cx<double>)));
    RD_TRY(dalloc(h, &h->tw64[2], (size_t)h->nx * sizeof(cx<double>)));
    RD_TRY(dalloc(h, &h->tw64[3], (size_t)h->ny * sizeof(cx<double>)));
    RD_CUDA(cudaMemcpy(h->tw64[0], twx.data(), twx.size() * sizeof(double), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(h->tw64[1], twy.data(), twy.size() * sizeof(double), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(h->tw64[2], dcx.data(), dcx.size() * sizeof(double), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(h->tw64[3], dcy.data(), dcy.size() * sizeof(double), cudaMemcpyHostToDevice));
    RD_TRY(dalloc(h, &h->mu64[0], (size_t)h->nx * sizeof(double)));
    RD_TRY(dalloc(h, &h->mu64[1], (size_t)h->ny * sizeof(double)));
    RD_CUDA(cudaMemcpy(h->mu64[0], mx.data(), mx.size() * sizeof(double), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(h->mu64[1], my.data(), my.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (h->nd3) {
      RD_TRY(dalloc(h, &h->tw64z[0], (size_t)h->nz * sizeof(cx<double>)));
      RD_TRY(dalloc(h, &h->tw64z[1], (size_t)h->nz * sizeof(cx<double>)));
      RD_TRY(dalloc(h, &h->mu64z, (size_t)h->nz * sizeof(double)));
      RD_CUDA(cudaMemcpy(h->tw64z[0], twz.data(), twz.size() * sizeof(double), cudaMemcpyHostToDevice));
      RD_CUDA(cudaMemcpy(h->tw64z[1], dcz.data(), dcz.size() * sizeof(double), cudaMemcpyHostToDevice));
      RD_CUDA(cudaMemcpy(h->mu64z, mz.data(), mz.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
  } else {
    RD_TRY(dalloc(h, &h->D32, n * sizeof(float)));
    RD_TRY(dalloc(h, &h->P32[0], n * sizeof(float)));
    RD_TRY(dalloc(h, &h->P32[1], n * sizeof(float)));
    RD_TRY(dalloc(h, &h->WY32, n * sizeof(float)));
    RD_TRY(dalloc(h, &h->r32, n * sizeof(float)));
    RD_TRY(dalloc(h, &h->u32, n * sizeof(float)));
    std::vector<float> f;
    auto up32 = [&](cx<float>** dst, const std::vector<double>& src, int len) -> rd_status {
      RD_TRY(dalloc(h, dst, (size_t)len * sizeof(cx<float>)));
      f.assign(src.begin(), src.end());
      RD_CUDA(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
      return RD_OK;
    };
    RD_TRY(up32(&h->tw32[0], twx, h->nx));
    RD_TRY(up32(&h->tw32[1], twy, h->ny));
    RD_TRY(up32(&h->tw32[2], dcx, h->nx));
    RD_TRY(up32(&h->tw32[3], dcy, h->ny));
    RD_TRY(dalloc(h, &h->mu32[0], (size_t)h->nx * sizeof(float)));
    RD_TRY(dalloc(h, &h->mu32[1], (size_t)h->ny * sizeof(float)));
    f.assign(mx.begin(), mx.end());
    RD_CUDA(cudaMemcpy(h->mu32[0], f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    f.assign(my.begin(), my.end());
    RD_CUDA(cudaMemcpy(h->mu32[1], f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (h->nd3) {
      RD_TRY(up32(&h->tw32z[0], twz, h->nz));
      RD_TRY(up32(&h->tw32z[1], dcz, h->nz));
      RD_TRY(dalloc(h, &h->mu32z, (size_t)h->nz * sizeof(float)));
      f.assign(mz.begin(), mz.end());
      RD_CUDA(cudaMemcpy(h->mu32z, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }

  // descriptors
  d64.dc = 0;
  d64.mode = MODE_PDHG;
  d64.meas_div_dt = h->opts.tol_kind == RD_TOL_RES_ABS;
  d64.X = h->U64;
  d64.base = nullptr;
  d64.rhs = h->rhs64;
  d64.P[0] = h->P64[0];
  d64.P[1] = h->P64[1];
  d64.WY = h->WY64;
  d64.scale = nullptr;
  d64.mux = h->mu64[0];
  d64.muy = h->mu64[1];
  symbol_coefficients(h, d64);
  d64.twx = h->tw64[0];
  d64.twy = h->tw64[1];
  d64.dcx = h->tw64[2];
  d64.dcy = h->tw64[3];
  d64.muz = h->mu64z;
  d64.twz = h->tw64z[0];
  d64.dcz = h->tw64z[1];
  d64.partials = h->partials;

  d32.dc = 1;
  d32.mode = MODE_PDHG;
  d32.meas_div_dt = 0;
  d32.stall_window = h->opts.dc_stall_window;
  d32.X = h->D32;
  d32.base = h->u32;
  d32.rhs = h->r32;
  d32.P[0] = h->P32[0];
  d32.P[1] = h->P32[1];
  d32.WY = h->WY32;
  d32.scale = nullptr;
  d32.mux = h->mu32[0];
  d32.muy = h->mu32[1];
  symbol_coefficients(h, d32);
  d32.twx = h->tw32[0];
  d32.twy = h->tw32[1];
  d32.dcx = h->tw32[2];
  d32.dcy = h->tw32[3];
  d32.muz = h->mu32z;
  d32.twz = h->tw32z[0];
  d32.dcz = h->tw32z[1];
  d32.partials = h->partials;

  Desc dpc = d64;
  dpc.mode = MODE_PRECOND_ONLY;
  dpc.X = h->P64[1];
  h->cfgpc = h->cfg64;

  h->h_desc[0] = d64;
  h->h_desc[1] = d32;
  h->h_desc[2] = dpc;
  RD_CUDA(cudaMemcpy(h->d_desc, h->h_desc, 3 * sizeof(Desc), cudaMemcpyHostToDevice));
  State st{};
  st.status = ST_IDLE;
  st.max_iter = h->opts.max_iter;
  State sts[3] = {st, st, st};
  RD_CUDA(cudaMemcpy(h->d_state, sts, sizeof(sts), cudaMemcpyHostToDevice));

  int usable = 0;
  if (h->dc) RD_CUDA(set_kernel_smem_limits<float>(&usable));
  else RD_CUDA(set_kernel_smem_limits<double>(&usable));
  if (h->nd3) {
    int dev = 0, optin = 0;
    RD_CUDA(cudaGetDevice(&dev));
    RD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RD_CUDA(h->dc ? allow3<float>(optin) : allow3<double>(optin));
    RD_CUDA(allow3<double>(optin));  // the preconditioner-only solve of rd_pdhg_apply_precond
  }
  const LaunchCfg& lc = h->dc ? h->cfg32 : h->cfg64;
  if (std::max(lc.smem_res, std::max(lc.smem_col, lc.smem_upd)) > usable)
    return fail(RD_ERR_UNSUPPORTED, "the grid needs more shared memory per block than this device offers");
  // FP32 defect correction on a grid whose whole inner solve fits one block: one launch per
  // inner solve (no band / column tiles to plan or tune)
  h->small = h->dc && !h->nd3 && !h->fch && transform && h->opts.small_solve
                 ? small_mode(h->nx, h->ny, h->nc,
                              rx->kind == RD_RX_NONE ? (op == RD_OP_NEG_BIHARMONIC ? KK_NONE_BIH : KK_NONE_LAP) : rx->kind,
                              bc == RD_BC_NEUMANN, usable)
                 : 0;
  if (h->small) {
    int dev = 0, optin = 0;
    RD_CUDA(cudaGetDevice(&dev));
    RD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RD_CUDA(allow_small(optin));
  }
  if (h->opts.autotune && !h->fch && !h->nd3 && !h->small && h->opts.band_rows == 0 && h->opts.col_width == 0 && h->opts.upd_rows == 0) {
    const int stage_base = h->dc && (rx->kind == RD_RX_CH_IMPLICIT || rx->kind == RD_RX_CH_SPLIT);
    RD_TRY(h->dc ? autotune_plan<float>(h, H, transform, stage_base, usable)
                 : autotune_plan<double>(h, H, transform, stage_base, usable));
  }
  if (h->dc && h->opts.fused_update && transform && !h->nd3 && !h->small) {
    const int stage_base = rx->kind == RD_RX_CH_IMPLICIT || rx->kind == RD_RX_CH_SPLIT;
    RD_TRY(plan_fused(h, H, stage_base, usable));
  }
  h->stats.fused_update = h->h_desc[1].fused;
  h->stats.small_solve = h->small;
  h->stats.line_kernels = h->nd3;
  h->stats.plan_band_rows = h->h_desc[h->dc ? 1 : 0].band_rows;
  h->stats.plan_upd_rows = h->h_desc[h->dc ? 1 : 0].upd_rows;
  h->stats.plan_col_width = h->h_desc[h->dc ? 1 : 0].col_width;
  RD_TRY(capture_graphs(h));
  RD_CUDA(cudaDeviceSynchronize());
  return RD_OK;
}

// Launch step graph `which`, read the three solve states back and account the launch.
rd_status graph_round(rd_pdhg* h, int which) {
  cudaStream_t s = h->stream;
  // graph 0 starts the step (k_begin resets the counters); graph 1 continues it
  const bool cont = h->dc && which == 1;
  const int upd_before = cont ? h->h_state[0].total : 0;
  const int launches_before = cont ? h->h_state[0].launches : 0;
  const int outer_before = cont ? h->h_state[0].n : 0;
  RD_CUDA(cudaGraphLaunch(h->gexec[which], s));
  RD_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, 3 * sizeof(State), cudaMemcpyDeviceToHost, s));
  RD_CUDA(cudaStreamSynchronize(s));
  const State& o = h->h_state[0];
  h->stats.graph_launches += 1;
  h->stats.host_syncs += 1;
  int updates, sweeps;
  if (h->dc) {
    updates = o.total - upd_before;
    sweeps = o.launches - launches_before;
    const int passes = o.n - outer_before;
    h->stats.residual_passes += passes;
    // the second k_resid64 and k_axpy_dc are captured in every round graph; k_begin and the
    // first k_resid64 in the first; k_mass in both
    h->stats.kernel_launches += (which == 0 ? 2 : 0) + 3;
  } else {
    updates = o.n;
    sweeps = (int)o.trips;
    h->stats.kernel_launches += 2;  // k_begin, k_mass (the P_0 clear is a memset node)
  }
  h->stats.pdhg_iterations += updates;
  if (h->small) {
    // one launch of the one-block inner solve per round graph; with the outer rounds on the
    // device (the first graph of a defect-correction step) four launches per round (inner
    // solve, u += d, FP64 residual, loop condition), counted by the outer state's trips, in
    // place of the one round the count above assumes
    if (h->dc && which == 0) h->stats.kernel_launches += 4LL * (long long)o.trips - 2;
    else h->stats.kernel_launches += 1;
    if (h->opts.profile && sweeps > 0) {
      float ms = 0.f;
      RD_CUDA(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
      h->stats.kernel_ms[0] += ms;
      h->stats.kernel_samples[0] += 1;
    }
    return RD_OK;
  }
  // every k_res launch (active or not) is followed by k_col and k_upd in the graph, and
  // k_loop_cond runs after the first and then after every graph_k of them; with the outer rounds
  // on the device (the first graph of a defect-correction step) each round adds its own first
  // iteration's loop condition and an outer loop condition, and the count above assumed one
  // round of u += d and FP64 residual
  h->stats.kernel_launches += (long long)sweeps * h->kernels_per_iter;
  if (h->dc && which == 0) {
    const long long R = o.trips;
    h->stats.kernel_launches += 4 * R - 2 + (sweeps - R) / h->opts.graph_k + (h->h_desc[1].fused ? R : 0);
  } else {
    h->stats.kernel_launches += sweeps > 0 ? 1 + (sweeps - 1) / h->opts.graph_k : 1;
  }
  if (h->opts.profile && sweeps > 0) {
    float ms = 0.f;
    RD_CUDA(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    h->stats.kernel_ms[0] += ms;
    h->stats.kernel_samples[0] += 1;
    if (updates > 0) {  // the first iteration updated: k_col and k_upd ran
      const int tr = (h->dc ? h->cfg32 : h->cfg64).transform;
      if (tr) {
        RD_CUDA(cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]));
        h->stats.kernel_ms[1] += ms;
        h->stats.kernel_samples[1] += 1;
      }
      RD_CUDA(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
      h->stats.kernel_ms[2] += ms;
      h->stats.kernel_samples[2] += 1;
    }
  }
  return RD_OK;
}

// RD_LOOP_HOST: launch the graph_k-iteration graph, read solve state `which` back and account.
rd_status iter_round(rd_pdhg* h, int which, bool start) {
  cudaStream_t s = h->stream;
  const int n_before = h->h_state[which].n;
  const bool first_graph = start && h->hexec1;
  RD_CUDA(cudaGraphLaunch(first_graph ? h->hexec1 : h->hexec, s));
  RD_CUDA(cudaMemcpyAsync(h->h_state + which, h->d_state + which, sizeof(State), cudaMemcpyDeviceToHost, s));
  RD_CUDA(cudaStreamSynchronize(s));
  const int updates = h->h_state[which].n - n_before;
  h->stats.graph_launches += 1;
  h->stats.kernel_launches += h->small ? 1 : (long long)h->opts.graph_k * h->kernels_per_iter + (first_graph ? 1 : 0);
  h->stats.host_syncs += 1;
  h->stats.pdhg_iterations += updates;
  if (h->small) {
    if (h->opts.profile) {
      float ms = 0.f;
      RD_CUDA(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
      h->stats.kernel_ms[0] += ms;
      h->stats.kernel_samples[0] += 1;
    }
    return RD_OK;
  }
  if (h->opts.profile && (first_graph || !h->hexec1)) {
    float ms = 0.f;
    RD_CUDA(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    h->stats.kernel_ms[0] += ms;
    h->stats.kernel_samples[0] += 1;
    if (updates > 0) {  // the first iteration updated: k_col and k_upd ran
      if ((h->dc ? h->cfg32 : h->cfg64).transform) {
        RD_CUDA(cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]));
        h->stats.kernel_ms[1] += ms;
        h->stats.kernel_samples[1] += 1;
      }
      RD_CUDA(cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
      h->stats.kernel_ms[2] += ms;
      h->stats.kernel_samples[2] += 1;
    }
  }
  return RD_OK;
}

// RD_LOOP_HOST: one implicit step with the loop decisions taken on the host.  The step kernels
// are the same as in the step graphs (k_resid64 applies the outer stopping rule and arms the
// inner solve, k_axpy_dc ends the step when the inner solve failed).
rd_status step_host(rd_pdhg* h, rd_step_info* info) {
  cudaStream_t s = h->stream;
  const Desc* d64 = h->d_desc + 0;
  State* st0 = h->d_state + 0;
  State* st1 = h->d_state + 1;
  const int nb = step_blocks(h);
  const int max_launch = h->opts.max_iter / h->opts.graph_k + 2;
  rd_step_info inf{};
  int final_status;
  RD_CUDA(begin_any(h, st0, h->U64, h->opts.tol, h->opts.tol_kind, nb, s));
  h->stats.kernel_launches += 2;  // k_begin, k_mass
  h->h_state[0].n = 0;
  h->h_state[1].n = 0;
  if (!h->dc) {
    RD_CUDA(cudaMemsetAsync(h->P64[0], 0, h->npts * sizeof(double), s));
    for (int it = 0; it <= max_launch; ++it) {
      RD_TRY(iter_round(h, 0, it == 0));
      if (h->h_state[0].status != ST_ACTIVE) break;
    }
    final_status = h->h_state[0].status;
    inf.iterations = h->h_state[0].n;
    inf.residual = h->h_state[0].r;
    if (final_status == ST_ACTIVE) return fail(RD_ERR_TIMEOUT, "PDHG loop exceeded its launch bound");
  } else {
    int inner_total = 0;
    for (int round = 0; round <= h->opts.dc_max_outer + 1; ++round) {
      RD_CUDA(resid64_any(h, st0, st1, h->U64, nullptr, h->r32, h->u32, h->D32, h->P32[0], 1, nb, s));
      RD_CUDA(cudaMemcpyAsync(h->h_state, h->d_state, 2 * sizeof(State), cudaMemcpyDeviceToHost, s));
      RD_CUDA(cudaStreamSynchronize(s));
      h->stats.kernel_launches += 1;
      h->stats.host_syncs += 1;
      if (h->h_state[0].status != ST_ACTIVE) break;  // converged, diverged, or out of rounds
      for (int it = 0; it <= max_launch; ++it) {
        RD_TRY(iter_round(h, 1, it == 0));
        if (h->h_state[1].status != ST_ACTIVE) break;
      }
      inner_total += h->h_state[1].n;
      RD_CUDA(launch_axpy_dc(h->U64, h->D32, h->npts, st0, st1, s));
      h->stats.kernel_launches += 1;
    }
    final_status = h->h_state[0].status;
    if (final_status == ST_ACTIVE) return fail(RD_ERR_TIMEOUT, "defect-correction loop exceeded its round bound");
    h->stats.residual_passes += h->h_state[0].n;  // FP64 evaluations k_resid64 counted
    inf.iterations = inner_total;
    inf.outer_rounds = h->h_state[0].n;
    inf.residual = h->h_state[0].r;
  }
  RD_CUDA(launch_mass(d64, h->d_state + 2, h->U64, nullptr, nb, s));
  RD_CUDA(cudaMemcpyAsync(h->h_state + 2, h->d_state + 2, sizeof(State), cudaMemcpyDeviceToHost, s));
  RD_CUDA(cudaStreamSynchronize(s));
  h->stats.host_syncs += 1;
  inf.mass = h->h_state[2].mass;
  inf.converged = final_status == ST_CONVERGED;
  inf.status = status_of(final_status);
  if (info) *info = inf;
  if (inf.status != RD_OK)
    return fail((rd_status)inf.status, inf.status == RD_ERR_DIVERGED ? "PDHG diverged" : "PDHG did not converge");
  return RD_OK;
}

// One implicit step on the handle's FP64 iterate U64 (holding U^k).  FP64: one graph launch
// runs the whole step.  Defect correction: the first graph runs the outer rounds in a device
// loop too; should that loop reach its bound with the step still active, the second graph
// takes one host-driven round at a time (the host reading the outer state between them).
rd_status step_impl(rd_pdhg* h, rd_step_info* info) {
  if (h->opts.solve_loop == RD_LOOP_HOST) return step_host(h, info);
  rd_step_info inf{};
  int final_status;
  RD_TRY(graph_round(h, 0));
  if (!h->dc) {
    final_status = h->h_state[0].status;
    inf.iterations = h->h_state[0].n;
    inf.residual = h->h_state[0].r;
    if (final_status == ST_ACTIVE) return fail(RD_ERR_TIMEOUT, "PDHG loop exceeded its launch bound");
  } else {
    for (int round = 1; h->h_state[0].status == ST_ACTIVE && round <= h->opts.dc_max_outer + 1; ++round)
      RD_TRY(graph_round(h, 1));
    final_status = h->h_state[0].status;
    if (final_status == ST_ACTIVE) return fail(RD_ERR_TIMEOUT, "defect-correction loop exceeded its round bound");
    inf.iterations = h->h_state[0].total;
    inf.outer_rounds = h->h_state[0].n;
    inf.residual = h->h_state[0].r;
  }
  inf.mass = h->h_state[2].mass;
  inf.converged = final_status == ST_CONVERGED;
  inf.status = status_of(final_status);
  if (info) *info = inf;
  if (inf.status != RD_OK)
    return fail((rd_status)inf.status, inf.status == RD_ERR_DIVERGED ? "PDHG diverged" : "PDHG did not converge");
  return RD_OK;
}

}  // namespace

extern "C" {

void rd_opts_default(rd_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->tol_kind = RD_TOL_RES_ABS;
  o->max_iter = 10000;
  o->omega = 1.0;
  o->precision = RD_PREC_FP64;
  o->dc_inner_rtol = 1e-5;
  o->dc_max_outer = 64;
  o->graph_k = 2;
  o->band_rows = 0;
  o->col_width = 0;
  o->upd_rows = 0;
  o->profile = 0;
  o->fft_buffers = 0;
  o->solve_loop = RD_LOOP_GRAPH;
  o->fft_unrolled = 1;
  o->autotune = 0;
  o->dc_stall_window = kDcStallWindow;
  o->fused_update = 1;
  o->small_solve = 1;
}

rd_status rd_pdhg_create(rd_pdhg** out, const rd_grid* grid, rd_bc bc, rd_operator op, const rd_reaction* reaction,
                         double dt, double tau, double sigma, const rd_precond* precond, const rd_opts* opts,
                         void* cuda_stream) {
  if (!out) return fail(RD_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  rd_status v = validate(grid, bc, op, reaction, dt, tau, sigma, precond, opts);
  if (v != RD_OK) return v;
  rd_pdhg* h = new (std::nothrow) rd_pdhg();
  if (!h) return fail(RD_ERR_OOM, "host allocation failed");
  rd_status s = create_impl(h, grid, bc, op, reaction, dt, tau, sigma, precond, opts, cuda_stream);
  if (s != RD_OK) {
    std::string keep = g_last_error;
    rd_pdhg_destroy(h);
    g_last_error = keep;
    return s;
  }
  *out = h;
  return RD_OK;
}

rd_status rd_pdhg_step(rd_pdhg* h, const double* u_n, double* u_np1, rd_step_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (!h || !u_n || !u_np1) return fail(RD_ERR_INVALID_ARG, "NULL handle or buffer");
  const size_t bytes = h->npts * sizeof(double);
  RD_CUDA(cudaMemcpyAsync(h->U64, u_n, bytes, cudaMemcpyDeviceToDevice, h->stream));
  rd_status s = step_impl(h, info);
  if (s == RD_OK || s == RD_ERR_NOT_CONVERGED || s == RD_ERR_DIVERGED) {
    std::string keep = g_last_error;
    RD_CUDA(cudaMemcpyAsync(u_np1, h->U64, bytes, cudaMemcpyDeviceToDevice, h->stream));
    RD_CUDA(cudaStreamSynchronize(h->stream));
    g_last_error = keep;
  }
  return s;
}

namespace {
// Algorithm 1's time loop on the handle's iterate U64.
rd_status solve_u64(rd_pdhg* h, int nsteps, rd_step_info* per_step) {
  for (int k = 0; k < nsteps; ++k) {
    rd_status s = step_impl(h, per_step ? per_step + k : nullptr);
    if (s != RD_OK) return s;
  }
  return RD_OK;
}
}  // namespace

rd_status rd_pdhg_solve(rd_pdhg* h, double* u, int nsteps, rd_step_info* per_step) {
  if (!h || !u) return fail(RD_ERR_INVALID_ARG, "NULL handle or buffer");
  if (nsteps < 0) return fail(RD_ERR_INVALID_ARG, "nsteps must be >= 0");
  const size_t bytes = h->npts * sizeof(double);
  if (per_step) std::memset(per_step, 0, sizeof(rd_step_info) * (size_t)nsteps);
  RD_CUDA(cudaMemcpyAsync(h->U64, u, bytes, cudaMemcpyDeviceToDevice, h->stream));
  rd_status s = solve_u64(h, nsteps, per_step);
  std::string keep = g_last_error;
  RD_CUDA(cudaMemcpyAsync(u, h->U64, bytes, cudaMemcpyDeviceToDevice, h->stream));
  RD_CUDA(cudaStreamSynchronize(h->stream));
  g_last_error = keep;
  return s;
}

rd_status rd_pdhg_solve_host(rd_pdhg* h, double* u_host, int nsteps, rd_step_info* per_step) {
  if (!h || !u_host) return fail(RD_ERR_INVALID_ARG, "NULL handle or buffer");
  if (nsteps < 0) return fail(RD_ERR_INVALID_ARG, "nsteps must be >= 0");
  const size_t bytes = h->npts * sizeof(double);
  if (per_step) std::memset(per_step, 0, sizeof(rd_step_info) * (size_t)nsteps);
  RD_CUDA(cudaMemcpyAsync(h->U64, u_host, bytes, cudaMemcpyHostToDevice, h->stream));
  rd_status s = solve_u64(h, nsteps, per_step);
  std::string keep = g_last_error;
  RD_CUDA(cudaMemcpyAsync(u_host, h->U64, bytes, cudaMemcpyDeviceToHost, h->stream));
  RD_CUDA(cudaStreamSynchronize(h->stream));
  g_last_error = keep;
  return s;
}

rd_status rd_pdhg_set_dt(rd_pdhg* h, double dt) {
  if (!h) return fail(RD_ERR_INVALID_ARG, "NULL handle");
  return set_dt_impl(h, dt);
}

namespace {
// The step-size rule of Section 2.2 after an accepted step of m PDHG iterations.
double next_dt(double dt, int m, double dt0, const rd_adapt* a) {
  if (m > a->n_hi) return a->eta * dt;
  if (m < a->n_lo) {
    const double up = dt / a->eta;
    return up <= dt0 ? up : dt;
  }
  return dt;
}
}  // namespace

rd_status rd_pdhg_solve_adaptive(rd_pdhg* h, double* u, const rd_adapt* a, rd_adapt_step* log, int log_cap,
                                 int* n_attempts, double* t_reached) {
  if (n_attempts) *n_attempts = 0;
  if (t_reached) *t_reached = 0.0;
  if (!h || !u || !a) return fail(RD_ERR_INVALID_ARG, "NULL handle, buffer or parameters");
  if (!(a->t_end > 0.0) || !std::isfinite(a->t_end) || !(a->eta > 0.0 && a->eta < 1.0) || a->n_lo < 0 ||
      a->n_lo > a->n_hi || a->max_attempts <= 0 || log_cap < 0 || (log_cap > 0 && !log))
    return fail(RD_ERR_INVALID_ARG, "bad adaptive step parameters");
  const size_t bytes = h->npts * sizeof(double);
  const double dt0 = h->dt;
  double dt = dt0, t = 0.0;
  int n = 0;
  rd_status result = RD_OK;
  while (a->t_end - t > 1e-12 * a->t_end) {
    if (n == a->max_attempts) {
      result = fail(RD_ERR_NOT_CONVERGED, "adaptive time stepping ran out of attempts");
      break;
    }
    const double rem = a->t_end - t;
    const double step = dt < rem ? dt : rem;
    rd_status s = set_dt_impl(h, step);
    if (s == RD_OK) {
      const cudaError_t e = cudaMemcpyAsync(h->U64, u, bytes, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) s = fail(RD_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    rd_step_info inf{};
    if (s == RD_OK) s = step_impl(h, &inf);
    if (s != RD_OK && s != RD_ERR_NOT_CONVERGED && s != RD_ERR_DIVERGED) {
      result = s;
      break;
    }
    const bool ok = s == RD_OK;
    if (n < log_cap) log[n] = rd_adapt_step{t, step, inf.iterations, inf.outer_rounds, (int)s, ok ? 1 : 0};
    ++n;
    if (ok) {
      const cudaError_t e = cudaMemcpyAsync(u, h->U64, bytes, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) {
        result = fail(RD_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
        break;
      }
      t = t + step;
      dt = next_dt(dt, inf.iterations, dt0, a);
    } else {
      dt = a->eta * dt;
    }
  }
  if (n_attempts) *n_attempts = n;
  if (t_reached) *t_reached = t;
  const std::string keep = g_last_error;
  const rd_status r = set_dt_impl(h, dt0);
  if (result == RD_OK && r != RD_OK) return r;
  RD_CUDA(cudaStreamSynchronize(h->stream));
  g_last_error = keep;
  return result;
}

rd_status rd_pdhg_residual(rd_pdhg* h, const double* u, const double* u_k, double* w) {
  if (!h || !u || !u_k || !w) return fail(RD_ERR_INVALID_ARG, "NULL handle or buffer");
  const int nb = step_blocks(h);
  RD_CUDA(begin_any(h, h->d_state + 2, u_k, 0.0, 0, nb, h->stream));
  if (h->fch) {
    RD_CUDA(launch_fch_residual(h->h_desc[0], nullptr, h->fchb, u, h->rhs64, w, 2 * nb, h->stream));
    RD_CUDA(cudaStreamSynchronize(h->stream));
    return RD_OK;
  }
  RD_CUDA(resid64_any(h, h->d_state + 2, h->d_state + 2, u, w, nullptr, nullptr, nullptr, nullptr, 0, nb, h->stream));
  RD_CUDA(cudaStreamSynchronize(h->stream));
  return RD_OK;
}

rd_status rd_pdhg_apply_precond(rd_pdhg* h, const double* w, double* y) {
  if (!h || !w || !y) return fail(RD_ERR_INVALID_ARG, "NULL handle or buffer");
  if (h->dc) return fail(RD_ERR_UNSUPPORTED, "apply_precond needs a handle created with RD_PREC_FP64");
  const size_t bytes = h->npts * sizeof(double);
  if (h->nd3) {
    // W into the transform buffer; the five transform passes leave Y in P64[1] (h_desc[2].X)
    if (h->precond == RD_PC_NONE) {
      RD_CUDA(cudaMemcpyAsync(y, w, bytes, cudaMemcpyDeviceToDevice, h->stream));
      RD_CUDA(cudaStreamSynchronize(h->stream));
      return RD_OK;
    }
    RD_CUDA(cudaMemcpyAsync(h->WY64, w, bytes, cudaMemcpyDeviceToDevice, h->stream));
    RD_CUDA(launch_precond3<double>(h->h_desc[2], h->d_state + 2, h->stream));
    RD_CUDA(cudaMemcpyAsync(y, h->P64[1], bytes, cudaMemcpyDeviceToDevice, h->stream));
    RD_CUDA(cudaStreamSynchronize(h->stream));
    return RD_OK;
  }
  RD_CUDA(cudaMemcpyAsync(h->P64[1], w, bytes, cudaMemcpyDeviceToDevice, h->stream));
  RD_CUDA(launch_iteration<double>(h->h_desc[2], h->d_state + 2, h->cfgpc, h->stream, nullptr));
  RD_CUDA(cudaMemcpyAsync(y, h->P64[1], bytes, cudaMemcpyDeviceToDevice, h->stream));
  RD_CUDA(cudaStreamSynchronize(h->stream));
  return RD_OK;
}

rd_status rd_pdhg_get_stats(const rd_pdhg* h, rd_stats* out) {
  if (!h || !out) return fail(RD_ERR_INVALID_ARG, "NULL handle or output");
  *out = h->stats;
  return RD_OK;
}

rd_status rd_pdhg_reset_stats(rd_pdhg* h) {
  if (!h) return fail(RD_ERR_INVALID_ARG, "NULL handle");
  const int pb = h->stats.plan_band_rows, pc = h->stats.plan_col_width, pu = h->stats.plan_upd_rows;
  const int fu = h->stats.fused_update, sm = h->stats.small_solve, lk = h->stats.line_kernels;
  h->stats = rd_stats{};
  h->stats.fused_update = fu;
  h->stats.small_solve = sm;
  h->stats.line_kernels = lk;
  h->stats.plan_band_rows = pb;
  h->stats.plan_col_width = pc;
  h->stats.plan_upd_rows = pu;
  return RD_OK;
}

void rd_pdhg_destroy(rd_pdhg* h) {
  if (!h) return;
  for (int i = 0; i < 4; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->body_stream) cudaStreamDestroy(h->body_stream);
  if (h->body_stream2) cudaStreamDestroy(h->body_stream2);
  delete h;
}

const char* rd_status_string(rd_status s) {
  switch (s) {
    case RD_OK: return "RD_OK";
    case RD_ERR_INVALID_ARG: return "RD_ERR_INVALID_ARG";
    case RD_ERR_UNSUPPORTED: return "RD_ERR_UNSUPPORTED";
    case RD_ERR_OOM: return "RD_ERR_OOM";
    case RD_ERR_CUDA: return "RD_ERR_CUDA";
    case RD_ERR_NOT_CONVERGED: return "RD_ERR_NOT_CONVERGED";
    case RD_ERR_DIVERGED: return "RD_ERR_DIVERGED";
    case RD_ERR_TIMEOUT: return "RD_ERR_TIMEOUT";
    case RD_ERR_BUSY: return "RD_ERR_BUSY";
  }
  return "RD_ERR_UNKNOWN";
}

const char* rd_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
