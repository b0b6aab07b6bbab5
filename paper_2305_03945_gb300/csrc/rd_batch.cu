// Batched, continuously served implicit steps (many independent solves of uneven grid sizes).
//
// Every admitted request owns a slot: device buffers cut from one arena sized by the caller's
// HBM budget, two descriptors (FP32 inner sweeps, FP64 outer loop) and a control block whose
// phase drives FP64 defect correction and the time-step loop on the device:
//   BEGIN  -> build the step's rhs from U^k and the outer threshold (k_step_b)
//   RESID  -> r = F(u) in FP64, outer stopping rule, arm the FP32 inner solve (k_step_b)
//   INNER  -> FP32 G-prox PDHG iterations on the correction equation (k_res_b, k_col_b,
//             k_upd_b), returning to AXPY when the inner solve stops
//   AXPY   -> u += d in FP64 (k_axpy_b)
//   DONE / FAILED after the last step or on divergence.
// One CUDA graph holds graph_k iterations of [axpy, step, res, col, upd] for each equation kind
// present; every launch covers all slots of that kind through a work list of (slot, block)
// pairs, so instances of different sizes share one launch.  A host worker thread admits queued
// requests when a slot and arena space are free, relaunches the graph, and retires finished
// slots while the others keep running (continuous batching).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rd_pdhg.h"
#include "rd_3d.cuh"
#include "rd_batch3.h"
#include "rd_launch3.h"
#include "rd_launch_small.h"

namespace rd {

// ---------------------------------------------------------------------------------------
// batched kernels
// ---------------------------------------------------------------------------------------
template <class T, int K>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value)
    k_res_b(const Desc* __restrict__ descs, Slot* __restrict__ slots, const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (*((volatile const int*)&slots[w.x].phase) != PH_INNER) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  res_body<T, K>(sd, &slots[w.x].inner, slots + w.x, w.y, smem_raw);
}

template <class T>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value)
    k_col_b(const Desc* __restrict__ descs, Slot* __restrict__ slots, const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (*((volatile const int*)&slots[w.x].phase) != PH_INNER) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  col_body<T, false>(sd, &slots[w.x].inner, slots + w.x, w.y, smem_raw);
}

template <class T, int K>
__global__ void __launch_bounds__(MaxThreads<T>::value, MinBlocks<T>::value)
    k_upd_b(const Desc* __restrict__ descs, Slot* __restrict__ slots, const int2* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  const int2 w = items[blockIdx.x];
  if (*((volatile const int*)&slots[w.x].phase) != PH_INNER) return;
  load_desc(sd, descs + w.x);
  __syncthreads();
  upd_body<T, K>(sd, &slots[w.x].inner, slots + w.x, w.y, smem_raw);
}

// FP64 state of a slot read through the boundary map
struct UAcc {
  const double* u;
  int nx, ny, bc;
  __device__ __forceinline__ double operator()(int i, int j) const {
    return u[(size_t)bcmap(i, ny, bc) * nx + bcmap(j, nx, bc)];
  }
};

// PH_BEGIN: rhs of the step from U^k (kind constants, the explicit part of the convex split),
//           ||U^k||, outer threshold, -> PH_RESID.
// PH_RESID: r = F(u) in FP64; r and u rounded to FP32 for the inner solve; d = 0, P_0 = 0;
//           outer stopping rule -> next step / DONE / FAILED, or arm the inner solve -> PH_INNER.
template <int K>
__global__ void __launch_bounds__(256) k_step_b(const Desc* __restrict__ d64s, Slot* __restrict__ slots,
                                                const int2* __restrict__ items) {
  __shared__ Desc sd;
  __shared__ double red[32];
  const int2 w = items[blockIdx.x];
  Slot* sl = slots + w.x;
  const int ph = *((volatile const int*)&sl->phase);
  if (ph != PH_BEGIN && ph != PH_RESID) return;
  load_desc(sd, d64s + w.x);
  __syncthreads();
  const Desc& d = sd;
  const int nx = d.nx, ny = d.ny, bc = d.bc;
  const size_t plane = (size_t)nx * ny;
  const int band = w.y;
  const int y0 = band * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  double* u = static_cast<double*>(d.X);
  double* rhs = static_cast<double*>(const_cast<void*>(d.rhs));
  constexpr int nc = KT<K>::two ? 2 : 1;
  State* outer = &sl->outer;
  if (ph == PH_BEGIN) {
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < nc * rows * nx; idx += blockDim.x) {
      const int c = idx / (rows * nx);
      const int rem = idx - c * rows * nx;
      const int r = rem / nx, j = rem - r * nx;
      const int i = y0 + r;
      const size_t o = c * plane + (size_t)i * nx + j;
      const double uv = u[o];
      double v = uv;
      if constexpr (K == KK_CH_SPLIT) {
        const UAcc f{u, nx, ny, bc};
        v = uv - d.dt * d.b * lap5(f, i, j, uv, d.hx2, d.hy2);
      } else if constexpr (K == KK_GS) {
        if (c == 0) v = uv + d.dt * d.p[2];
      } else if constexpr (K == KK_SCHNAK) {
        v = uv + d.dt * d.p[2] * (c == 0 ? d.p[3] : d.p[4]);
      }
      rhs[o] = v;
      acc += uv * uv;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) d.partials[band] = s;
    if (last_block(outer, d.nbands)) {
      __threadfence();
      const double tot = sum_partials(d.partials, d.nbands, red);
      if (threadIdx.x == 0) {
        outer->ticket = 0u;
        outer->aux = sqrt(tot);
        outer->thresh = sl->tol_kind == 1 ? sl->tol * sqrt(tot) : sl->tol;
        outer->n = 0;
        outer->r = 0.0;
        outer->r0 = 0.0;
        outer->status = ST_ACTIVE;
        sl->phase = PH_RESID;
      }
    }
    return;
  }
  // PH_RESID
  const UAcc f0{u, nx, ny, bc}, f1{u + plane, nx, ny, bc};
  double acc0 = 0.0, acc1 = 0.0;
  for (int idx = threadIdx.x; idx < rows * nx; idx += blockDim.x) {
    const int r = idx / nx, j = idx - r * nx;
    const int i = y0 + r;
    const size_t o = (size_t)i * nx + j;
    double wv[2] = {0.0, 0.0};
    residual_pt<double, K, false>(d, f0, f1, f0, f1, i, j, rhs[o], nc > 1 ? rhs[plane + o] : 0.0, wv);
    for (int c = 0; c < nc; ++c) {
      const size_t oc = c * plane + o;
      d.f32_r[oc] = (float)wv[c];
      d.f32_u[oc] = (float)u[oc];
      d.f32_d[oc] = 0.f;
      d.f32_p0[oc] = 0.f;
    }
    acc0 += wv[0] * wv[0];
    acc1 += wv[1] * wv[1];
  }
  const double s0 = block_sum(acc0, red);
  const double s1 = nc > 1 ? block_sum(acc1, red) : 0.0;
  if (threadIdx.x == 0) {
    d.partials[band] = s0;
    if (nc > 1) d.partials[d.nbands + band] = s1;
  }
  if (last_block(outer, d.nbands)) {
    __threadfence();
    double tot = 0.0;
    for (int c = 0; c < nc; ++c) tot += sqrt(sum_partials(d.partials + c * d.nbands, d.nbands, red));
    if (threadIdx.x == 0) {
      const double meas = d.meas_div_dt ? tot / d.dt : tot;
      const double prev = outer->r;
      outer->ticket = 0u;
      outer->r = meas;
      const int n = outer->n;
      if (n == 0) outer->r0 = meas;
      const double r0 = n == 0 ? meas : outer->r0;
      outer->n = n + 1;
      sl->outer_total += 1;
      if (meas <= outer->thresh) {
        outer->status = ST_CONVERGED;
        sl->steps_done += 1;
        sl->phase = sl->steps_done >= sl->nsteps ? PH_DONE : PH_BEGIN;
      } else if (!isfinite(meas) || meas > kDivergeFactor * r0 || outer->n > sl->max_outer) {
        outer->status = isfinite(meas) && meas <= kDivergeFactor * r0 ? ST_NOT_CONVERGED : ST_DIVERGED;
        sl->phase = PH_FAILED;
      } else {
        State* in = &sl->inner;
        in->stall_mul = next_stall_mul(n, meas, prev, in->stall_mul);
        in->n = 0;
        in->r = 0.0;
        in->r0 = 0.0;
        in->thresh = fmax(sl->rtol * tot, 0.5 * outer->thresh * (d.meas_div_dt ? d.dt : 1.0));
        in->status = ST_ACTIVE;
        in->ticket = 0u;
        sl->phase = PH_INNER;
      }
    }
  }
}

// PH_AXPY: u += d (FP64 += FP32), pointwise over the band, -> PH_RESID.
__global__ void __launch_bounds__(256) k_axpy_b(const Desc* __restrict__ d64s, Slot* __restrict__ slots,
                                                const int2* __restrict__ items) {
  const int2 w = items[blockIdx.x];
  Slot* sl = slots + w.x;
  if (*((volatile const int*)&sl->phase) != PH_AXPY) return;
  const Desc& d = d64s[w.x];
  const int nx = d.nx, ny = d.ny, nc = d.ncomp;
  const size_t plane = (size_t)nx * ny;
  const int y0 = w.y * d.band_rows;
  const int rows = min(d.band_rows, ny - y0);
  double* u = static_cast<double*>(d.X);
  const float* dl = d.f32_d;
  for (int idx = threadIdx.x; idx < nc * rows * nx; idx += blockDim.x) {
    const int c = idx / (rows * nx);
    const size_t o = c * plane + (size_t)y0 * nx + (idx - c * rows * nx);
    u[o] += (double)dl[o];
  }
  if (last_block(&sl->outer, d.nbands) && threadIdx.x == 0) {
    sl->outer.ticket = 0u;
    sl->phase = PH_RESID;
  }
}

}  // namespace rd

using namespace rd;

// ---------------------------------------------------------------------------------------
// host runtime
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kBatchThreads = 256;      // FP32 sweep blocks
constexpr int kBatchMaxSide = 1024;     // batch grids: sides 4 .. 1024, powers of two
constexpr int kBatchMaxSide3 = 512;     // 3-D batch grids: sides 4 .. 512
constexpr int kBatchMaxBlk3 = 1024;     // blocks per 3-D slot (plan3's cap)
constexpr int kBatchBandRows = 4;
constexpr int kBatchColWidth = 4;
constexpr int kBatchGroups = 7;         // equation kinds served
const int kGroupKey[kBatchGroups] = {KK_NONE_LAP, KK_AC, KK_CH_IMPL, KK_CH_SPLIT, KK_NONE_BIH, KK_GS, KK_SCHNAK};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// first-fit allocator over one device arena (offsets aligned to 256 bytes)
struct Arena {
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(char* b, size_t s) {
    base = b;
    size = s;
    free_.clear();
    free_[0] = s;
  }
  static size_t up(size_t v) { return (v + 255) & ~(size_t)255; }
  char* alloc(size_t n) {
    n = up(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        return base + off;
      }
    }
    return nullptr;
  }
  void release(char* p, size_t n) {
    n = up(n);
    size_t off = (size_t)(p - base);
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + n == nx->first) {
      n += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        off = pv->first;
        n += pv->second;
        free_.erase(pv);
      }
    }
    free_[off] = n;
  }
};

struct Request {
  uint64_t id = 0;
  rd_request req{};
  std::vector<double> u0;
  double t_submit = 0;
};

struct SlotHost {
  bool used = false;
  uint64_t id = 0;
  rd_request req{};
  int key = 0, group = 0;
  char* mem = nullptr;
  size_t mem_bytes = 0;
  size_t npts = 0;
  double t_submit = 0, t_admit = 0;
  bool nd3 = false;  // a 3-D request (the rd_batch3.cu kernels)
  int small = 0;     // a 2-D request whose inner solves run in one launch (1 one block, 2 a cluster)
  Desc d32{}, d64{};
};

size_t slot_bytes(const rd_request& r, size_t* npts_out) {
  const bool nd3 = r.grid.ndim == 3;
  const int nz = nd3 ? r.grid.n[2] : 1;
  const size_t npts = (size_t)r.reaction.ncomp * r.grid.n[0] * r.grid.n[1] * nz;
  if (npts_out) *npts_out = npts;
  const int nx = r.grid.n[0], ny = r.grid.n[1];
  size_t b = 0;
  if (nd3) {
    b += Arena::up(npts * 8) * 2;                       // u, rhs (FP64)
    b += Arena::up(npts * 4) * 5;                       // d, P, WY, r32, u32
    b += Arena::up((size_t)(nx + ny + nz) * 2 * 8);     // twiddles + rotations (FP32 complex)
    b += Arena::up((size_t)(nx + ny + nz) * 4);         // mu tables
    b += Arena::up((size_t)2 * kBatchMaxBlk3 * 8);      // partials
    return b;
  }
  b += Arena::up(npts * 8) * 2;                       // u, rhs (FP64)
  b += Arena::up(npts * 4) * 6;                       // d, P0, P1, WY, r32, u32
  b += Arena::up((size_t)(nx + ny) * 2 * 8) * 1;      // twiddles + rotations (FP32 complex)
  b += Arena::up((size_t)(nx + ny) * 4);              // mu tables
  b += Arena::up((size_t)2 * (ny / 2 + 1) * 8);  // partials (two-row bands at the finest tile)
  return b;
}

}  // namespace

struct rd_batch {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  rd_opts opts{};
  int max_slots = 0;
  size_t budget = 0;
  Arena arena;
  char* arena_mem = nullptr;
  Desc* d_d32 = nullptr;
  Desc* d_d64 = nullptr;
  Slot* d_slots = nullptr;
  Slot* h_slots = nullptr;  // pinned mirror
  int2* d_band_items[kBatchGroups] = {};
  int2* d_col_items[kBatchGroups] = {};
  int n_band[kBatchGroups] = {}, n_col[kBatchGroups] = {};
  std::vector<int2> h_band[kBatchGroups], h_col[kBatchGroups];
  // the step-phase kernels (axpy, step) run over the bands of every 2-D slot; the sweeps
  // (res, col, upd) over the slots without a one-launch inner solve, which run k_small_*_b on
  // their own work lists (one entry per slot) in a parallel branch of the graph
  int2* d_phase_items[kBatchGroups] = {};
  int n_phase[kBatchGroups] = {};
  std::vector<int2> h_phase[kBatchGroups];
  int2* d_small_items[kBatchGroups][2] = {};
  int n_small[kBatchGroups][2] = {};
  std::vector<int2> h_small[kBatchGroups][2];
  int smem_small[kBatchGroups][2] = {};
  int smem_usable = 0;
  cudaStream_t fork_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // 3-D slots: one work list of (slot, block) pairs per group, and the largest transform-pass
  // block and shared memory any of its slots needs
  int2* d_items3[kBatchGroups] = {};
  int n_items3[kBatchGroups] = {};
  std::vector<int2> h_items3[kBatchGroups];
  int thr3[kBatchGroups][3] = {}, smem3[kBatchGroups][3] = {};
  std::vector<SlotHost> slots;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_dirty = true;
  int smem_sweep = 0;
  int smem_sweep2 = 0;  // the band kernels of the two-species kinds
  // measured tiles per grid size (index log2 of the longer side; 0 = not measured)
  int tune_band[16] = {}, tune_col[16] = {};
  // queues.  mu guards the queues, outputs, stats, worker_error, stop and the arena's free list
  // (allocated and released by the worker, read by rd_batch_get_stats); never held across a
  // CUDA call that waits on the device.
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::deque<rd_result> done;
  std::map<uint64_t, double*> outputs;  // request id -> caller's host output buffer
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::string worker_error;
  rd_batch_stats stats{};
};

namespace {

rd_status bfail(rd_status s, const std::string& m) {
  rd::set_last_error(m.c_str());
  return s;
}

int key_of(const rd_request& r) {
  if (r.reaction.kind == RD_RX_NONE) return r.op == RD_OP_NEG_BIHARMONIC ? KK_NONE_BIH : KK_NONE_LAP;
  return r.reaction.kind;
}

int group_of(int key) {
  for (int g = 0; g < kBatchGroups; ++g)
    if (kGroupKey[g] == key) return g;
  return -1;
}

void host_tables(int n, bool neumann, double h, std::vector<float>& tw, std::vector<float>& dc, std::vector<float>& mu) {
  const long double pi = 3.141592653589793238462643383279502884L;
  tw.resize(2 * n);
  dc.resize(2 * n);
  mu.resize(n);
  for (int k = 0; k < n; ++k) {
    const long double t = 2.0L * pi * k / n;
    tw[2 * k] = (float)cosl(t);
    tw[2 * k + 1] = (float)(-sinl(t));
    const long double q = pi * k / (2.0L * n);
    dc[2 * k] = (float)cosl(q);
    dc[2 * k + 1] = (float)sinl(q);
    const long double sn = sinl(pi * k / ((neumann ? 2.0L : 1.0L) * n));
    mu[k] = (float)(4.0L / ((long double)h * h) * sn * sn);
  }
}

template <class T, int K>
cudaError_t allow_batch_kernels(int optin) {
  cudaFuncAttributes fa;
  cudaError_t e;
  if ((e = cudaFuncGetAttributes(&fa, k_res_b<T, K>)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_res_b<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncGetAttributes(&fa, k_upd_b<T, K>)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_upd_b<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

template <int K>
void launch_group(rd_batch* b, int g, cudaStream_t s) {
  const int np = b->n_phase[g], nb = b->n_band[g], ncl = b->n_col[g];
  if (np == 0) return;
  const int smem_res = KT<K>::two ? b->smem_sweep2 : b->smem_sweep, smem_col = b->smem_sweep;
  k_axpy_b<<<np, 256, 0, s>>>(b->d_d64, b->d_slots, b->d_phase_items[g]);
  k_step_b<K><<<np, 256, 0, s>>>(b->d_d64, b->d_slots, b->d_phase_items[g]);
  const bool fork = b->n_small[g][0] + b->n_small[g][1] > 0;
  if (fork) {
    // the one-launch inner solves of the small slots, beside the sweeps of the others
    cudaEventRecord(b->ev_fork, s);
    cudaStreamWaitEvent(b->fork_stream, b->ev_fork, 0);
    for (int m = 0; m < 2; ++m)
      launch_small_batch(K, m + 1, b->d_d32, b->d_slots, b->d_small_items[g][m], b->n_small[g][m], b->smem_small[g][m],
                         b->fork_stream);
    cudaEventRecord(b->ev_join, b->fork_stream);
  }
  if (nb) {
    k_res_b<float, K><<<nb, kBatchThreads, smem_res, s>>>(b->d_d32, b->d_slots, b->d_band_items[g]);
    k_col_b<float><<<ncl, kBatchThreads, smem_col, s>>>(b->d_d32, b->d_slots, b->d_col_items[g]);
    k_upd_b<float, K><<<nb, kBatchThreads, smem_res, s>>>(b->d_d32, b->d_slots, b->d_band_items[g]);
  }
  if (fork) cudaStreamWaitEvent(s, b->ev_join, 0);
}

void launch_iteration_all(rd_batch* b, cudaStream_t s) {
  for (int g = 0; g < kBatchGroups; ++g) {
    switch (kGroupKey[g]) {
      case KK_NONE_LAP: launch_group<KK_NONE_LAP>(b, g, s); break;
      case KK_AC: launch_group<KK_AC>(b, g, s); break;
      case KK_CH_IMPL: launch_group<KK_CH_IMPL>(b, g, s); break;
      case KK_CH_SPLIT: launch_group<KK_CH_SPLIT>(b, g, s); break;
      case KK_GS: launch_group<KK_GS>(b, g, s); break;
      case KK_SCHNAK: launch_group<KK_SCHNAK>(b, g, s); break;
      default: launch_group<KK_NONE_BIH>(b, g, s); break;
    }
    if (b->n_items3[g]) {
      Batch3Launch L{b->d_d32, b->d_d64, b->d_slots, b->d_items3[g], b->n_items3[g], {}, {}};
      for (int a = 0; a < 3; ++a) {
        L.thr[a] = b->thr3[g][a];
        L.smem[a] = b->smem3[g][a];
      }
      batch3_launch_group(kGroupKey[g], L, s);
    }
  }
}

// (Re)capture the graph of graph_k iterations over the current work lists.
rd_status rebuild_graph(rd_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(RD_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  for (int k = 0; k < b->opts.graph_k; ++k) launch_iteration_all(b, b->cap_stream);
  cudaError_t el = cudaGetLastError();
  e = cudaStreamEndCapture(b->cap_stream, &b->graph);
  if (el != cudaSuccess || e != cudaSuccess)
    return bfail(RD_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(el != cudaSuccess ? el : e));
  e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
  if (e != cudaSuccess) return bfail(RD_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
  b->graph_dirty = false;
  return RD_OK;
}

// Upload the work lists of all groups from the slot table.
rd_status rebuild_items(rd_batch* b) {
  for (int g = 0; g < kBatchGroups; ++g) {
    b->h_band[g].clear();
    b->h_col[g].clear();
    b->h_phase[g].clear();
    for (int m = 0; m < 2; ++m) {
      b->h_small[g][m].clear();
      b->smem_small[g][m] = 0;
    }
    b->h_items3[g].clear();
    for (int a = 0; a < 3; ++a) b->thr3[g][a] = b->smem3[g][a] = 0;
  }
  for (int s = 0; s < b->max_slots; ++s) {
    const SlotHost& sh = b->slots[s];
    if (!sh.used) continue;
    if (sh.nd3) {
      const Desc& d = sh.d32;
      for (int k = 0; k < d.blk3; ++k) b->h_items3[sh.group].push_back(make_int2(s, k));
      const int n_ax[3] = {d.nx, d.ny, d.nz};
      for (int a = 0; a < 3; ++a) {
        b->thr3[sh.group][a] = std::max(b->thr3[sh.group][a], d.thr3[a]);
        b->smem3[sh.group][a] = std::max(b->smem3[sh.group][a],
                                         lines3_smem_bytes<float>(n_ax[a], d.lw3[a], d.bc == BC_NEUMANN));
      }
      continue;
    }
    for (int band = 0; band < sh.d32.nbands; ++band) b->h_phase[sh.group].push_back(make_int2(s, band));
    if (sh.small) {
      const Desc& d = sh.d32;
      const int m = sh.small - 1;
      b->h_small[sh.group][m].push_back(make_int2(s, 0));
      b->smem_small[sh.group][m] = std::max(
          b->smem_small[sh.group][m], small_smem_of(sh.small, d.nx, d.ny, d.ncomp, sh.key, d.bc == BC_NEUMANN));
      continue;
    }
    for (int band = 0; band < sh.d32.nbands; ++band) b->h_band[sh.group].push_back(make_int2(s, band));
    for (int cb = 0; cb < sh.d32.ncomp * sh.d32.ncolblk; ++cb) b->h_col[sh.group].push_back(make_int2(s, cb));
  }
  for (int g = 0; g < kBatchGroups; ++g) {
    b->n_band[g] = (int)b->h_band[g].size();
    b->n_col[g] = (int)b->h_col[g].size();
    b->n_items3[g] = (int)b->h_items3[g].size();
    b->n_phase[g] = (int)b->h_phase[g].size();
    if (b->n_phase[g]) {
      cudaError_t e = cudaMemcpyAsync(b->d_phase_items[g], b->h_phase[g].data(), b->n_phase[g] * sizeof(int2),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return bfail(RD_ERR_CUDA, cudaGetErrorString(e));
    }
    for (int m = 0; m < 2; ++m) {
      b->n_small[g][m] = (int)b->h_small[g][m].size();
      if (b->n_small[g][m]) {
        cudaError_t e = cudaMemcpyAsync(b->d_small_items[g][m], b->h_small[g][m].data(),
                                        b->n_small[g][m] * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bfail(RD_ERR_CUDA, cudaGetErrorString(e));
      }
    }
    if (b->n_items3[g]) {
      cudaError_t e = cudaMemcpyAsync(b->d_items3[g], b->h_items3[g].data(), b->n_items3[g] * sizeof(int2),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return bfail(RD_ERR_CUDA, cudaGetErrorString(e));
    }
    if (b->n_band[g]) {
      cudaError_t e = cudaMemcpyAsync(b->d_band_items[g], b->h_band[g].data(), b->n_band[g] * sizeof(int2),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return bfail(RD_ERR_CUDA, cudaGetErrorString(e));
    }
    if (b->n_col[g]) {
      cudaError_t e = cudaMemcpyAsync(b->d_col_items[g], b->h_col[g].data(), b->n_col[g] * sizeof(int2),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return bfail(RD_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  b->graph_dirty = true;
  return RD_OK;
}

// Set-up of an admitted 3-D request in slot s (arena block mem): arrays, the FP32 and FP64
// descriptors with the 3-D plan, tables, state and control block.
void admit3(rd_batch* b, Request& q, int s, char* mem, size_t npts, rd_status* err) {
  SlotHost& sh = b->slots[s];
  const rd_request& r = q.req;
  const int nx = r.grid.n[0], ny = r.grid.n[1], nz = r.grid.n[2];
  char* p = mem;
  auto take = [&](size_t n) {
    char* q2 = p;
    p += Arena::up(n);
    return q2;
  };
  double* u = (double*)take(npts * 8);
  double* rhs = (double*)take(npts * 8);
  float* dl = (float*)take(npts * 4);
  float* p0 = (float*)take(npts * 4);
  float* wy = (float*)take(npts * 4);
  float* r32 = (float*)take(npts * 4);
  float* u32 = (float*)take(npts * 4);
  float* tabs = (float*)take((size_t)(nx + ny + nz) * 2 * 8);
  float* mus = (float*)take((size_t)(nx + ny + nz) * 4);
  double* parts = (double*)take((size_t)2 * kBatchMaxBlk3 * 8);
  const double hx = r.grid.length[0] / nx, hy = r.grid.length[1] / ny, hz = r.grid.length[2] / nz;
  Desc d{};
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.ncomp = 1;
  d.lognx = ilog2i(nx);
  d.logny = ilog2i(ny);
  d.lognz = ilog2i(nz);
  d.bc = r.bc;
  d.op = r.op;
  d.kind = r.reaction.kind;
  d.precond = 1;
  d.mode = MODE_PDHG;
  d.hx2 = 1.0 / (hx * hx);
  d.hy2 = 1.0 / (hy * hy);
  d.hz2 = 1.0 / (hz * hz);
  d.dt = r.dt;
  d.a = r.reaction.a;
  d.b = r.reaction.b;
  for (int k = 0; k < 6; ++k) d.p[k] = r.reaction.p[k];
  d.tau_u = r.tau;
  d.tau_p = r.sigma;
  d.omega = b->opts.omega;
  d.batched = 1;
  d.partials = parts;
  for (int c = 0; c < 2; ++c) {
    d.gc1[c] = r.op == RD_OP_LAPLACIAN ? r.reaction.a * r.dt : 0.0;
    d.gc2[c] = r.op == RD_OP_LAPLACIAN ? 0.0 : r.reaction.a * r.dt;
  }
  d.inv_nn = 1.0 / ((double)nx * ny * nz);
  const char* why = nullptr;
  if (!plan3(nx, ny, nz, 1, 4, r.bc == RD_BC_NEUMANN, 226 * 1024, d, &why)) {
    *err = bfail(RD_ERR_UNSUPPORTED, std::string("admission: ") + why);
    return;
  }
  Desc d64 = d, d32 = d;
  d64.dc = 0;
  d64.meas_div_dt = r.tol_kind == RD_TOL_RES_ABS;
  d64.X = u;
  d64.rhs = rhs;
  d64.f32_d = dl;
  d64.f32_p0 = p0;
  d64.f32_r = r32;
  d64.f32_u = u32;
  d32.dc = 1;
  d32.meas_div_dt = 0;
  d32.stall_window = b->opts.dc_stall_window > 0 ? b->opts.dc_stall_window : 8;
  d32.X = dl;
  d32.base = u32;
  d32.rhs = r32;
  d32.P[0] = p0;
  d32.P[1] = p0;
  d32.WY = wy;
  cx<float>* twx = reinterpret_cast<cx<float>*>(tabs);
  cx<float>* dcx = twx + nx;
  cx<float>* twy = dcx + nx;
  cx<float>* dcy = twy + ny;
  cx<float>* twz = dcy + ny;
  cx<float>* dcz = twz + nz;
  d32.twx = twx;
  d32.dcx = dcx;
  d32.twy = twy;
  d32.dcy = dcy;
  d32.twz = twz;
  d32.dcz = dcz;
  d32.mux = mus;
  d32.muy = mus + nx;
  d32.muz = mus + nx + ny;
  sh.d32 = d32;
  sh.d64 = d64;
  sh.nd3 = true;
  std::vector<float> tw, dc, mu, all_t, all_mu;
  const int n_ax[3] = {nx, ny, nz};
  const double h_ax[3] = {hx, hy, hz};
  for (int a = 0; a < 3; ++a) {
    host_tables(n_ax[a], r.bc == RD_BC_NEUMANN, h_ax[a], tw, dc, mu);
    all_t.insert(all_t.end(), tw.begin(), tw.end());
    all_t.insert(all_t.end(), dc.begin(), dc.end());
    all_mu.insert(all_mu.end(), mu.begin(), mu.end());
  }
  Slot ctl{};
  ctl.outer.max_iter = 1 << 30;
  ctl.inner.max_iter = b->opts.max_iter;
  ctl.phase = PH_BEGIN;
  ctl.nsteps = r.nsteps;
  ctl.max_outer = b->opts.dc_max_outer;
  ctl.tol = r.tol;
  ctl.rtol = b->opts.dc_inner_rtol;
  ctl.tol_kind = r.tol_kind;
  cudaStream_t st = b->stream;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tabs, all_t.data(), all_t.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mus, all_mu.data(), all_mu.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, q.u0.data(), npts * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_d32 + s, &sh.d32, sizeof(Desc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_d64 + s, &sh.d64, sizeof(Desc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_slots + s, &ctl, sizeof(Slot), cudaMemcpyHostToDevice, st);
  // the host vectors above are pageable: wait for the copies before they go out of scope
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) *err = bfail(RD_ERR_CUDA, std::string("admission: ") + cudaGetErrorString(e));
}

// Try to admit the request into a free slot.  Returns false when no slot or memory is free.
bool admit(rd_batch* b, Request& q, rd_status* err) {
  *err = RD_OK;
  int s = -1;
  for (int k = 0; k < b->max_slots; ++k)
    if (!b->slots[k].used) {
      s = k;
      break;
    }
  if (s < 0) return false;
  size_t npts = 0;
  const size_t bytes = slot_bytes(q.req, &npts);
  char* mem = nullptr;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    mem = b->arena.alloc(bytes);
  }
  if (!mem) return false;
  SlotHost& sh = b->slots[s];
  sh.used = true;
  sh.id = q.id;
  sh.req = q.req;
  sh.key = key_of(q.req);
  sh.group = group_of(sh.key);
  sh.mem = mem;
  sh.mem_bytes = bytes;
  sh.npts = npts;
  sh.t_submit = q.t_submit;
  sh.t_admit = now_s();
  sh.nd3 = false;
  if (q.req.grid.ndim == 3) {
    admit3(b, q, s, mem, npts, err);
    std::lock_guard<std::mutex> lk(b->mu);
    b->stats.admitted += 1;
    return true;
  }
  const rd_request& r = q.req;
  const int nx = r.grid.n[0], ny = r.grid.n[1], nc = r.reaction.ncomp;
  char* p = mem;
  auto take = [&](size_t n) {
    char* q2 = p;
    p += Arena::up(n);
    return q2;
  };
  double* u = (double*)take(npts * 8);
  double* rhs = (double*)take(npts * 8);
  float* dl = (float*)take(npts * 4);
  float* p0 = (float*)take(npts * 4);
  float* p1 = (float*)take(npts * 4);
  float* wy = (float*)take(npts * 4);
  float* r32 = (float*)take(npts * 4);
  float* u32 = (float*)take(npts * 4);
  float* tabs = (float*)take((size_t)(nx + ny) * 2 * 8);
  float* mus = (float*)take((size_t)(nx + ny) * 4);
  double* parts = (double*)take((size_t)2 * (ny / 2 + 1) * 8);
  const double hx = r.grid.length[0] / nx, hy = r.grid.length[1] / ny;
  // descriptors
  Desc d{};
  d.nx = nx;
  d.ny = ny;
  d.ncomp = nc;
  d.lognx = ilog2i(nx);
  d.logny = ilog2i(ny);
  d.bc = r.bc;
  d.op = r.op;
  d.kind = r.reaction.kind;
  d.precond = 1;
  d.mode = MODE_PDHG;
  // tiles: the measured best for this grid size (opts.autotune), else 4-row bands, 4 columns
  const int lg = ilog2i(std::max(nx, ny));
  d.band_rows = std::min(b->tune_band[lg] ? b->tune_band[lg] : kBatchBandRows, ny);
  d.nbands = (ny + d.band_rows - 1) / d.band_rows;
  d.col_width = std::min(b->tune_col[lg] ? b->tune_col[lg] : kBatchColWidth, nx);
  d.ncolblk = nx / d.col_width;
  d.hx2 = 1.0 / (hx * hx);
  d.hy2 = 1.0 / (hy * hy);
  d.dt = r.dt;
  d.a = r.reaction.a;
  d.b = r.reaction.b;
  for (int k = 0; k < 6; ++k) d.p[k] = r.reaction.p[k];
  d.tau_u = r.tau;
  d.tau_p = r.sigma;
  d.omega = b->opts.omega;
  d.batched = 1;
  d.partials = parts;
  const bool two = r.reaction.kind == RD_RX_GRAY_SCOTT || r.reaction.kind == RD_RX_SCHNAKENBERG;
  for (int c = 0; c < 2; ++c) {
    const double D = two ? r.reaction.p[c] : r.reaction.a;  // two species: each its own diffusivity
    d.gc1[c] = r.op == RD_OP_LAPLACIAN ? D * r.dt : 0.0;
    d.gc2[c] = r.op == RD_OP_LAPLACIAN ? 0.0 : r.reaction.a * r.dt;
  }
  d.inv_nn = 1.0 / ((double)nx * ny);
  Desc d64 = d, d32 = d;
  d64.dc = 0;
  d64.meas_div_dt = r.tol_kind == RD_TOL_RES_ABS;
  d64.X = u;
  d64.rhs = rhs;
  d64.f32_d = dl;
  d64.f32_p0 = p0;
  d64.f32_r = r32;
  d64.f32_u = u32;
  d32.dc = 1;
  d32.meas_div_dt = 0;
  d32.stall_window = b->opts.dc_stall_window > 0 ? b->opts.dc_stall_window : 8;
  d32.X = dl;
  d32.base = u32;
  d32.rhs = r32;
  d32.P[0] = p0;
  d32.P[1] = p1;
  d32.WY = wy;
  cx<float>* twx = reinterpret_cast<cx<float>*>(tabs);
  cx<float>* dcx = twx + nx;
  cx<float>* twy = dcx + nx;
  cx<float>* dcy = twy + ny;
  d32.twx = twx;
  d32.dcx = dcx;
  d32.twy = twy;
  d32.dcy = dcy;
  d32.mux = mus;
  d32.muy = mus + nx;
  sh.d32 = d32;
  sh.d64 = d64;
  // small grids: each inner solve in one launch (one block, or a cluster of eight)
  sh.small = b->opts.small_solve ? small_mode(nx, ny, nc, sh.key, r.bc == RD_BC_NEUMANN, b->smem_usable) : 0;
  // tables, state, control block
  std::vector<float> tw, dc, mu, all_t, all_mu;
  host_tables(nx, r.bc == RD_BC_NEUMANN, hx, tw, dc, mu);
  all_t.insert(all_t.end(), tw.begin(), tw.end());
  all_t.insert(all_t.end(), dc.begin(), dc.end());
  all_mu = mu;
  host_tables(ny, r.bc == RD_BC_NEUMANN, hy, tw, dc, mu);
  all_t.insert(all_t.end(), tw.begin(), tw.end());
  all_t.insert(all_t.end(), dc.begin(), dc.end());
  all_mu.insert(all_mu.end(), mu.begin(), mu.end());
  Slot ctl{};
  ctl.outer.max_iter = 1 << 30;
  ctl.inner.max_iter = b->opts.max_iter;
  ctl.phase = PH_BEGIN;
  ctl.nsteps = r.nsteps;
  ctl.max_outer = b->opts.dc_max_outer;
  ctl.tol = r.tol;
  ctl.rtol = b->opts.dc_inner_rtol;
  ctl.tol_kind = r.tol_kind;
  cudaStream_t st = b->stream;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tabs, all_t.data(), all_t.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mus, all_mu.data(), all_mu.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, q.u0.data(), npts * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_d32 + s, &sh.d32, sizeof(Desc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_d64 + s, &sh.d64, sizeof(Desc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_slots + s, &ctl, sizeof(Slot), cudaMemcpyHostToDevice, st);
  // the host vectors above are pageable: wait for the copies before they go out of scope
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) *err = bfail(RD_ERR_CUDA, std::string("admission: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(b->mu);
  b->stats.admitted += 1;
  return true;
}

void retire(rd_batch* b, int s, const Slot& ctl) {
  SlotHost& sh = b->slots[s];
  rd_result res{};
  res.id = sh.id;
  res.tag = sh.req.tag;
  res.status = ctl.phase == PH_DONE ? RD_OK
               : (ctl.outer.status == ST_DIVERGED || ctl.inner.status == ST_DIVERGED ? RD_ERR_DIVERGED
                                                                                   : RD_ERR_NOT_CONVERGED);
  res.steps = ctl.steps_done;
  res.iterations = ctl.inner_total;
  res.outer_rounds = ctl.outer_total;
  res.residual = ctl.outer.r;
  double* out = nullptr;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->outputs.find(sh.id);
    if (it != b->outputs.end()) {
      out = it->second;
      b->outputs.erase(it);
    }
  }
  // the result copy and the wait for it: a failure of either reports the request as RD_ERR_CUDA
  // (its host output would hold stale data) and is kept as the worker's error
  cudaError_t ce = cudaSuccess;
  if (out) ce = cudaMemcpyAsync(out, sh.d64.X, sh.npts * 8, cudaMemcpyDeviceToHost, b->stream);
  const cudaError_t se = cudaStreamSynchronize(b->stream);
  if (ce == cudaSuccess) ce = se;
  std::string copy_error;
  if (ce != cudaSuccess) {
    res.status = RD_ERR_CUDA;
    copy_error = std::string("result copy of request ") + std::to_string(sh.id) + ": " + cudaGetErrorString(ce);
  }
  res.t_submit = sh.t_submit;
  res.t_admit = sh.t_admit;
  res.t_done = now_s();
  char* mem = sh.mem;
  const size_t mem_bytes = sh.mem_bytes;
  Slot idle{};
  cudaMemcpyAsync(b->d_slots + s, &idle, sizeof(Slot), cudaMemcpyHostToDevice, b->stream);
  sh = SlotHost{};
  std::lock_guard<std::mutex> lk(b->mu);
  b->arena.release(mem, mem_bytes);
  b->stats.completed += 1;
  if (!copy_error.empty()) b->worker_error = copy_error;
  b->done.push_back(res);
  b->cv.notify_all();
}

// opts.autotune: for each square grid size the arena can hold, admit one scratch Allen-Cahn slot
// whose inner solve never stops, time graph-free launches of its three sweep kernels over 8
// iterations (best of three) for band rows {2, 4} x column widths {2, 4}, and keep the fastest
// per size; admission then takes the measured tiles.  Every candidate fits the launches' shared
// memory (sized for 4-row bands and 4 columns).
rd_status tune_batch_tiles(rd_batch* b) {
  cudaStream_t st = b->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(RD_ERR_CUDA, "tile tuning: events");
  const int g = group_of(KK_AC);
  rd_status res = RD_OK;
  for (int lg = 4; lg <= ilog2i(kBatchMaxSide) && res == RD_OK; ++lg) {
    const int n = 1 << lg;
    Request q;
    q.req.grid.ndim = 2;
    q.req.grid.n[0] = q.req.grid.n[1] = n;
    q.req.grid.length[0] = q.req.grid.length[1] = 1.0;
    q.req.bc = RD_BC_PERIODIC;
    q.req.op = RD_OP_LAPLACIAN;
    q.req.reaction.kind = RD_RX_ALLEN_CAHN;
    q.req.reaction.ncomp = 1;
    q.req.reaction.a = 0.05;
    q.req.reaction.b = 20.0;
    q.req.dt = 2e-3;
    q.req.tau = q.req.sigma = 1.0;
    q.req.tol = 1e-11;
    q.req.tol_kind = RD_TOL_F_REL;
    q.req.nsteps = 1;
    q.u0.assign((size_t)n * n, 0.0);
    rd_status err = RD_OK;
    const int small_opt = b->opts.small_solve;
    b->opts.small_solve = 0;  // time the sweeps, not the one-launch solve
    const bool ok = admit(b, q, &err);
    b->opts.small_solve = small_opt;
    if (!ok) break;  // the arena holds no larger grid
    int s = -1;
    for (int k = 0; k < b->max_slots; ++k)
      if (b->slots[k].used) s = k;
    SlotHost& sh = b->slots[s];
    const size_t npts = sh.npts;
    // base state and right-hand side nonzero, d = P = 0, an inner solve that never stops
    cudaMemsetAsync(const_cast<void*>(sh.d32.rhs), 0x3f, npts * 4, st);
    cudaMemsetAsync(const_cast<void*>(sh.d32.base), 0x3f, npts * 4, st);
    cudaMemsetAsync(sh.d32.X, 0, npts * 4, st);
    cudaMemsetAsync(sh.d32.P[0], 0, npts * 4, st);
    cudaMemsetAsync(sh.d32.P[1], 0, npts * 4, st);
    float best = 1e30f;
    int bb = kBatchBandRows, bc = kBatchColWidth;
    for (int band : {2, 4})
      for (int cw : {2, 4}) {
        if (band > n || cw > n) continue;
        Desc d32 = sh.d32, d64 = sh.d64;
        d32.band_rows = d64.band_rows = band;
        d32.nbands = d64.nbands = (n + band - 1) / band;
        d32.col_width = d64.col_width = cw;
        d32.ncolblk = d64.ncolblk = n / cw;
        std::vector<int2> bands, cols;
        for (int k = 0; k < d32.nbands; ++k) bands.push_back(make_int2(s, k));
        for (int k = 0; k < d32.ncolblk; ++k) cols.push_back(make_int2(s, k));
        Slot ctl{};
        ctl.phase = PH_INNER;
        ctl.inner.status = ST_ACTIVE;
        ctl.inner.max_iter = 1 << 30;
        ctl.inner.thresh = 0.0;
        ctl.inner.stall_mul = 1 << 20;
        cudaMemcpyAsync(b->d_d32 + s, &d32, sizeof(Desc), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->d_d64 + s, &d64, sizeof(Desc), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->d_slots + s, &ctl, sizeof(Slot), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->d_band_items[g], bands.data(), bands.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->d_col_items[g], cols.data(), cols.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
        float t_best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, st);
          for (int it = 0; it < 8; ++it) {
            k_res_b<float, KK_AC><<<(int)bands.size(), kBatchThreads, b->smem_sweep, st>>>(b->d_d32, b->d_slots, b->d_band_items[g]);
            k_col_b<float><<<(int)cols.size(), kBatchThreads, b->smem_sweep, st>>>(b->d_d32, b->d_slots, b->d_col_items[g]);
            k_upd_b<float, KK_AC><<<(int)bands.size(), kBatchThreads, b->smem_sweep, st>>>(b->d_d32, b->d_slots, b->d_band_items[g]);
          }
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            res = bfail(RD_ERR_CUDA, std::string("tile tuning: ") + cudaGetErrorString(cudaGetLastError()));
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          t_best = std::min(t_best, ms);
        }
        if (res != RD_OK) break;
        if (t_best < best) {
          best = t_best;
          bb = band;
          bc = cw;
        }
      }
    b->tune_band[lg] = bb;
    b->tune_col[lg] = bc;
    // release the scratch slot
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->arena.release(sh.mem, sh.mem_bytes);
      b->stats.admitted -= 1;
    }
    Slot idle{};
    cudaMemcpyAsync(b->d_slots + s, &idle, sizeof(Slot), cudaMemcpyHostToDevice, st);
    sh = SlotHost{};
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return res;
}

void worker_loop(rd_batch* b) {
  cudaStream_t st = b->stream;
  while (true) {
    // admit what fits
    bool changed = false;
    {
      std::unique_lock<std::mutex> lk(b->mu);
      int active = 0;
      for (const SlotHost& sh : b->slots) active += sh.used;
      if (active == 0)
        b->cv.wait(lk, [&] { return b->stop || !b->queue.empty(); });
      if (b->stop) return;  // destroy: running slots are abandoned
      while (!b->queue.empty()) {
        Request q = std::move(b->queue.front());
        b->queue.pop_front();
        lk.unlock();
        rd_status err;
        const bool ok = admit(b, q, &err);
        lk.lock();
        if (!ok) {
          b->queue.push_front(std::move(q));
          break;
        }
        if (err != RD_OK) b->worker_error = rd_last_error();
        changed = true;
      }
    }
    if (changed && rebuild_items(b) != RD_OK) b->worker_error = rd_last_error();
    int active = 0;
    for (const SlotHost& sh : b->slots) active += sh.used;
    if (active == 0) {
      std::lock_guard<std::mutex> lk(b->mu);
      if (b->stop && b->queue.empty()) return;
      continue;
    }
    if (b->graph_dirty && rebuild_graph(b) != RD_OK) {
      b->worker_error = rd_last_error();
      std::lock_guard<std::mutex> lk(b->mu);
      b->stop = true;
      b->cv.notify_all();
      return;
    }
    cudaGraphLaunch(b->gexec, st);
    cudaMemcpyAsync(b->h_slots, b->d_slots, sizeof(Slot) * b->max_slots, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      b->worker_error = std::string("batch graph: ") + cudaGetErrorString(cudaGetLastError());
      std::lock_guard<std::mutex> lk(b->mu);
      b->stop = true;
      b->cv.notify_all();
      return;
    }
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->stats.graph_launches += 1;
    }
    bool retired = false;
    for (int s = 0; s < b->max_slots; ++s) {
      if (!b->slots[s].used) continue;
      const Slot ctl = b->h_slots[s];
      if (ctl.phase == PH_DONE || ctl.phase == PH_FAILED) {
        retire(b, s, ctl);
        retired = true;
      }
    }
    if (retired) rebuild_items(b);
  }
}

}  // namespace

extern "C" {

rd_status rd_batch_create(rd_batch** out, size_t hbm_budget_bytes, int max_slots, const rd_opts* opts,
                          void* cuda_stream) {
  if (!out) return bfail(RD_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 4096) return bfail(RD_ERR_INVALID_ARG, "max_slots must be in [1, 4096]");
  if (hbm_budget_bytes < (1u << 20)) return bfail(RD_ERR_INVALID_ARG, "HBM budget below 1 MiB");
  rd_batch* b = new (std::nothrow) rd_batch();
  if (!b) return bfail(RD_ERR_OOM, "host allocation failed");
  if (opts) b->opts = *opts; else rd_opts_default(&b->opts);
  if (b->opts.graph_k < 1) b->opts.graph_k = 8;
  b->max_slots = max_slots;
  b->budget = hbm_budget_bytes;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->slots.assign(max_slots, SlotHost{});
  auto cleanup = [&](rd_status s) {
    rd_batch_destroy(b);
    return s;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->fork_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess)
    return cleanup(bfail(RD_ERR_CUDA, cudaGetErrorString(e)));
  if ((e = cudaMalloc(&b->arena_mem, hbm_budget_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(bfail(RD_ERR_OOM, std::string("arena: ") + cudaGetErrorString(e)));
  }
  b->arena.init(b->arena_mem, hbm_budget_bytes);
  const int max_items = max_slots * (kBatchMaxSide / 2);
  if ((e = cudaMalloc(&b->d_d32, sizeof(Desc) * max_slots)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_d64, sizeof(Desc) * max_slots)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_slots, sizeof(Slot) * max_slots)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_slots, sizeof(Slot) * max_slots)) != cudaSuccess)
    return cleanup(bfail(RD_ERR_OOM, cudaGetErrorString(e)));
  for (int g = 0; g < kBatchGroups; ++g) {
    if ((e = cudaMalloc(&b->d_band_items[g], sizeof(int2) * max_items)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_phase_items[g], sizeof(int2) * max_items)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_small_items[g][0], sizeof(int2) * max_slots)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_small_items[g][1], sizeof(int2) * max_slots)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_col_items[g], sizeof(int2) * max_items)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_items3[g], sizeof(int2) * max_slots * kBatchMaxBlk3)) != cudaSuccess)
      return cleanup(bfail(RD_ERR_OOM, cudaGetErrorString(e)));
  }
  cudaMemset(b->d_slots, 0, sizeof(Slot) * max_slots);
  // shared memory of the batched sweeps: the largest grid the batch accepts
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int tabs = table_bytes<float>(kBatchMaxSide, true, true);
  b->smem_sweep = std::max(res_smem_bytes<float>(1, kBatchBandRows, 2, kBatchMaxSide, 1, 0, tabs),
                           std::max(lines_smem_bytes<float>((kBatchBandRows + 4) / 2, kBatchMaxSide, 0, tabs),
                                    lines_smem_bytes<float>(kBatchColWidth / 2, kBatchMaxSide, 0, tabs)));
  if ((e = batch3_allow(optin)) != cudaSuccess || (e = allow_small(optin)) != cudaSuccess)
    return cleanup(bfail(RD_ERR_CUDA, cudaGetErrorString(e)));
  b->smem_usable = optin - 1024;
  b->smem_sweep2 = std::max(res_smem_bytes<float>(2, kBatchBandRows, 1, kBatchMaxSide, 0, 0, tabs),
                            lines_smem_bytes<float>(2 * ((kBatchBandRows + 2) / 2), kBatchMaxSide, 0, tabs));
  if ((e = allow_batch_kernels<float, KK_GS>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_SCHNAK>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_NONE_LAP>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_AC>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_CH_IMPL>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_CH_SPLIT>(optin)) != cudaSuccess ||
      (e = allow_batch_kernels<float, KK_NONE_BIH>(optin)) != cudaSuccess)
    return cleanup(bfail(RD_ERR_CUDA, cudaGetErrorString(e)));
  {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_col_b<float>);
    cudaFuncSetAttribute(k_col_b<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(bfail(RD_ERR_CUDA, cudaGetErrorString(e)));
  if (b->opts.autotune) {
    const rd_status ts = tune_batch_tiles(b);
    if (ts != RD_OK) return cleanup(ts);
  }
  b->worker = std::thread(worker_loop, b);
  *out = b;
  return RD_OK;
}

rd_status rd_batch_submit(rd_batch* b, const rd_request* req, double* u_out_host, uint64_t* id) {
  if (!b || !req || !req->u0_host) return bfail(RD_ERR_INVALID_ARG, "NULL batch, request or u0");
  const rd_request& r = *req;
  if (r.grid.ndim != 2 && r.grid.ndim != 3) return bfail(RD_ERR_UNSUPPORTED, "batch: 2-D and 3-D grids only");
  for (int k = 0; k < r.grid.ndim; ++k) {
    const int n = r.grid.n[k];
    if (r.grid.ndim == 2 && (n < 4 || n > kBatchMaxSide || (n & (n - 1))))
      return bfail(RD_ERR_UNSUPPORTED, "batch: sides must be powers of two in [4, 1024]");
    if (r.grid.ndim == 3 && (n < 4 || n > kBatchMaxSide3 || (n & (n - 1))))
      return bfail(RD_ERR_UNSUPPORTED, "batch: 3-D sides must be powers of two in [4, 512]");
    if (!(r.grid.length[k] > 0)) return bfail(RD_ERR_INVALID_ARG, "lengths must be > 0");
  }
  if (r.bc != RD_BC_PERIODIC && r.bc != RD_BC_NEUMANN) return bfail(RD_ERR_INVALID_ARG, "bad boundary condition");
  if (r.reaction.kind == RD_RX_FCH || r.op == RD_OP_FUNCTIONALIZED)
    return bfail(RD_ERR_UNSUPPORTED, "batch: the sixth-order equation is not batched");
  const bool two = r.reaction.kind == RD_RX_GRAY_SCOTT || r.reaction.kind == RD_RX_SCHNAKENBERG;
  if (group_of(key_of(r)) < 0) return bfail(RD_ERR_UNSUPPORTED, "batch: kind not served");
  if (r.reaction.ncomp != (two ? 2 : 1)) return bfail(RD_ERR_INVALID_ARG, "ncomp does not match the reaction kind");
  if (two && r.grid.ndim == 3) return bfail(RD_ERR_UNSUPPORTED, "batch: 3-D grids are served for the scalar kinds");
  if (two && r.op != RD_OP_LAPLACIAN) return bfail(RD_ERR_INVALID_ARG, "two species need RD_OP_LAPLACIAN");
  if (r.op != RD_OP_LAPLACIAN && r.op != RD_OP_NEG_BIHARMONIC) return bfail(RD_ERR_INVALID_ARG, "bad operator");
  if (r.reaction.kind == RD_RX_ALLEN_CAHN && r.op != RD_OP_LAPLACIAN)
    return bfail(RD_ERR_INVALID_ARG, "Allen-Cahn needs RD_OP_LAPLACIAN");
  if ((r.reaction.kind == RD_RX_CH_IMPLICIT || r.reaction.kind == RD_RX_CH_SPLIT) && r.op != RD_OP_NEG_BIHARMONIC)
    return bfail(RD_ERR_INVALID_ARG, "Cahn-Hilliard needs RD_OP_NEG_BIHARMONIC");
  if (!(r.reaction.a >= 0) || !(r.reaction.b >= 0)) return bfail(RD_ERR_INVALID_ARG, "a and b must be >= 0");
  if (r.tol_kind != RD_TOL_RES_ABS && r.tol_kind != RD_TOL_F_REL) return bfail(RD_ERR_INVALID_ARG, "bad tol_kind");
  if (!(r.dt > 0) || !(r.tau > 0) || !(r.sigma > 0)) return bfail(RD_ERR_INVALID_ARG, "dt, tau, sigma must be > 0");
  if (r.nsteps < 1) return bfail(RD_ERR_INVALID_ARG, "nsteps must be >= 1");
  size_t npts = 0;
  if (slot_bytes(r, &npts) > b->budget) return bfail(RD_ERR_BUSY, "request larger than the whole HBM budget");
  Request q;
  q.req = r;
  q.u0.assign(r.u0_host, r.u0_host + npts);
  q.t_submit = now_s();
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->stop) return bfail(RD_ERR_CUDA, "batch worker stopped: " + b->worker_error);
  q.id = b->next_id++;
  q.req.u0_host = nullptr;
  if (u_out_host) b->outputs[q.id] = u_out_host;
  if (id) *id = q.id;
  b->queue.push_back(std::move(q));
  b->stats.submitted += 1;
  b->cv.notify_all();
  return RD_OK;
}

rd_status rd_batch_poll(rd_batch* b, rd_result* done, int cap, int* n_done, double timeout_s) {
  if (!b || !n_done || (cap > 0 && !done)) return bfail(RD_ERR_INVALID_ARG, "NULL argument");
  *n_done = 0;
  std::unique_lock<std::mutex> lk(b->mu);
  if (timeout_s > 0 && b->done.empty() && !b->stop)
    b->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return !b->done.empty() || b->stop; });
  while (*n_done < cap && !b->done.empty()) {
    done[(*n_done)++] = b->done.front();
    b->done.pop_front();
  }
  if (b->stop && !b->worker_error.empty()) return bfail(RD_ERR_CUDA, "batch worker stopped: " + b->worker_error);
  return RD_OK;
}

rd_status rd_batch_get_stats(rd_batch* b, rd_batch_stats* out) {
  if (!b || !out) return bfail(RD_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  *out = b->stats;
  out->queued = (long long)b->queue.size();
  size_t fr = 0;
  for (auto& kv : b->arena.free_) fr += kv.second;
  out->arena_free_bytes = (long long)fr;
  return RD_OK;
}

void rd_batch_destroy(rd_batch* b) {
  if (!b) return;
  if (b->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->stop = true;
      b->queue.clear();
      b->cv.notify_all();
    }
    b->worker.join();
  }
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int g = 0; g < kBatchGroups; ++g) {
    if (b->d_band_items[g]) cudaFree(b->d_band_items[g]);
    if (b->d_col_items[g]) cudaFree(b->d_col_items[g]);
    if (b->d_items3[g]) cudaFree(b->d_items3[g]);
    if (b->d_phase_items[g]) cudaFree(b->d_phase_items[g]);
    for (int m = 0; m < 2; ++m)
      if (b->d_small_items[g][m]) cudaFree(b->d_small_items[g][m]);
  }
  if (b->d_d32) cudaFree(b->d_d32);
  if (b->d_d64) cudaFree(b->d_d64);
  if (b->d_slots) cudaFree(b->d_slots);
  if (b->h_slots) cudaFreeHost(b->h_slots);
  if (b->arena_mem) cudaFree(b->arena_mem);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->fork_stream) cudaStreamDestroy(b->fork_stream);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  delete b;
}

}  // extern "C"
