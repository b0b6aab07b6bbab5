// Allocation-free preconditioner solve Y = G^{-1} W.
//
// Some callers cannot allocate device memory at the moment they need this operation: code that
// runs under a fixed, pre-reserved memory budget (an embedding application that owns every byte
// of the device), code paths where the implicit device synchronisation of cudaMalloc/cudaFree is
// not acceptable (a latency-critical loop sharing the GPU with other work), or callers that hold
// no solver handle at all and only want this one operator.  For them this file offers a variant
// of the preconditioner-solve kernels whose scratch space (the intermediate transform array, the
// twiddle tables and the Laplacian eigenvalue tables) lives in one statically sized device array instead of
// buffers obtained from cudaMalloc.  The caller still passes the input W and the output Y.
//
// Limits and sharing rules:
//   * the scratch array is kNoAllocScratchBytes (2.5 MiB) on every device that loads the
//     library, held until the process exits; grids with ncomp*nx*ny > kNoAllocMaxPoints
//     (131072 points) or a side above 2048 are rejected with RD_ERR_UNSUPPORTED;
//   * every call on a device uses the same array, and the array keeps whatever the last call
//     left in it: this code rewrites every table and every transform entry it reads before
//     reading it, so nothing has to start at zero;
//   * two calls whose work overlaps on the GPU (e.g. issued on two streams without ordering)
//     race on the array and produce wrong results: order them on one stream or synchronise;
//   * the first call on a device looks up the array's device address (cudaGetSymbolAddress)
//     with that device current and raises the kernels' shared-memory limit; make that first
//     call before any stream capture is begun on the calling thread.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/rd_pdhg.h"
#include "rd_device.cuh"
#include "rd_launch.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 2621440;  // 2.5 MiB
constexpr size_t kNoAllocMaxPoints = 131072;      // ncomp * nx * ny
constexpr int kNoAllocMaxSide = 2048;             // keeps every block of the solve under 227 KB of shared memory
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_rd_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

rd_status nofail(rd_status s, const std::string& m) {
  rd::set_last_error(m.c_str());  // read back with rd_last_error()
  return s;
}

// Twiddles exp(-2 pi i k / n) and (cos, sin)(pi k / (2n)) for one axis, from sincospi.
__global__ void k_noalloc_twiddles(rd::cx<double>* tw, rd::cx<double>* dc, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * k / n, &s, &c);
    tw[k] = rd::cx<double>{c, -s};
    sincospi(0.5 * k / n, &s, &c);
    dc[k] = rd::cx<double>{c, s};
  }
}

// Eigenvalues of -Lap along one axis, mu(k) = 4/h^2 sin^2(pi k / (d n)), d = 1 periodic,
// 2 Neumann (the preconditioner symbol is built from mu_x(kx) + mu_y(ky) inside the kernels).
__global__ void k_noalloc_mu(double* mu, int n, int neumann, double h) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double sn = sinpi(k / ((neumann ? 2.0 : 1.0) * n));
    mu[k] = 4.0 / (h * h) * sn * sn;
  }
}

int ilog2n(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Device address of the scratch array on the current device (looked up once per device).
rd_status scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nofail(RD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nofail(RD_ERR_UNSUPPORTED, "device index beyond the set-up table");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rd_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return nofail(RD_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    int usable = 0;
    e = rd::set_kernel_smem_limits<double>(&usable);
    if (e != cudaSuccess) return nofail(RD_ERR_CUDA, std::string("shared-memory limits: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RD_OK;
}

}  // namespace

extern "C" RD_API rd_status rd_apply_precond_static(const rd_grid* grid, rd_bc bc, rd_operator op,
                                                    const rd_reaction* reaction, double dt, const double* w,
                                                    double* y, void* cuda_stream) {
  if (!grid || !reaction || !w || !y) return nofail(RD_ERR_INVALID_ARG, "NULL argument");
  if (grid->ndim != 2) return nofail(RD_ERR_UNSUPPORTED, "only 2-D grids");
  const int nx = grid->n[0], ny = grid->n[1];
  for (int k = 0; k < 2; ++k) {
    const int n = grid->n[k];
    if (n < 2 || (n & (n - 1)) != 0) return nofail(RD_ERR_UNSUPPORTED, "grid sides must be powers of two >= 2");
    if (n > kNoAllocMaxSide) return nofail(RD_ERR_UNSUPPORTED, "grid side above 2048 for the allocation-free solve");
    if (!(grid->length[k] > 0)) return nofail(RD_ERR_INVALID_ARG, "lengths must be > 0");
  }
  if (bc != RD_BC_PERIODIC && bc != RD_BC_NEUMANN) return nofail(RD_ERR_INVALID_ARG, "bad boundary condition");
  if (op != RD_OP_LAPLACIAN && op != RD_OP_NEG_BIHARMONIC) return nofail(RD_ERR_INVALID_ARG, "bad operator");
  if (reaction->kind == RD_RX_FCH) return nofail(RD_ERR_UNSUPPORTED, "the sixth-order equation has no static solve");
  if (!(dt > 0)) return nofail(RD_ERR_INVALID_ARG, "dt must be > 0");
  const bool two = reaction->kind == RD_RX_GRAY_SCOTT || reaction->kind == RD_RX_SCHNAKENBERG;
  const int nc = two ? 2 : 1;
  if (reaction->ncomp != nc) return nofail(RD_ERR_INVALID_ARG, "ncomp does not match the reaction kind");
  const size_t npts = (size_t)nc * nx * ny;
  if (npts > kNoAllocMaxPoints)
    return nofail(RD_ERR_UNSUPPORTED, "grid larger than the allocation-free limit of 131072 points (ncomp*nx*ny)");

  // carve the scratch array: transform buffer, twiddle tables, eigenvalue tables
  const size_t wy_bytes = npts * sizeof(double);
  const size_t tw_bytes = ((size_t)2 * nx + 2 * ny) * sizeof(rd::cx<double>);
  const size_t mu_bytes = ((size_t)nx + ny) * sizeof(double);
  if (wy_bytes + tw_bytes + mu_bytes > kNoAllocScratchBytes)
    return nofail(RD_ERR_UNSUPPORTED, "grid does not fit the allocation-free scratch array");

  void* base = nullptr;
  rd_status st = scratch_on_current_device(&base);
  if (st != RD_OK) return st;
  unsigned char* p = static_cast<unsigned char*>(base);
  double* wy = reinterpret_cast<double*>(p);
  rd::cx<double>* twx = reinterpret_cast<rd::cx<double>*>(p + wy_bytes);
  rd::cx<double>* dcx = twx + nx;
  rd::cx<double>* twy = dcx + nx;
  rd::cx<double>* dcy = twy + ny;
  double* mux = reinterpret_cast<double*>(dcy + ny);
  double* muy = mux + nx;

  const double hx = grid->length[0] / nx, hy = grid->length[1] / ny;
  const double d0 = two ? reaction->p[0] : reaction->a;
  const double d1 = two ? reaction->p[1] : reaction->a;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // launch shape: two-row bands, two-column blocks (small grids; every block stays < 227 KB)
  rd::Desc d{};
  d.nx = nx;
  d.ny = ny;
  d.ncomp = nc;
  d.lognx = ilog2n(nx);
  d.logny = ilog2n(ny);
  d.bc = bc;
  d.op = op;
  d.kind = reaction->kind;
  d.precond = 1;
  d.mode = rd::MODE_PRECOND_ONLY;
  d.band_rows = 2;
  d.nbands = ny / 2;
  d.col_width = 2;
  d.ncolblk = nx / 2;
  d.hx2 = 1.0 / (hx * hx);
  d.hy2 = 1.0 / (hy * hy);
  d.dt = dt;
  d.X = y;
  d.WY = wy;
  d.mux = mux;
  d.muy = muy;
  for (int c = 0; c < 2; ++c) {
    const double D = c == 0 ? d0 : d1;
    d.gc1[c] = op == RD_OP_LAPLACIAN ? D * dt : 0.0;
    d.gc2[c] = op == RD_OP_LAPLACIAN ? 0.0 : reaction->a * dt;
  }
  d.inv_nn = 1.0 / ((double)nx * (double)ny);
  d.twx = twx;
  d.twy = twy;
  d.dcx = dcx;
  d.dcy = dcy;

  auto threads = [](int lines, int n) {
    int t = (lines * n + 7) / 8;
    if (t < n / 8) t = n / 8;
    t = (t + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > 512) t = 512;
    return t;
  };
  rd::LaunchCfg cfg{};
  cfg.grid_bands = d.nbands;
  cfg.grid_cols = nc * d.ncolblk;
  cfg.thr_res = threads(nc, nx);
  cfg.thr_upd = threads(nc, nx);
  cfg.thr_col = threads(1, ny);
  cfg.smem_res = rd::res_smem_bytes<double>(nc, 2, 0, nx, 0, 0, 0);
  cfg.smem_upd = rd::lines_smem_bytes<double>(nc, nx, 0, 0);
  cfg.smem_col = rd::lines_smem_bytes<double>(1, ny, 0, 0);
  cfg.transform = 1;

  cudaError_t e;
  k_noalloc_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(twx, dcx, nx);
  k_noalloc_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(twy, dcy, ny);
  k_noalloc_mu<<<(nx + 255) / 256, 256, 0, s>>>(mux, nx, bc == RD_BC_NEUMANN, hx);
  k_noalloc_mu<<<(ny + 255) / 256, 256, 0, s>>>(muy, ny, bc == RD_BC_NEUMANN, hy);
  if ((e = cudaGetLastError()) != cudaSuccess) return nofail(RD_ERR_CUDA, cudaGetErrorString(e));
  if (y != w) {
    e = cudaMemcpyAsync(y, w, npts * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return nofail(RD_ERR_CUDA, std::string("copy w -> y: ") + cudaGetErrorString(e));
  }
  e = rd::launch_iteration<double>(d, nullptr, cfg, s, nullptr);
  if (e != cudaSuccess) return nofail(RD_ERR_CUDA, std::string("preconditioner kernels: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nofail(RD_ERR_CUDA, std::string("stream synchronise: ") + cudaGetErrorString(e));
  return RD_OK;
}
