// Plain FP64 C++ oracle of the G-prox PDHG solve of one implicit reaction-diffusion step
// (arxiv 2305.03945).  TEST INFRASTRUCTURE ONLY: it is built and called by the tests, by
// __graft_entry__.smoke() and by the CPU-baseline / reference legs of bench.py, never by the
// product library, and it shares no code, header or table with the CUDA path.
//
// It restates, in the paper's order and notation:
//   * the five-point Laplacian with the periodic wrap (block-circulant Lap^P, Section 2.1) or the
//     half-cell mirror ghost U_{-1} = U_0 (Lap^N, Remark 1); Lap^2 as Lap applied twice;
//   * the residual map F of each equation (eq. F(U) rd equation for Allen-Cahn, eq. F(U) CH for
//     Cahn-Hilliard with the sign reading lambda = -a, the convex-concave split, Section 3.3 for
//     the sixth-order equation, Section 3.4.1 for two species) and its adjoint Jacobian applied to
//     the extrapolated dual (the U-updates of the G-prox dynamics);
//   * the preconditioner G = A_lin^2 inverted in the Fourier basis (periodic) or the orthonormal
//     DCT-II basis (Neumann) (Section 2.1 "Choosing the matrix G", "Application of FFT",
//     Remark 1);
//   * the G-prox PDHG iteration (eqs. G-prox linearized pdhg dynamic 1-3) from U_0 = U^k, P_0 = 0,
//     stopped at the first U_n whose measure ||Res(U_n)||_2 is <= delta (Section 2.1, stopping
//     criterion), inside Algorithm 1's time loop.
// The transforms are its own: an iterative radix-2 complex FFT (bit reversal, then butterflies
// whose twiddles are cos/sin of 2 pi j / len), and the DCT-II / DCT-III through a 2N-point FFT of
// the even extension [x_0 .. x_{N-1}, x_{N-1} .. x_0] -- not the N-point reordering the GPU uses.
// Loops over rows and columns may run under OpenMP (timing only); every reduction sums per-row
// partials in row order, so results do not depend on the thread count.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

enum { BC_PERIODIC = 0, BC_NEUMANN = 1 };
enum { OP_LAPLACIAN = 0, OP_NEG_BIHARMONIC = 1, OP_FUNCTIONALIZED = 2 };
enum { K_NONE = 0, K_AC = 1, K_CH_IMPLICIT = 2, K_CH_SPLIT = 3, K_GRAY_SCOTT = 4, K_SCHNAKENBERG = 5, K_FCH = 6 };
enum { PC_NONE = 0, PC_LINEAR = 1, PC_STABILIZED = 2 };
enum { TOL_RES_ABS = 0, TOL_F_REL = 1 };
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_DIVERGED = 2 };
constexpr double kDivergeFactor = 1e8;

}  // namespace

extern "C" {

// Parameters of one implicit step (the same fields as the Python oracle's Problem record).
typedef struct {
  int nx, ny;          // grid points along x (contiguous) and y
  double lx, ly;       // side lengths; h_x = lx / nx, h_y = ly / ny
  int bc, op, kind;    // boundary condition, linear operator, reaction kind (enums above)
  double dt, a, b;     // h_t and the diffusion / reaction scales
  double p[6];         // Gray-Scott (Du, Dv, F, k); Schnakenberg (D1, D2, kappa, a, b)
  double tau_u, tau_p, omega;
  int precond;         // PC_NONE (G = I), PC_LINEAR (G = A_lin^2) or PC_STABILIZED (A_lin with
                       // the nonlinear factor replaced by the constant `shift`, squared)
  double tol;
  int tol_kind;
  int max_iter;
  int nz;              // points along z of a 3-D grid (1: a 2-D grid)
  double lz;           // side length along z; h_z = lz / nz
  double shift;        // PC_STABILIZED: the constant in place of the nonlinear factor
} rdo_problem;

}  // extern "C"

namespace {

int ncomp_of(const rdo_problem& pb) { return (pb.kind == K_GRAY_SCOTT || pb.kind == K_SCHNAKENBERG) ? 2 : 1; }

// ------------------------------------------------------------------------------------------
// grid operators
// ------------------------------------------------------------------------------------------

// index i + s along an axis of n points with the boundary rule of bc (|s| <= 1)
inline int nb(int i, int s, int n, int bc) {
  int j = i + s;
  if (j >= 0 && j < n) return j;
  if (bc == BC_PERIODIC) return j < 0 ? j + n : j - n;
  return j < 0 ? 0 : n - 1;  // half-cell mirror: U_{-1} = U_0, U_n = U_{n-1}
}

int nzof(const rdo_problem& pb) { return pb.nz > 1 ? pb.nz : 1; }
size_t npts_of(const rdo_problem& pb) { return (size_t)pb.nx * pb.ny * nzof(pb); }

// out = Lap x on one component (nz * ny * nx values): the five-point Laplacian on each plane,
// plus the second difference along z on 3-D grids (seven points)
void lap(const rdo_problem& pb, const double* x, double* out) {
  const int nx = pb.nx, ny = pb.ny, nz = nzof(pb);
  const double hx2 = 1.0 / ((pb.lx / nx) * (pb.lx / nx)), hy2 = 1.0 / ((pb.ly / ny) * (pb.ly / ny));
  const double hz2 = nz > 1 ? 1.0 / ((pb.lz / nz) * (pb.lz / nz)) : 0.0;
  const size_t plane = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
  for (int r = 0; r < nz * ny; ++r) {
    const int l = r / ny, i = r - l * ny;
    const int im = nb(i, -1, ny, pb.bc), ip = nb(i, 1, ny, pb.bc);
    const int lm = nz > 1 ? nb(l, -1, nz, pb.bc) : l, lp = nz > 1 ? nb(l, 1, nz, pb.bc) : l;
    const double* xp = x + l * plane;
    for (int j = 0; j < nx; ++j) {
      const int jm = nb(j, -1, nx, pb.bc), jp = nb(j, 1, nx, pb.bc);
      const double c = xp[(size_t)i * nx + j];
      double v = (xp[(size_t)i * nx + jp] + xp[(size_t)i * nx + jm] - 2.0 * c) * hx2 +
                 (xp[(size_t)ip * nx + j] + xp[(size_t)im * nx + j] - 2.0 * c) * hy2;
      if (nz > 1) v += (x[lp * plane + (size_t)i * nx + j] + x[lm * plane + (size_t)i * nx + j] - 2.0 * c) * hz2;
      out[l * plane + (size_t)i * nx + j] = v;
    }
  }
}

using vec = std::vector<double>;

vec lapv(const rdo_problem& pb, const double* x) {
  vec o(npts_of(pb));
  lap(pb, x, o.data());
  return o;
}

// ------------------------------------------------------------------------------------------
// the residual map F and its adjoint Jacobian
// ------------------------------------------------------------------------------------------

// Sixth-order equation (Section 3.3): mu(U) = a Lap U - b W'(U), A(U) x = a Lap x - b W''(U) x + a x
vec fch_mu(const rdo_problem& pb, const double* U) {
  const size_t n = npts_of(pb);
  vec L = lapv(pb, U), m(n);
  for (size_t q = 0; q < n; ++q) m[q] = pb.a * L[q] - pb.b * (U[q] * U[q] * U[q] - U[q]);
  return m;
}

vec fch_A(const rdo_problem& pb, const double* U, const double* x) {
  const size_t n = npts_of(pb);
  vec L = lapv(pb, x), o(n);
  for (size_t q = 0; q < n; ++q) o[q] = pb.a * L[q] - pb.b * (3.0 * U[q] * U[q] - 1.0) * x[q] + pb.a * x[q];
  return o;
}

// W = F(U) for U^k = Uk; arrays component-major [ncomp][ny][nx]
void residual(const rdo_problem& pb, const double* U, const double* Uk, double* W) {
  const size_t n = npts_of(pb);
  const double dt = pb.dt, a = pb.a, b = pb.b;
  switch (pb.kind) {
    case K_NONE: {
      vec L = lapv(pb, U);
      if (pb.op == OP_LAPLACIAN) {                                  // (I - a dt Lap) U - U^k
        for (size_t q = 0; q < n; ++q) W[q] = U[q] - Uk[q] - dt * a * L[q];
      } else {                                                      // (I + a dt Lap^2) U - U^k
        vec LL = lapv(pb, L.data());
        for (size_t q = 0; q < n; ++q) W[q] = U[q] + dt * a * LL[q] - Uk[q];
      }
      return;
    }
    case K_AC: {                                                    // U - U^k - dt (a Lap U + f(U)), f = -b W'
      vec L = lapv(pb, U);
      for (size_t q = 0; q < n; ++q) {
        const double f = -b * (U[q] * U[q] * U[q] - U[q]);
        W[q] = U[q] - Uk[q] - dt * (a * L[q] + f);
      }
      return;
    }
    case K_CH_IMPLICIT:
    case K_CH_SPLIT: {
      // implicit: (I + a dt Lap^2) U - U^k - b dt Lap (U^3 - U)
      // split   : (I + a dt Lap^2) U - U^k - b dt Lap U^3 + b dt Lap U^k
      vec L = lapv(pb, U), LL = lapv(pb, L.data()), c(n);
      const bool impl = pb.kind == K_CH_IMPLICIT;
      for (size_t q = 0; q < n; ++q) c[q] = U[q] * U[q] * U[q] - (impl ? U[q] : 0.0);
      vec Lc = lapv(pb, c.data());
      vec Lk;
      if (!impl) Lk = lapv(pb, Uk);
      for (size_t q = 0; q < n; ++q) {
        W[q] = U[q] + dt * a * LL[q] - Uk[q] - dt * b * Lc[q];
        if (!impl) W[q] += dt * b * Lk[q];
      }
      return;
    }
    case K_GRAY_SCOTT: {                                            // two species, standard form
      const double Du = pb.p[0], Dv = pb.p[1], F = pb.p[2], k = pb.p[3];
      const double *u = U, *v = U + n;
      vec Lu = lapv(pb, u), Lv = lapv(pb, v);
      for (size_t q = 0; q < n; ++q) {
        const double uvv = u[q] * v[q] * v[q];
        W[q] = u[q] - Uk[q] - dt * (Du * Lu[q] - uvv + F * (1.0 - u[q]));
        W[n + q] = v[q] - Uk[n + q] - dt * (Dv * Lv[q] + uvv - (F + k) * v[q]);
      }
      return;
    }
    case K_SCHNAKENBERG: {                                          // Section 3.4.1, F_u and F_v
      const double D1 = pb.p[0], D2 = pb.p[1], kap = pb.p[2], as = pb.p[3], bs = pb.p[4];
      const double *u = U, *v = U + n;
      vec Lu = lapv(pb, u), Lv = lapv(pb, v);
      for (size_t q = 0; q < n; ++q) {
        const double u2v = u[q] * u[q] * v[q];
        W[q] = u[q] - Uk[q] - dt * (D1 * Lu[q] + kap * (as - u[q] + u2v));
        W[n + q] = v[q] - Uk[n + q] - dt * (D2 * Lv[q] + kap * (bs - u2v));
      }
      return;
    }
    case K_FCH: {                                                   // U - U^k - dt Lap A(U) mu(U)
      vec m = fch_mu(pb, U);
      vec Am = fch_A(pb, U, m.data());
      vec L = lapv(pb, Am.data());
      for (size_t q = 0; q < n; ++q) W[q] = U[q] - Uk[q] - dt * L[q];
      return;
    }
  }
}

// g = dF(U)^T Pt (the derivative taken at the current iterate U_n)
void grad_F_T(const rdo_problem& pb, const double* U, const double* Pt, double* g) {
  const size_t n = npts_of(pb);
  const double dt = pb.dt, a = pb.a, b = pb.b;
  switch (pb.kind) {
    case K_NONE: {
      vec L = lapv(pb, Pt);
      if (pb.op == OP_LAPLACIAN) {
        for (size_t q = 0; q < n; ++q) g[q] = Pt[q] - dt * a * L[q];
      } else {
        vec LL = lapv(pb, L.data());
        for (size_t q = 0; q < n; ++q) g[q] = Pt[q] + dt * a * LL[q];
      }
      return;
    }
    case K_AC: {                                                    // Pt - dt a Lap Pt - dt f'(U) Pt
      vec L = lapv(pb, Pt);
      for (size_t q = 0; q < n; ++q) {
        const double fp = -b * (3.0 * U[q] * U[q] - 1.0);
        g[q] = Pt[q] - dt * a * L[q] - dt * fp * Pt[q];
      }
      return;
    }
    case K_CH_IMPLICIT:
    case K_CH_SPLIT: {                                              // (I + a dt Lap^2) Pt - b dt W''(U) Lap Pt
      vec L = lapv(pb, Pt), LL = lapv(pb, L.data());
      const double sh = pb.kind == K_CH_IMPLICIT ? 1.0 : 0.0;
      for (size_t q = 0; q < n; ++q) g[q] = Pt[q] + dt * a * LL[q] - dt * b * (3.0 * U[q] * U[q] - sh) * L[q];
      return;
    }
    case K_GRAY_SCOTT: {
      const double Du = pb.p[0], Dv = pb.p[1], F = pb.p[2], k = pb.p[3];
      const double *u = U, *v = U + n, *P = Pt, *Q = Pt + n;
      vec LP = lapv(pb, P), LQ = lapv(pb, Q);
      for (size_t q = 0; q < n; ++q) {
        g[q] = P[q] - dt * Du * LP[q] + dt * (v[q] * v[q] + F) * P[q] - dt * v[q] * v[q] * Q[q];
        g[n + q] = Q[q] - dt * Dv * LQ[q] + 2.0 * dt * u[q] * v[q] * P[q] - dt * (2.0 * u[q] * v[q] - (F + k)) * Q[q];
      }
      return;
    }
    case K_SCHNAKENBERG: {                                          // Section 3.4.1 U and V updates
      const double D1 = pb.p[0], D2 = pb.p[1], kap = pb.p[2];
      const double *u = U, *v = U + n, *P = Pt, *Q = Pt + n;
      vec LP = lapv(pb, P), LQ = lapv(pb, Q);
      for (size_t q = 0; q < n; ++q) {
        g[q] = P[q] - dt * (D1 * LP[q] + kap * (-P[q] + 2.0 * u[q] * v[q] * (P[q] - Q[q])));
        g[n + q] = Q[q] - dt * (D2 * LQ[q] + kap * (u[q] * u[q] * (P[q] - Q[q])));
      }
      return;
    }
    case K_FCH: {
      // dF^T P = P - dt B A Lap P + dt b mu W'''(U) Lap P, B = a Lap - b W''(U)
      vec qv = lapv(pb, Pt);
      vec r = fch_A(pb, U, qv.data());
      vec Lr = lapv(pb, r.data());
      vec m = fch_mu(pb, U);
      for (size_t q = 0; q < n; ++q) {
        const double s = a * Lr[q] - b * (3.0 * U[q] * U[q] - 1.0) * r[q];
        g[q] = Pt[q] - dt * s + dt * b * m[q] * (6.0 * U[q]) * qv[q];
      }
      return;
    }
  }
}

// ------------------------------------------------------------------------------------------
// transforms
// ------------------------------------------------------------------------------------------

// In-place unnormalised radix-2 complex DFT of length n (a power of two):
// X_k = sum_j x_j exp(sgn 2 pi i j k / n), sgn = -1 forward, +1 inverse.
void fft(cplx* x, int n, int sgn) {
  for (int i = 1, j = 0; i < n; ++i) {  // bit-reversal permutation
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1;
    for (int k = 0; k < half; ++k) {
      const double ang = sgn * 2.0 * kPi * k / len;
      const cplx w(std::cos(ang), std::sin(ang));
      for (int s = 0; s < n; s += len) {
        const cplx t = w * x[s + k + half];
        x[s + k + half] = x[s + k] - t;
        x[s + k] += t;
      }
    }
  }
}

// Orthonormal DCT-II of x (length n) into X, through the 2n-point FFT V of the even extension:
// V_k = 2 exp(i pi k / 2n) C_k with C_k = sum_j x_j cos(pi k (2j + 1) / 2n).
void dct2(const double* x, double* X, int n, std::vector<cplx>& buf) {
  buf.assign(2 * n, cplx(0, 0));
  for (int j = 0; j < n; ++j) {
    buf[j] = x[j];
    buf[2 * n - 1 - j] = x[j];
  }
  fft(buf.data(), 2 * n, -1);
  for (int k = 0; k < n; ++k) {
    const double ph = -kPi * k / (2.0 * n);
    const double C = 0.5 * (buf[k] * cplx(std::cos(ph), std::sin(ph))).real();
    X[k] = C * (k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n));
  }
}

// Orthonormal DCT-III (the inverse of dct2): x_j = sum_k s_k X_k cos(pi k (2j + 1) / 2n), through
// the 2n-point inverse FFT of Z_k = s_k X_k exp(i pi k / 2n) (Z_0 doubled, Z_n = 0, Z_{2n-k} = conj
// Z_k): its real part is 2 x_j for j < n.
void dct3(const double* X, double* x, int n, std::vector<cplx>& buf) {
  buf.assign(2 * n, cplx(0, 0));
  for (int k = 0; k < n; ++k) {
    const double s = k == 0 ? 2.0 * std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    const double ph = kPi * k / (2.0 * n);
    buf[k] = s * X[k] * cplx(std::cos(ph), std::sin(ph));
    if (k > 0) buf[2 * n - k] = std::conj(buf[k]);
  }
  fft(buf.data(), 2 * n, +1);
  for (int j = 0; j < n; ++j) x[j] = 0.5 * buf[j].real();
}

// eigenvalues mu >= 0 of -Lap on the transform grid (row-major [nz][ny][nx]):
//   periodic  4/h_x^2 sin^2(pi kx / nx) + 4/h_y^2 sin^2(pi ky / ny) [+ 4/h_z^2 sin^2(pi kz / nz)]
//   Neumann   4/h_x^2 sin^2(pi kx / 2nx) + 4/h_y^2 sin^2(pi ky / 2ny) [+ 4/h_z^2 sin^2(pi kz / 2nz)]
// (Fourier modes, resp. DCT-II modes; the z term on 3-D grids only)
vec symbol_mu(const rdo_problem& pb) {
  const int nx = pb.nx, ny = pb.ny, nz = nzof(pb);
  const double hx = pb.lx / nx, hy = pb.ly / ny, d = pb.bc == BC_PERIODIC ? 1.0 : 2.0;
  const double hz = nz > 1 ? pb.lz / nz : 1.0;
  vec mu(npts_of(pb));
  for (int l = 0; l < nz; ++l)
    for (int i = 0; i < ny; ++i)
      for (int j = 0; j < nx; ++j) {
        const double sx = std::sin(kPi * j / (d * nx)), sy = std::sin(kPi * i / (d * ny));
        double m = 4.0 / (hx * hx) * sx * sx + 4.0 / (hy * hy) * sy * sy;
        if (nz > 1) {
          const double sz = std::sin(kPi * l / (d * nz));
          m += 4.0 / (hz * hz) * sz * sz;
        }
        mu[((size_t)l * ny + i) * nx + j] = m;
      }
  return mu;
}

// eigenvalues of G = A_lin^2 per component
vec ghat(const rdo_problem& pb) {
  const int nc = ncomp_of(pb);
  const size_t n = npts_of(pb);
  vec g(nc * n, 1.0);
  if (pb.precond == PC_NONE) return g;
  vec mu = symbol_mu(pb);
  const double dt = pb.dt;
  for (int c = 0; c < nc; ++c)
    for (size_t q = 0; q < n; ++q) {
      const double m = mu[q];
      double r;
      const bool stab = pb.precond == PC_STABILIZED;
      const double s = pb.shift;
      if (nc == 2) r = 1.0 + pb.p[c] * dt * m;                                          // (I - D dt Lap)
      else if (pb.op == OP_LAPLACIAN) r = 1.0 + (stab ? pb.b * dt * s : 0.0) + pb.a * dt * m;  // ((1 + b dt s) I - a dt Lap)
      else if (pb.op == OP_FUNCTIONALIZED)
        r = 1.0 + dt * pb.a * m * m * (pb.a * m + (stab ? s : 2.0) * pb.b - pb.a);
      else r = 1.0 + (stab ? pb.b * s * dt * m : 0.0) + pb.a * dt * m * m;             // (I + a dt Lap^2 - b s dt Lap)
      g[c * n + q] = r * r;
    }
  return g;
}

// Apply fn(line) to every line of length len and element stride `stride` of an array of n
// values (the lines along one axis); fn gets the line's first index.
template <class Fn>
void for_lines(size_t n, int len, size_t stride, Fn fn) {
  const size_t block = (size_t)len * stride, nlines = n / len;
#pragma omp parallel for schedule(static)
  for (long long m = 0; m < (long long)nlines; ++m) {
    const size_t outer = (size_t)m / stride, inner = (size_t)m % stride;
    fn(outer * block + inner);
  }
}

// Y = G^{-1} W on one component: FFT along every axis (periodic) or orthonormal DCT-II along every
// axis (Neumann), divide by g, inverse transforms
void ginv_component(const rdo_problem& pb, const double* W, const double* g, double* Y) {
  const int nx = pb.nx, ny = pb.ny, nz = nzof(pb);
  const size_t n = npts_of(pb);
  const int len[3] = {nx, ny, nz};
  const size_t str[3] = {1, (size_t)nx, (size_t)nx * ny};
  const int naxes = nz > 1 ? 3 : 2;
  if (pb.bc == BC_PERIODIC) {
    std::vector<cplx> z(n);
    for (size_t q = 0; q < n; ++q) z[q] = W[q];
    auto pass = [&](int ax, int sgn) {
      for_lines(n, len[ax], str[ax], [&](size_t q0) {
        std::vector<cplx> line(len[ax]);
        for (int t = 0; t < len[ax]; ++t) line[t] = z[q0 + t * str[ax]];
        fft(line.data(), len[ax], sgn);
        for (int t = 0; t < len[ax]; ++t) z[q0 + t * str[ax]] = line[t];
      });
    };
    for (int ax = 0; ax < naxes; ++ax) pass(ax, -1);
    for (size_t q = 0; q < n; ++q) z[q] /= g[q];
    for (int ax = naxes - 1; ax >= 0; --ax) pass(ax, +1);
    for (size_t q = 0; q < n; ++q) Y[q] = z[q].real() / (double)n;
    return;
  }
  vec t(W, W + n);
  auto pass = [&](int ax, bool fwd) {
    for_lines(n, len[ax], str[ax], [&](size_t q0) {
      std::vector<cplx> buf;
      vec a(len[ax]), b(len[ax]);
      for (int k = 0; k < len[ax]; ++k) a[k] = t[q0 + k * str[ax]];
      if (fwd) dct2(a.data(), b.data(), len[ax], buf);
      else dct3(a.data(), b.data(), len[ax], buf);
      for (int k = 0; k < len[ax]; ++k) t[q0 + k * str[ax]] = b[k];
    });
  };
  for (int ax = 0; ax < naxes; ++ax) pass(ax, true);
  for (size_t q = 0; q < n; ++q) t[q] /= g[q];
  for (int ax = naxes - 1; ax >= 0; --ax) pass(ax, false);
  std::memcpy(Y, t.data(), n * sizeof(double));
}

void apply_ginv(const rdo_problem& pb, const double* W, const vec& g, double* Y) {
  const int nc = ncomp_of(pb);
  const size_t n = npts_of(pb);
  if (pb.precond == PC_NONE) {
    std::memcpy(Y, W, nc * n * sizeof(double));
    return;
  }
  for (int c = 0; c < nc; ++c) ginv_component(pb, W + c * n, g.data() + c * n, Y + c * n);
}

// sum of squares of one component, as row partials summed in row order
double sumsq(const rdo_problem& pb, const double* x) {
  const int nx = pb.nx, nrows = pb.ny * nzof(pb);
  vec rows(nrows);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int j = 0; j < nx; ++j) s += x[(size_t)i * nx + j] * x[(size_t)i * nx + j];
    rows[i] = s;
  }
  double s = 0.0;
  for (int i = 0; i < nrows; ++i) s += rows[i];
  return s;
}

// the stopping measure (sum of the components' l2 norms of F, over dt for RD_TOL_RES_ABS) and its
// threshold (delta, or tol ||U^k||_2)
void measure(const rdo_problem& pb, const double* W, const double* Uk, double* r, double* thr) {
  const int nc = ncomp_of(pb);
  const size_t n = npts_of(pb);
  double s = 0.0, uk2 = 0.0;
  for (int c = 0; c < nc; ++c) {
    s += std::sqrt(sumsq(pb, W + c * n));
    uk2 += sumsq(pb, Uk + c * n);
  }
  if (pb.tol_kind == TOL_RES_ABS) {
    *r = s / pb.dt;
    *thr = pb.tol;
  } else {
    *r = s;
    *thr = pb.tol * std::sqrt(uk2);
  }
}

}  // namespace

extern "C" {

// Number of OpenMP threads the oracle uses (n <= 0: one per processor; 1 when built without
// OpenMP); returns the number set.
int rdo_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void rdo_residual(const rdo_problem* pb, const double* U, const double* Uk, double* W) { residual(*pb, U, Uk, W); }

void rdo_grad_F_T(const rdo_problem* pb, const double* U, const double* Pt, double* g) { grad_F_T(*pb, U, Pt, g); }

void rdo_apply_ginv(const rdo_problem* pb, const double* W, double* Y) { apply_ginv(*pb, W, ghat(*pb), Y); }

void rdo_ghat(const rdo_problem* pb, double* g) {
  vec v = ghat(*pb);
  std::memcpy(g, v.data(), v.size() * sizeof(double));
}

// Testing hooks of the transforms: complex DFT (sgn -1 / +1, unnormalised, n a power of two) of
// n interleaved (re, im) pairs in place, and the orthonormal DCT-II / DCT-III of n reals.
void rdo_fft(double* x, int n, int sgn) { fft(reinterpret_cast<cplx*>(x), n, sgn); }
void rdo_dct2(const double* x, double* X, int n) {
  std::vector<cplx> buf;
  dct2(x, X, n, buf);
}
void rdo_dct3(const double* X, double* x, int n) {
  std::vector<cplx> buf;
  dct3(X, x, n, buf);
}

// One implicit step by G-prox PDHG from U^k = Uk (Algorithm 1 inner loop):
//   W = F(U_n); r = measure; stop if r <= threshold (ties stop); DIVERGED if r is not finite or
//   > 1e8 r_0; NOT_CONVERGED after max_iter updates; else Y = G^{-1} W,
//   Pt = P + (1 + omega) tau_p Y, P += tau_p Y, U -= tau_u dF(U_n)^T Pt.
// U (out) receives the stopping iterate; *iterations the number of updates; *status ST_*;
// *residual the last measure; history (may be NULL) the first hist_cap measures.
void rdo_pdhg_step(const rdo_problem* pbp, const double* Uk, double* U, int* iterations, int* status,
                   double* residual_out, double* history, int hist_cap) {
  const rdo_problem& pb = *pbp;
  const size_t N = (size_t)ncomp_of(pb) * npts_of(pb);
  std::memcpy(U, Uk, N * sizeof(double));                 // U_0 = U^k
  vec P(N, 0.0), W(N), Y(N), Pt(N), g(N);                 // P_0 = 0
  const vec gh = ghat(pb);
  double r0 = 0.0, r = 0.0, thr = 0.0;
  int n = 0, st = ST_OK;
  while (true) {
    residual(pb, U, Uk, W.data());                        // W_n = F(U_n)
    measure(pb, W.data(), Uk, &r, &thr);
    if (history && n < hist_cap) history[n] = r;
    if (n == 0) r0 = r;
    if (r <= thr) { st = ST_OK; break; }
    if (!std::isfinite(r) || r > kDivergeFactor * r0) { st = ST_DIVERGED; break; }
    if (n == pb.max_iter) { st = ST_NOT_CONVERGED; break; }
    apply_ginv(pb, W.data(), gh, Y.data());               // G Y = W
    for (size_t q = 0; q < N; ++q) {
      Pt[q] = P[q] + (1.0 + pb.omega) * pb.tau_p * Y[q];  // P~ = P_{n+1} + omega (P_{n+1} - P_n)
      P[q] = P[q] + pb.tau_p * Y[q];                      // P_{n+1} = P_n + tau_p G^{-1} F(U_n)
    }
    grad_F_T(pb, U, Pt.data(), g.data());                 // dF(U_n)^T P~
    for (size_t q = 0; q < N; ++q) U[q] -= pb.tau_u * g[q];  // U_{n+1} = U_n - tau_u dF^T P~
    ++n;
  }
  *iterations = n;
  *status = st;
  *residual_out = r;
}

}  // extern "C"
